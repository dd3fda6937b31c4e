#!/usr/bin/env python
"""Benchmark of the RAK label-propagation path on GB300.

One step = the whole hot path on one graph already resident in HBM:
ingest (validation + degree bucketing of a borrowed device CSR), RAK to
convergence, modularity of the result.  ``value`` = CSR entries traversed per
second over the timed steps (GTEPS: iterations x m / step time), timed with
CUDA events on the stream the library launches on.

Workloads (synthetic stand-ins for the paper's SuiteSparse classes):
  rmat22    R-MAT scale 22, edge factor 16, weights 1-4, asynchronous (default)
  rmat21    the same at scale 21 (profiling size)
  road4096  4096 x 4096 road-like grid, weights 1-16 (sync or async)
  sbm10k    planted partition, 10,000 vertices, synchronous
  kmer8m    k-mer-like chains, 8M vertices

Extra keys: ``roofline`` (dominant sweep kernel vs measured HBM bandwidth),
``sweep`` (all sweep kernels of one iteration vs the same peak), ``e2e``
(the same metric through the C ABI from pinned host buffers, copies timed),
``cpu_baseline`` (the CPU oracle on a bounded sample), ``clocks``
(nvidia-smi samples during the timed region), ``gpu_launches``.

``--impl reference`` times the CPU oracle (the only reference this method
has: the paper publishes no code) on the same workload and metric.
Multi-GPU (torchrun): every rank runs its own replica of the workload;
``value`` = entries traversed by all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 129 * 2**20

WORKLOADS = {
    "rmat22": dict(mode="async", waves=2, strict=True, tolerance=0.05, max_iter=20),
    "rmat21": dict(mode="async", waves=2, strict=True, tolerance=0.05, max_iter=20),
    "road4096": dict(mode="async", waves=31, strict=True, tolerance=0.05, max_iter=20),
    "sbm10k": dict(mode="sync", waves=31, strict=True, tolerance=0.05, max_iter=20),
    "kmer8m": dict(mode="async", waves=31, strict=True, tolerance=0.05, max_iter=20),
}


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat22")
    ap.add_argument("--mode", choices=["sync", "async"], default=None)
    ap.add_argument("--waves", type=int, default=None)
    ap.add_argument("--non-strict", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--cpu-sweeps", type=int, default=4,
                    help="oracle sweeps in the CPU baseline sample")
    return ap.parse_args()


def workload_params(args):
    p = dict(WORKLOADS[args.workload])
    if args.mode:
        p["mode"] = args.mode
    if args.waves:
        p["waves"] = args.waves
    if args.non_strict:
        p["strict"] = False
    return p


def measured_peak_gbs():
    try:
        with open(PEAKS_FILE) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id, enabled=True):
        self.proc = None
        self.path = None
        if not enabled:
            return
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_id}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def nvsmi_id(torch, local):
    """nvidia-smi id of this rank's GPU (UUID when torch reports it)."""
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[local] if vis else str(local)


def reduce_across_ranks(t_ms, entries, device=None):
    """(max of t_ms, sum of entries) over the ranks of the default process
    group; the identity without one."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t_ms), float(entries)
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    e = torch.tensor([float(entries)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def gen_graph(name):
    import graphgen as gg

    return gg.workload(name)


def alg_bytes_per_sweep(g):
    """Algorithmic HBM bytes of one sweep over the whole graph: row pointer,
    own label read and label write per non-isolated vertex, column index (and
    weight) per entry."""
    deg = np.diff(g.offsets)
    nz = int(np.count_nonzero(deg))
    return 12 * nz + (8 if g.weights is not None else 4) * g.m


# --------------------------------------------------------------------------
# reference arm: the CPU oracle
# --------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    p = workload_params(args)
    g = gen_graph(args.workload)
    oracle.build()
    mode = p["mode"]
    waves = p["waves"] if mode == "async" else 0
    # one step = `sweeps` oracle sweeps from unique labels (bounded sample)
    sweeps = max(1, args.cpu_sweeps // 2)

    def step():
        t0 = time.perf_counter()
        _, it, _, _ = oracle.rak(g.offsets, g.indices, g.weights, 0.0, sweeps, mode,
                                 strict=p["strict"], waves=waves)
        return it, time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    tot_it, tot_t = 0, 0.0
    for _ in range(args.steps):
        it, t = step()
        tot_it += it
        tot_t += t
    value = tot_it * g.m / tot_t / 1e9
    line = {
        "impl": "reference", "metric": f"RAK GTEPS ({args.workload})", "value": value,
        "unit": "GTEPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "n": g.n, "m": g.m, **p},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                         "sample": f"{sweeps} {mode} sweeps of the full graph per step"},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(g, p, sweeps):
    import oracle

    oracle.build()
    mode = p["mode"]
    waves = p["waves"] if mode == "async" else 0
    t0 = time.perf_counter()
    _, it, _, _ = oracle.rak(g.offsets, g.indices, g.weights, 0.0, sweeps, mode,
                             strict=p["strict"], waves=waves)
    t = time.perf_counter() - t0
    return {"value": it * g.m / t / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{it} {mode} sweeps of the full {g.n}-vertex graph from unique labels "
                      f"({t:.1f} s, single thread)"}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args):
    import torch

    import paper_2301_09125_gb300 as lp
    from paper_2301_09125_gb300 import build

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    build.build()
    lp.load()

    p = workload_params(args)
    g = gen_graph(args.workload)
    stream = torch.cuda.current_stream(dev)
    off = torch.from_numpy(g.offsets).to(dev)
    idx = torch.from_numpy(g.indices).to(dev)
    w = None if g.weights is None else torch.from_numpy(g.weights).to(dev)
    params, _ = lp.make_params(tolerance=p["tolerance"], max_iter=p["max_iter"], mode=p["mode"],
                               strict=p["strict"], waves=p["waves"])
    torch.cuda.synchronize()

    def step():
        h = lp.lp_graph_create(off, idx, w, borrow=True, stream=stream.cuda_stream)
        r = lp.lp_rak_run(h, params)
        q = lp.lp_modularity(h)
        lp.lp_graph_destroy(h)
        return r, q

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(nvsmi_id(torch, local), enabled=not args.no_clocks)
    lp.lp_profile_reset()
    lp.lp_profile_enable(True)
    launches0 = lp.lp_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    iters, qs, run_ms = [], [], []
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        r, q = step()
        iters.append(r.iterations)
        qs.append(q)
        run_ms.append(r.gpu_ms)
    e1.record(stream)
    barrier()
    launches = lp.lp_launch_count() - launches0
    lp.lp_profile_enable(False)
    prof = lp.lp_profile_read()
    clock_info = clocks.stop()
    t_ms = e0.elapsed_time(e1)

    t_ms, entries_all = reduce_across_ranks(t_ms, sum(iters) * g.m, device=dev)

    value = entries_all / (t_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak_gbs()

    # dominant sweep kernel: the largest share of profiled sweep time
    kern = {k: v for k, v in prof.items() if v["launches"] > 0}
    dom_name = max(kern, key=lambda k: kern[k]["total_ms"])
    dom = kern[dom_name]
    achieved = dom["bytes"] / (dom["total_ms"] * 1e-3) / 1e9
    sweep_ms = sum(v["total_ms"] for v in kern.values())
    total_sweeps = sum(iters)
    sweep_bytes = alg_bytes_per_sweep(g)
    per_sweep_ms = sweep_ms / total_sweeps
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom_name,
                "peak_source": peak_kind}
    line = {
        "metric": f"RAK GTEPS ({args.workload})", "value": value, "unit": "GTEPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "n": g.n, "m": g.m, **p,
                   "iterations_per_step": statistics.mean(iters),
                   "modularity": statistics.mean(qs),
                   "step": "ingest (validate + bucket, borrowed device CSR) + RAK to "
                           "convergence + modularity",
                   "l2": ("inputs larger than L2" if g.offsets.nbytes + g.indices.nbytes +
                          (0 if g.weights is None else g.weights.nbytes) > L2_BYTES
                          else "inputs smaller than L2, no flush"),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "sweep": {"ms_per_sweep": per_sweep_ms, "gteps": g.m / (per_sweep_ms * 1e-3) / 1e9,
                  "alg_bytes": sweep_bytes,
                  "hbm_frac": sweep_bytes / (per_sweep_ms * 1e-3) / 1e9 / peak,
                  "run_ms_per_step": statistics.mean(run_ms)},
        "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"],
                        "share": v["total_ms"] / sweep_ms,
                        "gbs": v["bytes"] / (v["total_ms"] * 1e-3) / 1e9}
                    for k, v in kern.items()},
        "gpu_launches": int(launches),
        "clocks": clock_info,
    }

    # end to end through the C ABI from pinned host buffers
    if not args.no_e2e:
        hoff = torch.from_numpy(g.offsets).pin_memory()
        hidx = torch.from_numpy(g.indices).pin_memory()
        hw = None if g.weights is None else torch.from_numpy(g.weights).pin_memory()
        hlab = torch.empty(g.n, dtype=torch.int32).pin_memory()

        def e2e_step():
            h = lp.lp_graph_create(hoff, hidx, hw, stream=stream.cuda_stream)
            r = lp.lp_rak_run(h, params)
            lp.lp_modularity(h)
            lp.lp_labels_get(h, hlab)
            lp.lp_graph_destroy(h)
            return r.iterations

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        e_iters = [e2e_step() for _ in range(args.steps)]
        barrier()
        t = time.perf_counter() - t0
        h2d = g.offsets.nbytes + g.indices.nbytes + (0 if g.weights is None else g.weights.nbytes)
        line["e2e"] = {"value": sum(e_iters) * g.m * world / t / 1e9, "unit": "GTEPS",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(g.n * 4 + 8)}

    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, p, args.cpu_sweeps)

    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
