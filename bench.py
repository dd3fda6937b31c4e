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
  batch     4096 planted-partition graphs (n log-uniform 1k-200k, 5-500 blocks,
            mean degree 8-32, mixing 0.3) in one arena, synchronous; metric
            graphs/s, compared with the same graphs run one at a time
  serve     Poisson request stream (mean 200 req/s, 60 s) of SBM / R-MAT /
            grid graphs (n log-uniform 10k-2M, weights 1-8) drawn from a pool
            of 96 distinct graphs, served with continuous batching; graphs/s
            and p50/p99 latency, compared with the same arrivals served one
            graph at a time

The default run (rmat22) also measures the batched and served configurations
and adds them as the ``batch`` and ``serve`` sub-records (``--no-batch`` /
``--no-serve`` leave them out).

Extra keys: ``roofline`` (dominant sweep kernel vs measured HBM bandwidth),
``sweep`` (all sweep kernels of one iteration vs the same peak), ``e2e``
(the same metric through the C ABI from pinned host buffers, copies timed),
``cpu_baseline`` (the CPU oracle on a bounded sample), ``clocks``
(nvidia-smi samples during the timed region), ``gpu_launches``.

``--impl reference`` times the CPU oracle (the only reference this method
has: the paper publishes no code) on the same workload and metric.

``--experiment tolerance`` runs the paper's tolerance / tie-rule study
(Sec. 3.2) on the synthetic classes instead: tolerance 0.1 down to 0.0001,
strict and non-strict ties, synchronous and asynchronous updates, each with
and without a self-loop on every vertex (Sec. 3.1), max_iter 100.  It prints
one JSON line per setting (iterations, convergence, run time, GTEPS,
modularity of the labels on the graph without self-loops).
``--experiment split`` times the split of disconnected communities after
each class's benchmark run (communities and modularity before and after).
``--experiment copra`` / ``--experiment slpa`` time COPRA (Sec. 3.3, 4 labels,
tolerance 0.01) and SLPA (Sec. 3.4, memory of 20) on each class, with their
first iteration checked against the oracle at full size.
``--experiment noalloc`` times the allocation-free sweep against lp_rak_run's.
``--experiment gather`` measures the ceiling of a label-gathering sweep: one
pass streaming the rows, and one that also gathers every entry's neighbour
label, on each class as generated and renumbered by decreasing degree.
Multi-GPU (torchrun): on a single graph every rank runs its own replica;
the batch and the serving stream shard whole graphs over the ranks
(size-balanced; requests r, r + N, ... to rank r) with no collective on the
data path, and per-graph results are gathered on rank 0.  ``value`` = the
work of all ranks / the slowest rank's time.
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
    # waves coprime with the grid width (4096): vertical neighbours fall in
    # different waves; modularity within 0.006 of the sequential order
    "road4096": dict(mode="async", waves=3, strict=True, tolerance=0.05, max_iter=20),
    "sbm10k": dict(mode="sync", waves=31, strict=True, tolerance=0.05, max_iter=20),
    # path neighbours have random ids: enough waves that few fall in one wave
    # (modularity within 0.008 of the sequential order from 127 waves on)
    "kmer8m": dict(mode="async", waves=127, strict=True, tolerance=0.05, max_iter=20),
    "batch": dict(mode="sync", waves=31, strict=True, tolerance=0.05, max_iter=20),
    "serve": dict(mode="sync", waves=31, strict=True, tolerance=0.05, max_iter=20),
}


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
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
    ap.add_argument("--batch-count", type=int, default=4096, help="graphs of the batch workload")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="arrival window (serve)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="mean arrivals per second")
    ap.add_argument("--serve-saturation", type=int, default=512,
                    help="requests of the burst that measures service capacity")
    ap.add_argument("--serve-pool", type=int, default=96, help="distinct graphs in the pool")
    ap.add_argument("--serve-cohort", type=int, default=None,
                    help="requests iterated together in one batch (server default if unset)")
    ap.add_argument("--serve-admitters", type=int, default=None,
                    help="ingest threads of the server (server default if unset)")
    ap.add_argument("--serve-cohort-entries", type=int, default=None,
                    help="largest graph (CSR entries) that joins a cohort")
    ap.add_argument("--serve-baseline-seconds", type=float, default=10.0,
                    help="arrival window replayed one graph at a time")
    ap.add_argument("--no-batch", action="store_true",
                    help="single-graph workloads: leave out the batch sub-record")
    ap.add_argument("--no-serve", action="store_true",
                    help="single-graph workloads: leave out the serve sub-record")
    ap.add_argument("--per-graph-sample", type=int, default=256,
                    help="graphs of the batch timed one at a time")
    ap.add_argument("--experiment",
                    choices=["tolerance", "split", "gather", "copra", "slpa", "noalloc"],
                    default=None,
                    help="run the tolerance / tie-rule study, or time the split of "
                         "disconnected communities, instead of the benchmark")
    ap.add_argument("--classes", default="sbm10k,rmat22,road4096,kmer8m",
                    help="workloads of the study (comma-separated)")
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
                 "--format=csv,noheader,nounits", "-lms", "20"],
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


def shard_graphs(sizes, rank, world):
    """Indices of the graphs rank `rank` of `world` takes: whole graphs, in
    decreasing size each to the rank with the least work so far (ties to the
    lowest rank), listed in increasing index order."""
    load = [0] * world
    mine = []
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += sizes[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def gather_results(local, world):
    """Per-graph results of every rank merged into one dict (index -> result),
    on every rank; the identity without a process group."""
    if world == 1:
        return dict(local)
    import torch.distributed as dist

    parts = [None] * world
    dist.all_gather_object(parts, dict(local))
    merged = {}
    for part in parts:
        for k, v in part.items():
            assert k not in merged, f"graph {k} was run on two ranks"
            merged[k] = v
    return merged


def code_lines(text):
    """The lines of a C/CUDA source without its // comments and blank lines
    (what the compiler sees, up to whitespace at the line ends)."""
    out = []
    for line in text.splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code.strip():
            out.append(code)
    return "\n".join(out)


def sweep_sources_hash():
    """First 16 hex digits of the SHA-256 of the sweep kernel sources' code
    (comments and blank lines left out, so a comment edit keeps the hash)."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2301_09125_gb300",
                        "csrc")
    for f in ("lp_sweep.cu", "lp_device.cuh", "lp_internal.cuh"):
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(code_lines(fh.read()).encode())
    return h.hexdigest()[:16]


def traffic_ratio(kernel):
    """DRAM traffic / algorithmic bytes of a bucket launch from the committed
    ncu summary, or None when the sweep sources changed since it was taken."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles",
                        "dram_traffic_rmat22_async_w2.md")
    try:
        lines = [ln.split() for ln in open(path) if ln.strip().startswith(("traffic_ratio",
                                                                           "sweep_sources"))]
    except OSError:
        return None
    src = [x[1] for x in lines if x[0] == "sweep_sources_sha256_16"]
    if not src or src[0] != sweep_sources_hash():
        return None
    r = [float(x[2]) for x in lines if x[0] == "traffic_ratio" and x[1] == kernel]
    return r[0] if r else None


def gen_graph(name):
    import graphgen as gg

    return gg.workload(name)


def alg_bytes_per_sweep(g):
    """Algorithmic HBM bytes of one sweep over the whole graph: the row
    pointer array (4 (n + 1)), the own label read and the label write (4 n
    each), over every vertex, and the column index (and weight) per entry."""
    return 4 * (g.n + 1) + 8 * g.n + (8 if g.weights is not None else 4) * g.m


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
    # one step = `sweeps` oracle sweeps from unique labels (bounded sample:
    # about 60 sweeps over the whole run, so that it ends within minutes)
    sweeps = max(1, min(args.cpu_sweeps // 2, 60 // max(1, args.steps + args.warmup)))

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


def run_reference_batch(args):
    """The CPU oracle on graphs of the batch workload (bounded sample per step)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import graphgen as gg
    import oracle

    p = workload_params(args)
    params = gg.batch_sbm_params(count=args.batch_count, seed=1000)
    sample = [gg.sbm_mixing(q["n"], q["k"], q["avg_degree"], q["mu"], seed=q["seed"])
              for q in params[::256][:4]]
    oracle.build()

    def step():
        t0 = time.perf_counter()
        for g in sample:
            oracle.rak(g.offsets, g.indices, g.weights, p["tolerance"], p["max_iter"], p["mode"],
                       strict=p["strict"])
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    tot = sum(step() for _ in range(args.steps))
    value = len(sample) * args.steps / tot
    print(json.dumps({
        "impl": "reference", "metric": f"batched graphs/s ({args.batch_count} SBM graphs)",
        "value": value, "unit": "graphs/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "batch", "graphs": args.batch_count, **p},
        "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": 1, "kind": "oracle",
                         "sample": f"{len(sample)} graphs of the batch (every 256th) per step"},
        "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)
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
    launches0 = lp.lp_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    iters, qs, run_ms = [], [], []
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        r, q = step()  # a fresh handle per step: the run is launched from the host
        iters.append(r.iterations)
        qs.append(q)
        run_ms.append(r.gpu_ms)
    e1.record(stream)
    barrier()
    launches = lp.lp_launch_count() - launches0
    clock_info = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    # profiled pass over the same steps: CUDA events around every sweep launch
    # on the library's stream (runs then go iteration by iteration)
    lp.lp_profile_reset()
    lp.lp_profile_enable(True)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    barrier()
    p0.record(stream)
    for _ in range(args.steps):
        step()
    p1.record(stream)
    barrier()
    lp.lp_profile_enable(False)
    prof = lp.lp_profile_read()
    prof_ms = p0.elapsed_time(p1)

    # the ceiling of a label-gathering sweep on this graph: one pass streaming
    # its entries and gathering one label per entry, with no per-row work
    m4 = (g.m // 4) * 4
    ceil_ms = lp.lp_probe_gather(g.n, idx[:m4], None if w is None else w[:m4],
                                 torch.arange(g.n, dtype=torch.int32, device=dev), mode=1,
                                 repeats=10, stream=stream.cuda_stream)

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
    # the ratios were measured on R-MAT-22 only: other graphs report none
    ratio = traffic_ratio(dom_name) if args.workload == "rmat22" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": None if ratio is None else ratio * dom["bytes"] / dom["launches"],
                "kernel": dom_name, "peak_source": peak_kind,
                "traffic_source": "profiles/dram_traffic_rmat22_async_w2.md (ratio to "
                                  "algorithmic bytes over a whole run, applied to this launch)"}
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
                  "gather_ceiling_ms": ceil_ms,
                  "of_gather_ceiling": ceil_ms / per_sweep_ms,
                  "run_ms_per_step": statistics.mean(run_ms),
                  "profiled_ms_per_step": prof_ms / args.steps,
                  "how": "steps timed with each RAK run launched from the host ahead of "
                         "its device-side tolerance test; kernel "
                         "times from a second pass of the same steps with CUDA events "
                         "around every sweep launch"},
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

    # the batched and served configurations, measured after the headline
    if args.workload == "rmat22" and not (args.no_batch and args.no_serve):
        del off, idx, w
        torch.cuda.empty_cache()
        ctx = Ctx(torch, lp, dev, rank, world, local)
        if not args.no_batch:
            line["batch"] = measure_batch(args, ctx, sub=True)
        if not args.no_serve:
            line["serve"] = measure_serve(args, ctx)

    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# batched graphs (one arena) against one graph at a time
# --------------------------------------------------------------------------
def batch_graphs(count):
    import graphgen as gg

    return gg.batch_sbm(gg.batch_sbm_params(count=count, seed=1000))


class Ctx:
    """What a measurement needs from the process set-up."""

    def __init__(self, torch, lp, dev, rank, world, local):
        self.torch, self.lp, self.dev = torch, lp, dev
        self.rank, self.world, self.local = rank, world, local
        self.stream = torch.cuda.current_stream(dev)

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist

            dist.barrier()
        self.torch.cuda.synchronize()


def setup_ctx():
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
    return Ctx(torch, lp, dev, rank, world, local)


def finish_ctx(ctx):
    if ctx.world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


def measure_batch(args, ctx, sub=False):
    """The batch workload: graphs shard whole over the ranks (size-balanced),
    each rank runs its share as one arena; value = graphs of all ranks / the
    slowest rank's time.  sub: the reduced form embedded in the single-graph
    line (3 timed steps, 128 graphs one at a time, one end-to-end step)."""
    torch, lp = ctx.torch, ctx.lp
    p = dict(WORKLOADS["batch"])
    count = args.batch_count
    steps = min(args.steps, 3) if sub else args.steps
    warmup = 1 if sub else args.warmup
    import graphgen as gg

    t0 = time.perf_counter()
    params_all = gg.batch_sbm_params(count=count, seed=1000)
    sizes = [q["n"] * q["avg_degree"] for q in params_all]
    mine = shard_graphs(sizes, ctx.rank, ctx.world)
    graphs = [gg.sbm_mixing(params_all[i]["n"], params_all[i]["k"], params_all[i]["avg_degree"],
                            params_all[i]["mu"], seed=params_all[i]["seed"]) for i in mine]
    gen_s = time.perf_counter() - t0
    n_tot = sum(g.n for g in graphs)
    m_tot = sum(g.m for g in graphs)
    stream = ctx.stream
    triples = [(g.offsets, g.indices, g.weights) for g in graphs]
    params, _ = lp.make_params(tolerance=p["tolerance"], max_iter=p["max_iter"], mode=p["mode"],
                               strict=p["strict"], waves=p["waves"])
    h = lp.lp_batch_create(triples, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    tune = lp.lp_batch_autotune(h, params, sweeps=5)  # outside the timed region
    tune_s = time.perf_counter() - t0

    def step():
        res = lp.lp_batch_run(h, len(graphs), params)
        lp.lp_batch_modularity(h, 0)  # computes every graph's modularity
        return res

    for _ in range(warmup):
        step()
    clocks = ClockSampler(nvsmi_id(torch, ctx.local), enabled=not args.no_clocks)
    launches0 = lp.lp_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ctx.barrier()
    e0.record(stream)
    iters_entries = 0
    for _ in range(steps):
        res = step()  # the batch's run is one CUDA graph launch
        iters_entries += sum(r.iterations * g.m for r, g in zip(res, graphs))
    e1.record(stream)
    ctx.barrier()
    launches = lp.lp_launch_count() - launches0
    clock_info = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    local_res = {i: (res[j].iterations, int(res[j].converged), lp.lp_batch_modularity(h, j))
                 for j, i in enumerate(mine)}
    lp.lp_profile_reset()
    lp.lp_profile_enable(True)
    step()
    torch.cuda.synchronize()
    lp.lp_profile_enable(False)
    prof = lp.lp_profile_read()
    t_ms, graphs_all = reduce_across_ranks(t_ms, len(graphs) * steps, device=ctx.dev)
    _, entries_all = reduce_across_ranks(0.0, iters_entries, device=ctx.dev)
    value = graphs_all / (t_ms * 1e-3)
    gteps = entries_all / (t_ms * 1e-3) / 1e9
    lp.lp_batch_destroy(h)
    assembled = gather_results(local_res, ctx.world)

    # e2e: every step creates the batch from pinned host buffers (host-to-device
    # copies and ingest inside the timed region), runs it, and reads every
    # graph's modularity back
    e2e = None
    if not args.no_e2e:
        total = sum(a.size for t in triples for a in t if a is not None)
        try:
            flat_t = torch.empty(total, dtype=torch.int32, pin_memory=True)
            host_kind = "pinned"
        except RuntimeError:
            flat_t = torch.empty(total, dtype=torch.int32)
            host_kind = "pageable (the pinned allocation failed)"
        flat = flat_t.numpy()
        pos, host_triples = 0, []
        for t in triples:
            views = []
            for a in t:
                if a is None:
                    views.append(None)
                    continue
                v = flat[pos:pos + a.size]
                v[:] = a
                views.append(v)
                pos += a.size
            host_triples.append(tuple(views))

        def e2e_step():
            hb = lp.lp_batch_create(host_triples, stream=stream.cuda_stream)
            lp.lp_batch_run(hb, len(graphs), params)
            lp.lp_batch_modularity(hb, 0)  # every graph's, read back to the host
            lp.lp_batch_destroy(hb)

        if not sub:
            e2e_step()
        ctx.barrier()
        e2e_steps = 1 if sub else min(steps, 3)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        ctx.barrier()
        e2e_s, _ = reduce_across_ranks((time.perf_counter() - t0) / e2e_steps, 0,
                                       device=ctx.dev)
        e2e = {"value": count / e2e_s, "unit": "graphs/s",
               "h2d_bytes_per_step": int(4 * total), "d2h_bytes_per_step": int(32 * len(graphs)),
               "steps": e2e_steps,
               "how": f"lp_batch_create from {host_kind} host buffers + one run + every "
                      "graph's modularity back on the host"}
        del flat, flat_t, host_triples

    # the same graphs one at a time: device-resident CSR, create + run + modularity
    n_sample = 128 if sub else args.per_graph_sample
    sample = list(range(0, len(graphs), max(1, len(graphs) // n_sample)))
    dev_csr = [tuple(None if a is None else torch.from_numpy(a).to(ctx.dev) for a in triples[i])
               for i in sample]
    for j in range(min(3, len(sample))):
        hh = lp.lp_graph_create(*dev_csr[j], borrow=True, stream=stream.cuda_stream)
        lp.lp_rak_run(hh, params)
        lp.lp_graph_destroy(hh)
    torch.cuda.synchronize()
    lat = []
    t0 = time.perf_counter()
    for j in range(len(sample)):
        s0 = time.perf_counter()
        hh = lp.lp_graph_create(*dev_csr[j], borrow=True, stream=stream.cuda_stream)
        lp.lp_rak_run(hh, params)
        lp.lp_modularity(hh)
        lp.lp_graph_destroy(hh)
        lat.append(time.perf_counter() - s0)
    per_graph_gps = len(sample) / (time.perf_counter() - t0)
    del dev_csr

    peak, peak_kind = measured_peak_gbs()
    kern = {k: v for k, v in prof.items() if v["launches"] > 0}
    dom_name = max(kern, key=lambda k: kern[k]["total_ms"])
    dom = kern[dom_name]
    achieved = dom["bytes"] / (dom["total_ms"] * 1e-3) / 1e9
    sweep_ms = sum(v["total_ms"] for v in kern.values())
    line = {
        "metric": f"batched graphs/s ({count} SBM graphs)", "value": value, "unit": "graphs/s",
        "n_gpus": ctx.world, "steps": steps, "warmup": warmup,
        "ms_per_step": t_ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "batch", "graphs": count, "graphs_this_rank": len(graphs),
                   "n_this_rank": n_tot, "m_this_rank": m_tot, **p,
                   "step": "lp_batch_run (all graphs, per-graph convergence on the device, one "
                           "CUDA graph launch) + modularity of every graph, arena resident in "
                           "HBM",
                   "l2": "inputs larger than L2", "generation_s": round(gen_s, 1),
                   "autotune": {**tune.as_dict(), "seconds": round(tune_s, 2)},
                   "parallelism": (f"graph-level sharding over {ctx.world} ranks (size-balanced)"
                                   if ctx.world > 1 else "single GPU")},
        "gteps": gteps,
        "assembled_graphs": len(assembled),
        "per_graph_launch": {"graphs_per_s": per_graph_gps, "sample": len(sample),
                             "p50_ms": 1e3 * statistics.median(lat),
                             "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                             "how": "lp_graph_create (borrowed device CSR) + lp_rak_run + "
                                    "lp_modularity per graph, sequentially, this rank's graphs"},
        "speedup_vs_per_graph": value / ctx.world / per_graph_gps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": dom_name,
                     "peak_source": peak_kind},
        "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"],
                        "share": v["total_ms"] / sweep_ms} for k, v in kern.items()},
        "gpu_launches": int(launches),
        "clocks": clock_info,
        "e2e": e2e,
    }
    if ctx.rank == 0 and not sub and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        t0 = time.perf_counter()
        done = 0
        for g in graphs[::64][:16]:
            oracle.rak(g.offsets, g.indices, g.weights, p["tolerance"], p["max_iter"], p["mode"],
                       strict=p["strict"])
            oracle.modularity(g.offsets, g.indices, g.weights, np.arange(g.n, dtype=np.int32))
            done += 1
            if time.perf_counter() - t0 > 25:
                break
        t = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / t, "unit": "graphs/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"{done} graphs of the batch (every 64th), full runs"}
    return line


def run_batch(args):
    ctx = setup_ctx()
    line = measure_batch(args, ctx)
    finish_ctx(ctx)
    if ctx.rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# serving with continuous batching against one request at a time
# --------------------------------------------------------------------------
def serve_pool(count, seed=7, n_lo=10_000, n_hi=2_000_000):
    """Graphs of the serving stream: type uniform over SBM (mean degree 16,
    mixing 0.3), R-MAT (edge factor 8, 2^round(log2 n) vertices) and grid
    (side floor(sqrt n)); n log-uniform in [n_lo, n_hi] (10k-2M); weights 1-8."""
    import math

    import graphgen as gg

    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))
        kind = i % 3
        if kind == 0:
            out.append(gg.sbm_mixing(n, max(2, n // 500), 16.0, 0.3, seed=seed + i, wmin=1, wmax=8))
        elif kind == 1:
            out.append(gg.rmat(int(round(math.log2(n))), edge_factor=8, seed=seed + i, wmin=1,
                               wmax=8))
        else:
            out.append(gg.grid_road(int(math.isqrt(n)), seed=seed + i, wmin=1, wmax=8))
    return out


def measure_serve(args, ctx):
    """The serving workload: a Poisson stream of requests drawn from a pool of
    distinct graphs, served with continuous batching; under torchrun rank r
    serves the requests r, r + N, ... on its own GPU (graph-level sharding)
    and the latencies of every rank are pooled."""
    torch, lp = ctx.torch, ctx.lp
    p = dict(WORKLOADS["serve"])
    t0 = time.perf_counter()
    pool = serve_pool(args.serve_pool)
    gen_s = time.perf_counter() - t0
    pinned = [tuple(torch.from_numpy(a).pin_memory() for a in (g.offsets, g.indices, g.weights))
              for g in pool]
    rng = np.random.default_rng(11)
    n_all = int(rng.poisson(args.serve_rate * args.serve_seconds))
    arrivals_all = np.sort(rng.uniform(0, args.serve_seconds, n_all))
    picks_all = rng.integers(0, len(pool), n_all)
    mine = [rid for rid in range(n_all) if rid % ctx.world == ctx.rank]
    params, _ = lp.make_params(tolerance=p["tolerance"], max_iter=p["max_iter"], mode=p["mode"],
                               strict=p["strict"], waves=p["waves"])
    cfg = lp.lp_server_config_default()
    cfg.hbm_budget = 64 << 30
    cfg.max_active = 64
    cfg.streams = 8
    if args.serve_cohort is not None:
        cfg.max_cohort = args.serve_cohort
    if args.serve_admitters is not None:
        cfg.admitters = args.serve_admitters
    if args.serve_cohort_entries is not None:
        cfg.cohort_max_entries = args.serve_cohort_entries

    # warm-up: every pool graph once through the server
    srv = lp.lp_server_create(cfg, params)
    for i, (o, x, w) in enumerate(pinned):
        lp.lp_server_submit(srv, i, o, x, w)
    lp.lp_server_drain(srv)
    lp.lp_server_poll(srv, capacity=len(pool))

    ctx.barrier()
    launches0 = lp.lp_launch_count()
    clocks = ClockSampler(nvsmi_id(torch, ctx.local), enabled=not args.no_clocks)
    outs, done = {}, []
    start = time.perf_counter()
    for rid in mine:
        delay = start + arrivals_all[rid] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        o, x, w = pinned[picks_all[rid]]
        outs[rid] = np.empty(pool[picks_all[rid]].n, np.int32)
        lp.lp_server_submit(srv, rid, o, x, w, outs[rid])
        for r in lp.lp_server_poll(srv, capacity=256):
            done.append(r)
            outs.pop(r.request_id, None)
    lp.lp_server_drain(srv)
    done += lp.lp_server_poll(srv, capacity=len(mine) + 1)
    makespan = time.perf_counter() - start
    clock_info = clocks.stop()
    launches = lp.lp_launch_count() - launches0
    cohorts = lp.lp_server_stats(srv)
    lp.lp_server_destroy(srv)
    local = {r.request_id: (r.latency_ms, r.queued_ms, r.status, r.iterations) for r in done}
    merged = gather_results(local, ctx.world)
    makespan, _ = reduce_across_ranks(makespan, 0, device=ctx.dev)
    lat = np.array([v[0] for v in merged.values()])
    queued = np.array([v[1] for v in merged.values()])
    errors = sum(1 for v in merged.values() if v[2] != 0)
    entries = sum(v[3] * pool[picks_all[k]].m for k, v in merged.items())

    # the same arrivals, one graph at a time (no overlap, no batching), on rank 0
    nb = int(np.searchsorted(arrivals_all, args.serve_baseline_seconds))
    base_lat = []
    bstart = time.perf_counter()
    for rid in range(nb):
        delay = bstart + arrivals_all[rid] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        o, x, w = pinned[picks_all[rid]]
        h = lp.lp_graph_create(o, x, w)
        lp.lp_rak_run(h, params)
        lp.lp_modularity(h)
        lp.lp_labels_get(h)
        lp.lp_graph_destroy(h)
        base_lat.append(1e3 * (time.perf_counter() - bstart - arrivals_all[rid]))
    base_span = time.perf_counter() - bstart
    base_lat = np.array(base_lat) if base_lat else np.zeros(1)

    # saturation: the same burst of requests submitted at once, served with
    # continuous batching and one graph at a time (service capacity)
    sat_picks = np.random.default_rng(13).integers(0, len(pool), args.serve_saturation)
    srv = lp.lp_server_create(cfg, params)
    sstart = time.perf_counter()
    for rid, k in enumerate(sat_picks):
        o, x, w = pinned[k]
        outs[("sat", rid)] = np.empty(pool[k].n, np.int32)
        lp.lp_server_submit(srv, rid, o, x, w, outs[("sat", rid)])
    lp.lp_server_drain(srv)
    sat_span = time.perf_counter() - sstart
    sat_done = lp.lp_server_poll(srv, capacity=len(sat_picks) + 1)
    sat_cohorts = lp.lp_server_stats(srv)
    lp.lp_server_destroy(srv)
    sat_err = sum(1 for r in sat_done if r.status != 0)
    sstart = time.perf_counter()
    for k in sat_picks:
        o, x, w = pinned[k]
        h = lp.lp_graph_create(o, x, w)
        lp.lp_rak_run(h, params)
        lp.lp_modularity(h)
        lp.lp_labels_get(h)
        lp.lp_graph_destroy(h)
    seq_span = time.perf_counter() - sstart

    # a burst of small graphs (n 1k-20k), where launches dominate and
    # cohorts share them: served against one graph at a time
    small = serve_pool(64, seed=17, n_lo=1_000, n_hi=20_000)
    small_pinned = [tuple(torch.from_numpy(a).pin_memory() for a in (g.offsets, g.indices,
                                                                      g.weights))
                    for g in small]
    small_picks = np.random.default_rng(19).integers(0, len(small), 4 * args.serve_saturation)

    def small_burst(config):
        srv = lp.lp_server_create(config, params)
        t = time.perf_counter()
        for rid, k in enumerate(small_picks):
            o, x, w = small_pinned[k]
            lp.lp_server_submit(srv, rid, o, x, w)
        lp.lp_server_drain(srv)
        span = time.perf_counter() - t
        got = lp.lp_server_poll(srv, capacity=len(small_picks) + 1)
        st = lp.lp_server_stats(srv)
        lp.lp_server_destroy(srv)
        return span, sum(1 for r in got if r.status != 0), st

    small_burst(cfg)  # warm-up
    sm_span, sm_err, sm_cohorts = small_burst(cfg)
    single = lp.lp_server_config_default()
    single.hbm_budget, single.max_active, single.streams = cfg.hbm_budget, cfg.max_active, cfg.streams
    single.max_cohort = 1
    sm1_span, sm1_err, _ = small_burst(single)
    t = time.perf_counter()
    for k in small_picks:
        o, x, w = small_pinned[k]
        h = lp.lp_graph_create(o, x, w)
        lp.lp_rak_run(h, params)
        lp.lp_modularity(h)
        lp.lp_labels_get(h)
        lp.lp_graph_destroy(h)
    sm_seq = time.perf_counter() - t
    return {
        "metric": f"served graphs/s (Poisson {args.serve_rate:g} req/s)",
        "value": len(merged) / makespan, "unit": "graphs/s", "n_gpus": ctx.world,
        "steps": n_all, "warmup": len(pool), "ms_per_step": 1e3 * makespan / max(1, len(merged)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "serve", **p, "requests": n_all, "window_s": args.serve_seconds,
                   "pool_graphs": len(pool), "pool_generation_s": round(gen_s, 1),
                   "max_active": cfg.max_active, "streams": cfg.streams,
                   "max_cohort": cfg.max_cohort, "admitters": cfg.admitters,
                   "cohort_max_entries": cfg.cohort_max_entries,
                   "hbm_budget_gib": cfg.hbm_budget >> 30,
                   "l2": "graphs resident per request, no flush",
                   "parallelism": (f"requests sharded over {ctx.world} ranks"
                                   if ctx.world > 1 else "single GPU")},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean_queued": float(queued.mean())},
        "gteps": entries / makespan / 1e9,
        "errors": errors,
        "per_graph_launch": {"requests": nb, "graphs_per_s": nb / base_span,
                             "p50_ms": float(np.percentile(base_lat, 50)),
                             "p99_ms": float(np.percentile(base_lat, 99)),
                             "window_s": args.serve_baseline_seconds},
        "saturation": {"requests": len(sat_picks), "errors": sat_err,
                       "served_graphs_per_s": len(sat_picks) / sat_span,
                       "per_graph_launch_graphs_per_s": len(sat_picks) / seq_span,
                       "cohorts": sat_cohorts,
                       "how": "all requests submitted at t=0; the per-graph arm runs the same "
                              "requests one after another through lp_graph_create/lp_rak_run"},
        "saturation_small": {"requests": len(small_picks), "errors": sm_err + sm1_err,
                             "pool": "64 graphs, n log-uniform 1k-20k, same kinds and weights",
                             "served_graphs_per_s": len(small_picks) / sm_span,
                             "served_without_cohorts_graphs_per_s": len(small_picks) / sm1_span,
                             "per_graph_launch_graphs_per_s": len(small_picks) / sm_seq,
                             "cohorts": sm_cohorts},
        "cohorts": cohorts,
        "gpu_launches": int(launches),
        "clocks": clock_info,
        "e2e": {"value": len(merged) / makespan, "unit": "graphs/s",
                "h2d_bytes_per_step": int(np.mean([pool[i].offsets.nbytes + pool[i].indices.nbytes
                                                   + pool[i].weights.nbytes for i in picks_all])),
                "d2h_bytes_per_step": int(np.mean([pool[i].n * 4 for i in picks_all])),
                "how": "submit from pinned host CSR -> labels and modularity back on the host"},
    }


def run_serve(args):
    ctx = setup_ctx()
    line = measure_serve(args, ctx)
    finish_ctx(ctx)
    if ctx.rank == 0:
        print(json.dumps(line), flush=True)
    return 0


EXPERIMENT_TOLERANCES = (0.1, 0.05, 0.01, 0.001, 0.0001)


def run_experiment(args):
    """Tolerance / tie-rule / update-order study (Sec. 3.2; self-loops,
    Sec. 3.1) on the synthetic classes: one JSON line per setting."""
    import torch

    import graphgen as gg
    import paper_2301_09125_gb300 as lp
    from paper_2301_09125_gb300 import build

    build.build()
    lp.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    for name in [c for c in args.classes.split(",") if c]:
        base = gen_graph(name)
        waves = WORKLOADS[name]["waves"]
        plain = [torch.from_numpy(a).to(dev) if a is not None else None
                 for a in (base.offsets, base.indices, base.weights)]
        h_plain = lp.lp_graph_create(*plain, borrow=True, stream=stream.cuda_stream)
        lab = torch.empty(base.n, dtype=torch.int32, device=dev)
        for loops in (False, True):
            g = gg.with_self_loops(base) if loops else base
            arrs = [torch.from_numpy(a).to(dev) if a is not None else None
                    for a in (g.offsets, g.indices, g.weights)]
            h = lp.lp_graph_create(*arrs, borrow=True, stream=stream.cuda_stream)
            for mode in ("sync", "async"):
                for strict in (True, False):
                    for tol in EXPERIMENT_TOLERANCES:
                        params, _ = lp.make_params(tolerance=tol, max_iter=100, mode=mode,
                                                   strict=strict, waves=waves, seed=1)
                        lp.lp_rak_run(h, params)  # warm-up
                        lp.lp_rak_run(h, params)  # repeated parameters: captured as a graph
                        torch.cuda.synchronize()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        r = lp.lp_rak_run(h, params)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        ms = e0.elapsed_time(e1)
                        lp.lp_labels_get(h, lab)
                        q = lp.lp_modularity(h_plain, lab)
                        print(json.dumps({
                            "experiment": "tolerance", "workload": name, "n": base.n,
                            "m": base.m, "self_loops": loops, "mode": mode,
                            "waves": waves if mode == "async" else 1, "strict": strict,
                            "tolerance": tol, "iterations": r.iterations,
                            "converged": bool(r.converged), "run_ms": ms,
                            "gteps": r.iterations * g.m / (ms * 1e-3) / 1e9,
                            "modularity": q}), flush=True)
            lp.lp_graph_destroy(h)
        lp.lp_graph_destroy(h_plain)
    return 0


def run_split_experiment(args):
    """Split of disconnected communities after RAK (each class's benchmark
    parameters): communities before and after, modularity before and after,
    time of the split (CUDA events on the library's stream), its roofline,
    and the oracle's split of the same labels (checked equal, and timed)."""
    import torch

    import oracle

    import paper_2301_09125_gb300 as lp
    from paper_2301_09125_gb300 import build

    build.build()
    lp.load()
    oracle.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    for name in [c for c in args.classes.split(",") if c]:
        g = gen_graph(name)
        p = WORKLOADS[name]
        params, _ = lp.make_params(tolerance=p["tolerance"], max_iter=p["max_iter"],
                                   mode=p["mode"], strict=p["strict"], waves=p["waves"])
        arrs = [torch.from_numpy(a).to(dev) if a is not None else None
                for a in (g.offsets, g.indices, g.weights)]
        times = []
        for rep in range(4):
            h = lp.lp_graph_create(*arrs, borrow=True, stream=stream.cuda_stream)
            lp.lp_rak_run(h, params)
            before = lp.lp_labels_get(h)
            q0 = lp.lp_modularity(h)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            k = lp.lp_split_communities(h)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep:  # the first split pays for its scratch allocation
                times.append(e0.elapsed_time(e1))
            q1 = lp.lp_modularity(h)
            after = lp.lp_labels_get(h)
            lp.lp_graph_destroy(h)
        ms = statistics.median(times)
        # the oracle's split of the same labels, on one host core; its result
        # is the GPU's (component ids are the smallest vertices)
        t0 = time.perf_counter()
        ref, ref_k = oracle.split(g.offsets, g.indices, before)
        cpu_s = time.perf_counter() - t0
        # algorithmic bytes: the CSR's offsets and column indices once, the
        # labels read and the component ids written once
        alg = 4 * (g.n + 1) + 4 * g.m + 8 * g.n
        peak, peak_kind = measured_peak_gbs()
        print(json.dumps({"experiment": "split", "workload": name, "n": g.n, "m": g.m,
                          "mode": p["mode"], "communities_before": int(len(np.unique(before))),
                          "communities_after": k, "modularity_before": q0,
                          "modularity_after": q1, "split_ms": ms,
                          "gteps": g.m / (ms * 1e-3) / 1e9,
                          "equals_oracle": bool(ref_k == k and np.array_equal(ref, after)),
                          "roofline": {"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9,
                                       "peak": peak, "unit": "GB/s",
                                       "frac": alg / (ms * 1e-3) / 1e9 / peak, "traffic": None,
                                       "alg_bytes": alg, "peak_source": peak_kind},
                          "cpu_baseline": {"value": g.m / cpu_s / 1e9, "unit": "GTEPS",
                                           "cores": 1, "kind": "oracle",
                                           "sample": f"the split of the same labels on the full "
                                                     f"graph ({cpu_s:.1f} s, single thread)"}}),
              flush=True)
    return 0


# COPRA (Sec. 3.3) and SLPA (Sec. 3.4) on the synthetic classes
METHOD_DEFAULTS = {
    # the paper's suggestion for COPRA: tolerance 0.01, 4 labels for
    # non-road graphs, asynchronous updates (each class's wave count)
    "copra": dict(max_labels=4, tolerance=0.01, max_iter=20),
    "slpa": dict(memory_size=20, tolerance=0.05),
}


def method_alg_bytes(method, g, max_labels):
    """Algorithmic HBM bytes of one iteration: the CSR once (4 (n + 1) + 4 or
    8 per entry); COPRA reads the previous sets and writes the new ones (8
    bytes per pair and vertex each way: label and belonging, every speaker's
    set counted once); SLPA reads the previous slot and writes the new one (4
    per vertex each)."""
    csr = 4 * (g.n + 1) + (8 if g.weights is not None else 4) * g.m
    if method == "copra":
        return csr + 16 * max_labels * g.n
    return csr + 8 * g.n


def run_method_experiment(args):
    """COPRA or SLPA on each class: one run to convergence timed with CUDA
    events on the library's stream (best of 3 after a warm-up run), GTEPS
    (iterations x m / run time), the iteration's algorithmic bytes against
    the measured HBM peak, the first iteration compared with the oracle at
    full size, and the oracle's first iteration timed as the CPU baseline."""
    import torch

    import oracle
    import paper_2301_09125_gb300 as lp
    from paper_2301_09125_gb300 import build

    method = args.experiment
    build.build()
    lp.load()
    oracle.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = measured_peak_gbs()
    d = METHOD_DEFAULTS[method]
    for name in [c for c in args.classes.split(",") if c]:
        g = gen_graph(name)
        p = WORKLOADS[name]
        arrs = [torch.from_numpy(a).to(dev) if a is not None else None
                for a in (g.offsets, g.indices, g.weights)]
        h = lp.lp_graph_create(*arrs, borrow=True, stream=stream.cuda_stream)
        if method == "copra":
            kw = dict(max_labels=d["max_labels"], tolerance=d["tolerance"],
                      max_iter=d["max_iter"], mode=p["mode"], waves=p["waves"],
                      strict=p["strict"], seed=1)
            run = lambda **o: lp.lp_copra_run(h, **{**kw, **o})  # noqa: E731
            settings = {k: kw[k] for k in ("max_labels", "tolerance", "max_iter", "mode",
                                           "strict")}
            settings["waves"] = p["waves"] if p["mode"] == "async" else 1
        else:
            kw = dict(memory_size=d["memory_size"], tolerance=d["tolerance"],
                      strict=p["strict"], seed=1)
            run = lambda **o: lp.lp_slpa_run(h, **{**kw, **o})  # noqa: E731
            settings = dict(kw, mode="sync")
            settings.pop("seed")
        # first iteration against the oracle, full arrays (and its CPU time)
        o_waves = p["waves"] if p["mode"] == "async" else 0
        t0 = time.perf_counter()
        if method == "copra":
            _, ref_l, ref_b, _, _, _ = oracle.copra(
                g.offsets, g.indices, g.weights, max_labels=kw["max_labels"], tolerance=0.0,
                max_iter=1, mode=p["mode"], waves=o_waves, strict=p["strict"], seed=1)
        else:
            _, ref_mem, _, _, _ = oracle.slpa(g.offsets, g.indices, g.weights, memory_size=2,
                                              tolerance=0.0, strict=p["strict"], seed=1)
        cpu_s = time.perf_counter() - t0
        if method == "copra":
            run(max_iter=1, tolerance=0.0)
            sl, sb = lp.lp_copra_sets_get(h, kw["max_labels"])
            exact = bool(np.array_equal(sb, ref_b) and
                         np.array_equal(np.where(ref_b > 0, sl, 0), np.where(ref_b > 0, ref_l, 0)))
            del sl, sb, ref_l, ref_b
        else:
            run(memory_size=2, tolerance=0.0)
            exact = bool(np.array_equal(lp.lp_slpa_memory_get(h, 2), ref_mem))
            del ref_mem
        run()  # warm-up: scratch allocation
        launches0 = lp.lp_launch_count()
        clocks = ClockSampler(nvsmi_id(torch, 0), enabled=not args.no_clocks)
        best = None
        for _ in range(3):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if best is None or ms < best[0]:
                best = (ms, r.iterations, bool(r.converged))
        clock_info = clocks.stop()
        launches = (lp.lp_launch_count() - launches0) // 3
        q = lp.lp_modularity(h)
        lp.lp_graph_destroy(h)
        ms, iters, conv = best
        alg = method_alg_bytes(method, g, kw.get("max_labels", 1))
        it_ms = ms / max(iters, 1)
        achieved = alg / (it_ms * 1e-3) / 1e9
        print(json.dumps({
            "experiment": method, "metric": f"{method.upper()} GTEPS ({name})",
            "workload": name, "n": g.n, "m": g.m, **settings,
            "iterations": iters, "converged": conv, "run_ms": ms, "ms_per_iteration": it_ms,
            "value": iters * g.m / (ms * 1e-3) / 1e9, "unit": "GTEPS", "modularity": q,
            "first_iteration_bit_exact": exact,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "whole iteration", "alg_bytes": alg,
                         "peak_source": peak_kind},
            "cpu_baseline": {"value": g.m / cpu_s / 1e9, "unit": "GTEPS", "cores": 1,
                             "kind": "oracle",
                             "sample": f"first iteration on the full graph ({cpu_s:.1f} s, "
                                       f"single thread)"},
            "gpu_launches": launches, "clocks": clock_info}), flush=True)
        del arrs
        torch.cuda.empty_cache()
    return 0


def run_noalloc_experiment(args):
    """lp_rak_sweep_noalloc (one synchronous sweep, no allocation) on each
    class whose rows fit its limit of 4096 entries: the first sweep from
    unique labels and a second one from its result, each timed with CUDA
    events (best of 5), against the sweeps of a 3-iteration synchronous
    lp_rak_run of the same graph; the first sweep's labels are compared with
    lp_rak_run's one-iteration labels."""
    import torch

    import paper_2301_09125_gb300 as lp
    from paper_2301_09125_gb300 import build

    build.build()
    lp.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    for name in [c for c in args.classes.split(",") if c]:
        g = gen_graph(name)
        maxdeg = int(np.diff(g.offsets.astype(np.int64)).max())
        if maxdeg > 4096:
            print(json.dumps({"experiment": "noalloc", "workload": name, "skipped":
                              f"longest row {maxdeg} entries, beyond the 4096 of the entry point"}),
                  flush=True)
            continue
        off, idx, w = (torch.from_numpy(a).to(dev) if a is not None else None
                       for a in (g.offsets, g.indices, g.weights))
        lab0 = torch.arange(g.n, dtype=torch.int32, device=dev)
        lab1 = torch.empty_like(lab0)
        lab2 = torch.empty_like(lab0)

        def timed(src, dst):
            best = None
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                lp.lp_rak_sweep_noalloc(off, idx, w, src, dst, strict=True)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            return best

        lp.lp_rak_sweep_noalloc(off, idx, w, lab0, lab1, strict=True)  # warm-up
        first_ms = timed(lab0, lab1)
        second_ms = timed(lab1, lab2)
        h = lp.lp_graph_create(off, idx, w, borrow=True, stream=stream.cuda_stream)
        params, _ = lp.make_params(tolerance=0.0, max_iter=1, mode="sync", strict=True)
        lp.lp_rak_run(h, params)
        same = bool(torch.equal(lp.lp_labels_get(h, torch.empty_like(lab0)), lab1))
        params3, _ = lp.make_params(tolerance=0.0, max_iter=3, mode="sync", strict=True)
        lp.lp_rak_run(h, params3)
        r = lp.lp_rak_run(h, params3)
        lp.lp_graph_destroy(h)
        print(json.dumps({"experiment": "noalloc", "workload": name, "n": g.n, "m": g.m,
                          "first_sweep_ms": first_ms, "second_sweep_ms": second_ms,
                          "noalloc_gteps": g.m / (second_ms * 1e-3) / 1e9,
                          "lp_rak_run_ms_per_sweep": r.gpu_ms / max(r.iterations, 1),
                          "first_sweep_equals_lp_rak_run": same}), flush=True)
        del off, idx, w, lab0, lab1, lab2
        torch.cuda.empty_cache()
    return 0


def degree_renumbered(g):
    """The graph with vertices renumbered by decreasing degree (stable), rows
    in the new order: a layout where the most gathered labels sit together."""
    n, m = g.n, g.m
    deg = np.diff(g.offsets.astype(np.int64))
    order = np.argsort(-deg, kind="stable")
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n)
    d2 = deg[order]
    off2 = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(d2, out=off2[1:])
    rowid = np.repeat(np.arange(n), d2)
    src = g.offsets[:-1].astype(np.int64)[order][rowid] + (np.arange(m) - off2[:-1][rowid])
    idx2 = pos[g.indices[src]].astype(np.int32)
    w2 = None if g.weights is None else g.weights[src]
    return idx2, w2


def run_gather_experiment(args):
    """The ceiling a label-gathering sweep can reach on each class: one pass
    streaming the column indices and weights (mode 0), and the same pass also
    gathering every entry's neighbour label (mode 1), on the graph as given
    and renumbered by decreasing degree.  Bytes are the sweep's algorithmic
    HBM bytes (4 (n + 1) + 8 n + 4 or 8 per entry)."""
    import torch

    import paper_2301_09125_gb300 as lp
    from paper_2301_09125_gb300 import build

    build.build()
    lp.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peak, peak_kind = measured_peak_gbs()
    for name in [c for c in args.classes.split(",") if c]:
        g = gen_graph(name)
        alg = alg_bytes_per_sweep(g)
        for numbering in ("as generated", "by decreasing degree"):
            if numbering == "as generated":
                idx, w = g.indices, g.weights
            else:
                idx, w = degree_renumbered(g)
            m4 = (g.m // 4) * 4
            t_idx = torch.from_numpy(np.ascontiguousarray(idx[:m4])).to(dev)
            t_w = None if w is None else torch.from_numpy(np.ascontiguousarray(w[:m4])).to(dev)
            lab = torch.arange(g.n, dtype=torch.int32, device=dev)
            for mode in (0, 1):
                ms = lp.lp_probe_gather(g.n, t_idx, t_w, lab, mode=mode, repeats=20)
                moved = (4 if w is None else 8) * m4  # the bytes the pass streams
                print(json.dumps({"experiment": "gather", "workload": name, "n": g.n, "m": g.m,
                                  "numbering": numbering,
                                  "pass": "stream" if mode == 0 else "stream + label gather",
                                  "ms": ms, "g_entries_per_s": g.m / (ms * 1e-3) / 1e9,
                                  "moved_gbs": moved / (ms * 1e-3) / 1e9,
                                  "moved_frac": moved / (ms * 1e-3) / 1e9 / peak,
                                  "l2_resident": moved < L2_BYTES,
                                  "sweep_alg_gbs": alg / (ms * 1e-3) / 1e9,
                                  "hbm_frac": alg / (ms * 1e-3) / 1e9 / peak,
                                  "peak_gbs": peak, "peak_source": peak_kind}), flush=True)
            del t_idx, t_w, lab
    return 0


def main():
    args = parse()
    if args.experiment == "gather":
        return run_gather_experiment(args)
    if args.experiment == "split":
        return run_split_experiment(args)
    if args.experiment in ("copra", "slpa"):
        return run_method_experiment(args)
    if args.experiment == "noalloc":
        return run_noalloc_experiment(args)
    if args.experiment:
        return run_experiment(args)
    if args.workload == "serve":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the serving workload has no CPU reference arm; see the batch and "
                              "single-graph workloads"}))
            return 0
        return run_serve(args)
    if args.workload == "batch":
        if args.impl == "reference":
            return run_reference_batch(args)
        return run_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
