"""Host-side logic of bench.py that needs no GPU: the cross-rank reduction of
the multi-GPU path, the graph-level sharding of the batch and serving
workloads and the assembly of per-graph results (gloo, world size 2), and the
reference arm's rank rule."""
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

from conftest import ROOT


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench

    t, e = bench.reduce_across_ranks(10.0 + rank, 100 * (rank + 1))
    out[rank] = (t, e)
    dist.destroy_process_group()


def test_reduce_across_ranks_gloo():
    import random

    port = random.randint(20000, 40000)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        assert out[0] == (11.0, 300.0) and out[1] == (11.0, 300.0)


def test_reduce_without_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_across_ranks(3.5, 7) == (3.5, 7.0)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_traffic_summary_is_well_formed():
    """The committed DRAM-traffic summary carries one ratio per sweep bucket
    and a sources hash in the form bench.py checks; bench.py returns its
    ratio when the hash matches the current sweep sources, and None when
    they differ."""
    sys.path.insert(0, ROOT)
    import bench

    path = os.path.join(ROOT, "profiles", "dram_traffic_rmat22_async_w2.md")
    lines = [ln.split() for ln in open(path)
             if ln.strip().startswith(("traffic_ratio", "sweep_sources"))]
    ratios = {x[1]: float(x[2]) for x in lines if x[0] == "traffic_ratio"}
    assert set(ratios) == {"sweep_small", "sweep_warp", "sweep_cta", "sweep_cta2", "sweep_hub"}
    assert all(0.5 < r < 10 for r in ratios.values())
    hashes = [x[1] for x in lines if x[0] == "sweep_sources_sha256_16"]
    assert len(hashes) == 1 and len(hashes[0]) == 16
    current = bench.sweep_sources_hash()
    expect = ratios["sweep_hub"] if hashes[0] == current else None
    assert bench.traffic_ratio("sweep_hub") == expect


def _shard_worker(rank, world, port, sizes, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench

    mine = bench.shard_graphs(sizes, rank, world)
    merged = bench.gather_results({i: (rank, i * i) for i in mine}, world)
    out[rank] = (mine, merged)
    dist.destroy_process_group()


def test_graph_sharding_and_assembly_gloo():
    """Each graph runs on exactly one rank; every rank ends with every graph's
    result."""
    import random

    sizes = [int(x) for x in (1000 * (1 + (7 * i) % 13) for i in range(37))]
    port = random.randint(20000, 40000)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_shard_worker, args=(2, port, sizes, out), nprocs=2, join=True)
        shards = [out[0][0], out[1][0]]
        assert sorted(shards[0] + shards[1]) == list(range(len(sizes)))
        for r in (0, 1):
            merged = out[r][1]
            assert sorted(merged) == list(range(len(sizes)))
            assert all(merged[i] == (0 if i in shards[0] else 1, i * i) for i in merged)


def test_graph_sharding_balances_work():
    sys.path.insert(0, ROOT)
    import bench

    sizes = [int(1000 * 1.7 ** (i % 11)) for i in range(200)]
    for world in (1, 2, 3, 8):
        parts = [bench.shard_graphs(sizes, r, world) for r in range(world)]
        assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    assert bench.gather_results({3: "x"}, 1) == {3: "x"}


@pytest.mark.parametrize("steps, sweeps", [(2, 2), (40, 1)])
def test_reference_arm_bounds_its_sample(steps, sweeps):
    """The reference arm (the oracle on one host core) takes two sweeps per
    step, but at most about 60 over the whole run, so a long --steps still
    ends within minutes; its line reports the same metric as the GPU arm."""
    import json

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "sbm10k", "--steps", str(steps), "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])
    assert line["impl"] == "reference" and line["steps"] == steps
    assert line["metric"] == "RAK GTEPS (sbm10k)" and line["value"] > 0
    assert line["cpu_baseline"]["sample"].startswith(f"{sweeps} sync sweeps")
