"""Host-side logic of bench.py that needs no GPU: the cross-rank reduction of
the multi-GPU path (gloo, world size 2) and the reference arm's rank rule."""
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

    path = os.path.join(ROOT, "profiles", "dram_traffic_rmat21_async_w2.md")
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
