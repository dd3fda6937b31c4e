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
