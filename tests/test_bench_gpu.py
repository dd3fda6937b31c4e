"""The benchmark's study modes on the smallest class (GPU): every setting
prints one well-formed JSON line and the split never loses a vertex."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return [json.loads(line) for line in out.stdout.splitlines() if line.startswith("{")]


def test_tolerance_study_lines():
    rows = run_bench("--experiment", "tolerance", "--classes", "sbm10k")
    assert len(rows) == 2 * 2 * 2 * 5  # self-loops x mode x ties x tolerances
    for r in rows:
        assert r["workload"] == "sbm10k" and 1 <= r["iterations"] <= 100
        assert -0.5 <= r["modularity"] <= 1.0 and r["run_ms"] > 0


def test_split_study_lines():
    rows = run_bench("--experiment", "split", "--classes", "sbm10k")
    assert len(rows) == 1
    r = rows[0]
    assert r["communities_after"] >= r["communities_before"] >= 1
    assert r["modularity_after"] >= r["modularity_before"] - 1e-9


def test_gather_ceiling_lines():
    rows = run_bench("--experiment", "gather", "--classes", "sbm10k")
    assert len(rows) == 4  # numbering x (stream, stream + gather)
    assert {r["numbering"] for r in rows} == {"as generated", "by decreasing degree"}
    for r in rows:
        assert r["ms"] > 0 and r["hbm_frac"] > 0


def test_probe_rejects_out_of_range_indices():
    import numpy as np
    import torch

    sys.path.insert(0, ROOT)
    import __graft_entry__

    __graft_entry__.build()
    import paper_2301_09125_gb300 as lp

    dev = torch.device("cuda")
    idx = torch.from_numpy(np.array([0, 1, 2, 3, 1, 2, 3, 9], np.int32)).to(dev)
    lab = torch.arange(4, dtype=torch.int32, device=dev)
    with pytest.raises(lp.LPError, match="outside"):
        lp.lp_probe_gather(4, idx, None, lab, mode=1)
    assert lp.lp_probe_gather(4, idx[:4].contiguous(), None, lab, mode=1, repeats=2) > 0
