import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workload, minutes")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def csr_from_adj(adj, w=None):
    """CSR arrays from row lists (rows kept in the given order)."""
    n = len(adj)
    offsets = np.zeros(n + 1, dtype=np.int32)
    for v, row in enumerate(adj):
        offsets[v + 1] = offsets[v] + len(row)
    indices = np.array([u for row in adj for u in row], dtype=np.int32)
    weights = None if w is None else np.array([x for row in w for x in row], dtype=np.int32)
    return offsets, indices, weights


def random_graph(n, p, seed, wmax=1, self_loops=False):
    """Small random undirected graph as a symmetric CSR (numpy, for tests).
    Rows are shuffled: the adjacency order is part of the input."""
    rng = np.random.default_rng(seed)
    a = np.triu(rng.random((n, n)) < p, 0 if self_loops else 1)
    wt = np.triu(rng.integers(1, wmax + 1, size=(n, n)))
    a = a | a.T
    wt = wt + np.triu(wt, 1).T
    rows, ws = [], []
    for v in range(n):
        nb = np.nonzero(a[v])[0]
        rng.shuffle(nb)
        rows.append([int(u) for u in nb])
        ws.append([int(wt[v, u]) for u in nb])
    off, idx, w = csr_from_adj(rows, ws)
    return off, idx, (w if wmax > 1 else None)


@pytest.fixture(scope="session")
def golden_traces():
    return load_golden("rak_traces.json")["cases"]
