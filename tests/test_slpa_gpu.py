"""SLPA (Sec. 3.4) on the GPU against the CPU oracle, through the C ABI: the
whole memory (every filled slot), the communities, the iteration count, the
convergence flag and the per-iteration changed counts are bit-exact, for
rows of every degree bucket and both tie rules; modularity of the
communities within 1e-9."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from conftest import csr_from_adj, random_graph
from test_rak_gpu import hub_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lp():
    import torch

    import __graft_entry__

    assert torch.cuda.is_available()
    __graft_entry__.build()
    import paper_2301_09125_gb300 as lp

    return lp


def slpa_parity(lp, off, idx, w, memory_size=8, tolerance=0.0, strict=True, seed=0):
    ref_lab, ref_mem, ref_it, ref_conv, ref_hist = oracle.slpa(
        off, idx, w, memory_size=memory_size, tolerance=tolerance, strict=strict, seed=seed)
    with lp.Graph(off, idx, w) as G:
        r = G.slpa(memory_size=memory_size, tolerance=tolerance, strict=strict, seed=seed)
        assert r.iterations == ref_it and bool(r.converged) == ref_conv, (r.as_dict(), ref_it)
        mem = G.slpa_memory(ref_it + 1)
        for t in range(ref_it + 1):
            bad = np.nonzero(mem[t] != ref_mem[t])[0]
            assert bad.size == 0, f"slot {t}: {bad.size} vertices differ, first {bad[:5]}"
        assert np.array_equal(G.history(), ref_hist)
        assert np.array_equal(G.labels(), ref_lab)
        q = G.modularity()
    assert abs(q - oracle.modularity(off, idx, w, ref_lab)) <= 1e-9
    return r


@pytest.mark.parametrize("strict", [True, False])
@pytest.mark.parametrize("shape", ["small", "warp", "cta", "cta2", "hub", "mixed"])
def test_slpa_parity_per_bucket(lp, shape, strict):
    if shape == "small":
        off, idx, w = random_graph(3000, 6 / 3000, 31, wmax=3)
    elif shape == "warp":
        off, idx, w = random_graph(2000, 70 / 2000, 32, wmax=4)
    elif shape == "cta":
        off, idx, w = random_graph(2500, 300 / 2500, 33, wmax=3)
    elif shape == "cta2":
        off, idx, w = random_graph(2000, 800 / 2000, 34, wmax=4)
    elif shape == "hub":
        off, idx, w = hub_graph(35, n=20_000, hubs=2, hub_deg=7_000)
    else:
        g = gg.rmat(14, seed=36)
        off, idx, w = g.offsets, g.indices, g.weights
    slpa_parity(lp, off, idx, w, memory_size=8, tolerance=0.0, strict=strict, seed=5)


def test_slpa_converges_like_the_oracle(lp):
    g = gg.sbm_planted(3000, 10, 0.03, 0.001, seed=4)
    r = slpa_parity(lp, g.offsets, g.indices, g.weights, memory_size=20, tolerance=0.05, seed=2)
    assert r.iterations >= 1


def test_slpa_edge_cases(lp):
    # memory of one slot: no iteration, every vertex its own community
    g = gg.rmat(10, seed=7)
    with lp.Graph(g.offsets, g.indices, g.weights) as G:
        r = G.slpa(memory_size=1)
        assert r.iterations == 0 and not r.converged
        assert np.array_equal(G.labels(), np.arange(g.n))
        assert np.array_equal(G.slpa_memory(1)[0], np.arange(g.n))
        with pytest.raises(lp.LPError):
            G.slpa_memory(2)
        for bad in (dict(memory_size=0), dict(memory_size=65), dict(tolerance=1.5)):
            with pytest.raises(lp.LPError):
                G.slpa(**bad)
    # isolated vertices repeat their slot; an empty graph
    off, idx, w = csr_from_adj([[1, 2], [0, 2], [0, 1], [], [5], [4]])
    slpa_parity(lp, off, idx, w, memory_size=6)
    empty = gg.CSR(np.zeros(1, np.int32), np.zeros(0, np.int32), None)
    with lp.Graph(empty.offsets, empty.indices, None) as G:
        r = G.slpa(memory_size=4)
        assert r.iterations >= 0


@pytest.mark.slow
def test_slpa_rmat22(lp):
    g = gg.workload("rmat22")
    slpa_parity(lp, g.offsets, g.indices, g.weights, memory_size=6, tolerance=0.05, seed=1)
