"""COPRA (Sec. 3.3) on the GPU against the CPU oracle, through the C ABI:
every vertex's final set (labels and fixed-point belongings), the best
labels, the iteration count, the convergence flag and the per-iteration
changed counts are bit-exact, for rows whose tables fit shared memory and
rows that need the global tables, both tie rules, synchronous and
wave-ordered asynchronous updates and several max_labels."""
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


def copra_parity(lp, off, idx, w, max_labels=4, tolerance=0.0, max_iter=6, mode="sync",
                 waves=1, strict=True, seed=0):
    o_waves = waves if mode == "async" else 0
    ref_lab, ref_l, ref_b, it, conv, hist = oracle.copra(
        off, idx, w, max_labels=max_labels, tolerance=tolerance, max_iter=max_iter, mode=mode,
        waves=o_waves, strict=strict, seed=seed)
    with lp.Graph(off, idx, w) as G:
        r = G.copra(max_labels=max_labels, tolerance=tolerance, max_iter=max_iter, mode=mode,
                    waves=waves, strict=strict, seed=seed)
        assert r.iterations == it and bool(r.converged) == conv, (r.as_dict(), it, conv)
        assert np.array_equal(G.history(), hist)
        sl, sb = G.copra_sets()
        bad = np.nonzero((sb != ref_b).any(axis=1) | ((sl != ref_l) & (ref_b > 0)).any(axis=1))[0]
        assert bad.size == 0, f"{bad.size} sets differ, first at {bad[:5]}"
        assert np.array_equal(G.labels(), ref_lab)
        q = G.modularity()
    assert abs(q - oracle.modularity(off, idx, w, ref_lab)) <= 1e-9
    return r


SHAPES = ["small", "warp", "cta", "hub", "bighub", "mixed"]


def shape_graph(shape):
    if shape == "small":
        return random_graph(2000, 6 / 2000, 51, wmax=3)
    if shape == "warp":
        return random_graph(1500, 70 / 1500, 52, wmax=4)
    if shape == "cta":  # 300 entries x 8 labels: more pairs than the shared table holds
        return random_graph(2000, 300 / 2000, 53, wmax=3)
    if shape == "hub":
        return hub_graph(54, n=15_000, hubs=2, hub_deg=6_000)
    if shape == "bighub":  # rows with more labels than the long-row shared table holds
        return hub_graph(56, n=30_000, hubs=3, hub_deg=9_000)
    g = gg.rmat(13, seed=55)
    return g.offsets, g.indices, g.weights


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("max_labels", [1, 4, 8, 16])
def test_copra_sync_parity(lp, shape, max_labels):
    off, idx, w = shape_graph(shape)
    copra_parity(lp, off, idx, w, max_labels=max_labels, mode="sync", max_iter=5)


@pytest.mark.parametrize("shape", ["small", "cta", "bighub", "mixed"])
@pytest.mark.parametrize("strict", [True, False])
def test_copra_async_parity(lp, shape, strict):
    off, idx, w = shape_graph(shape)
    copra_parity(lp, off, idx, w, max_labels=4, mode="async", waves=3, strict=strict, seed=7,
                 max_iter=5)


def test_copra_sequential_order_and_convergence(lp):
    g = gg.sbm_planted(1500, 6, 0.03, 0.001, seed=3)
    r = copra_parity(lp, g.offsets, g.indices, g.weights, max_labels=4, mode="async",
                     waves=g.n, tolerance=0.01, max_iter=30)
    assert r.converged


def test_copra_edge_cases_and_errors(lp):
    off, idx, w = csr_from_adj([[1, 2], [0, 2], [0, 1], [], [5], [4]])
    copra_parity(lp, off, idx, w, max_labels=2, max_iter=4)
    g = gg.rmat(9, seed=2)
    with lp.Graph(g.offsets, g.indices, g.weights) as G:
        with pytest.raises(lp.LPError):
            G.copra_sets()  # no run yet
        for bad in (dict(max_labels=0), dict(max_labels=65), dict(tolerance=-0.1),
                    dict(max_iter=0), dict(mode="async", waves=0)):
            with pytest.raises(lp.LPError):
                G.copra(**bad)


@pytest.mark.slow
def test_copra_rmat20(lp):
    g = gg.rmat(20, seed=1)
    copra_parity(lp, g.offsets, g.indices, g.weights, max_labels=4, mode="async", waves=2,
                 tolerance=0.01, max_iter=4)


@pytest.mark.parametrize("shape", ["small", "mixed"])
@pytest.mark.parametrize("mode", ["sync", "async"])
def test_copra_more_labels_than_a_warp(lp, shape, mode):
    # max_labels above 32: every row (rows without entries included) takes a CTA
    off, idx, w = shape_graph(shape)
    copra_parity(lp, off, idx, w, max_labels=40, mode=mode, waves=3, max_iter=4, strict=False,
                 seed=5)


@pytest.mark.parametrize("strict", [True, False])
@pytest.mark.parametrize("waves", [31, 4000])
def test_copra_many_waves_of_short_rows(lp, strict, waves):
    # k-mer-like paths (at most 32 pairs per row with 4 labels: the 8-lane
    # kernel) and many waves, later waves reading the sets earlier waves wrote;
    # with 16 labels the same rows take a listed warp each
    g = gg.kmer_like(4000, mean_path=50, branch_frac=0.05, seed=9)
    assert int(np.diff(g.offsets).max()) * 4 <= 32
    copra_parity(lp, g.offsets, g.indices, g.weights, max_labels=4, mode="async", waves=waves,
                 strict=strict, seed=3, max_iter=6)
    copra_parity(lp, g.offsets, g.indices, g.weights, max_labels=16, mode="async", waves=waves,
                 strict=strict, seed=3, max_iter=6)
