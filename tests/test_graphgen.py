"""Structure checks of the seeded synthetic inputs (CPU)."""
import numpy as np
import pytest

import graphgen as gg


def check_symmetric_simple(g):
    n, off, idx = g.n, g.offsets, g.indices
    assert off[0] == 0 and off[-1] == g.m and np.all(np.diff(off) >= 0)
    assert idx.size == 0 or (idx.min() >= 0 and idx.max() < n)
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    assert not np.any(src == idx), "self-loop"
    key = src * n + idx
    # rows sorted strictly ascending -> no duplicates
    same_row = src[1:] == src[:-1]
    assert np.all(idx[1:][same_row] > idx[:-1][same_row])
    rkey = idx.astype(np.int64) * n + src
    order = np.argsort(key)
    rorder = np.argsort(rkey)
    assert np.array_equal(key[order], rkey[rorder]), "not symmetric"
    if g.weights is not None:
        assert np.array_equal(g.weights[order], g.weights[rorder]), "weights not symmetric"


def test_sbm_planted_shape_and_determinism():
    g = gg.workload("sbm10k")
    check_symmetric_simple(g)
    assert g.weights is None
    # expected entries 2 * (sum of p over pairs): blocks of 500
    exp = 2 * (20 * 500 * 499 / 2 * 0.02 + (10000 * 9999 / 2 - 20 * 500 * 499 / 2) * 0.0005)
    assert abs(g.m - exp) < 6 * np.sqrt(exp)
    g2 = gg.workload("sbm10k")
    assert np.array_equal(g.indices, g2.indices)
    g3 = gg.workload("sbm10k", seed=2)
    assert not np.array_equal(g.indices, g3.indices)
    # inside-block share ~ p_in part
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    inside = np.mean(src // 500 == g.indices // 500)
    assert 0.6 < inside < 0.75


def test_rmat_small():
    g = gg.rmat(12, edge_factor=16, seed=3)
    check_symmetric_simple(g)
    assert g.n == 4096
    assert g.weights.min() >= 1 and g.weights.max() <= 4
    d = np.diff(g.offsets)
    assert d.max() > 20 * d.mean()  # heavy tail
    assert np.array_equal(gg.rmat(12, seed=3).indices, g.indices)


def test_grid_road_small():
    side = 64
    g = gg.grid_road(side, seed=5)
    check_symmetric_simple(g)
    assert g.n == side * side
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    dr = np.abs(src // side - g.indices // side)
    dc = np.abs(src % side - g.indices % side)
    assert np.all(np.maximum(dr, dc) <= 8)
    grid_entries = 2 * 2 * side * (side - 1)
    assert abs(np.sum(dr + dc == 1) / grid_entries - 0.85) < 0.03
    assert g.weights.min() >= 1 and g.weights.max() <= 16
    assert 3.0 < g.m / g.n < 3.8


def test_kmer_and_mixing():
    g = gg.kmer_like(50_000, seed=2)
    check_symmetric_simple(g)
    assert 1.9 < g.m / g.n < 2.3
    g = gg.sbm_mixing(20_000, 40, 16.0, 0.3, seed=4)
    check_symmetric_simple(g)
    assert abs(g.m / g.n - 16.0) < 0.5


def test_batch_params():
    ps = gg.batch_sbm_params(count=256, seed=1000)
    ns = np.array([p["n"] for p in ps])
    assert ns.min() >= 1000 and ns.max() <= 200_000
    assert all(p["k"] <= max(1, p["n"] / (2 * p["avg_degree"])) for p in ps)
    assert ps == gg.batch_sbm_params(count=256, seed=1000)


def test_rejects_bad_parameters():
    with pytest.raises(ValueError):
        gg.rmat(0)
    with pytest.raises(ValueError):
        gg.sbm_planted(10, 0, 0.1, 0.1)


def test_with_self_loops_appends_one_loop_per_row():
    g = gg.sbm_planted(300, 3, 0.05, 0.01, seed=4)
    s = gg.with_self_loops(g, weight=2)
    assert s.n == g.n and s.m == g.m + g.n
    assert np.array_equal(np.diff(s.offsets), np.diff(g.offsets) + 1)
    for v in (0, 17, 299):
        row = s.indices[s.offsets[v]:s.offsets[v + 1]]
        w = s.weights[s.offsets[v]:s.offsets[v + 1]]
        assert row[-1] == v and w[-1] == 2
        assert np.array_equal(row[:-1], g.indices[g.offsets[v]:g.offsets[v + 1]])
        assert (w[:-1] == 1).all()

