"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

* synchronous mode and asynchronous mode with W waves (strict and
  non-strict): labels, iteration count, convergence flag and per-iteration
  changed counts are bit-exact against the oracle run with the same W;
* asynchronous mode against the oracle's plain in-place ascending order
  (every vertex its own wave): on the R-MAT and road configurations the run
  must converge with modularity within 1e-2 of the oracle's;
* modularity: within 1e-9 of the oracle for the same labels.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from conftest import csr_from_adj, random_graph

pytestmark = pytest.mark.gpu

Q_SYNC_TOL = 1e-9
Q_ASYNC_TOL = 1e-2


@pytest.fixture(scope="module")
def lp():
    import torch

    import __graft_entry__

    assert torch.cuda.is_available()
    __graft_entry__.build()
    import paper_2301_09125_gb300 as lp

    return lp


def gpu_run(lp, off, idx, w, **kw):
    with lp.Graph(off, idx, w) as G:
        r = G.rak(**kw)
        return G.labels(), r, G.history(), G.modularity()


def assert_sync_parity(lp, off, idx, w, strict=True, seed=0, tol=0.05, max_iter=20):
    labels, r, hist, q = gpu_run(lp, off, idx, w, tolerance=tol, max_iter=max_iter,
                                 mode="sync", strict=strict, seed=seed)
    ref, iters, conv, ref_hist = oracle.rak(off, idx, w, tol, max_iter, "sync", strict=strict,
                                            seed=seed)
    assert r.iterations == iters
    assert bool(r.converged) == conv
    assert np.array_equal(hist, ref_hist)
    mism = np.nonzero(labels != ref)[0]
    assert mism.size == 0, f"{mism.size} labels differ, first at vertex {mism[:5]}"
    assert r.last_changed == ref_hist[-1]
    assert abs(q - oracle.modularity(off, idx, w, ref)) <= Q_SYNC_TOL
    return r


def assert_async_parity(lp, off, idx, w, waves, strict=True, seed=0, tol=0.05, max_iter=20):
    labels, r, hist, q = gpu_run(lp, off, idx, w, tolerance=tol, max_iter=max_iter,
                                 mode="async", strict=strict, seed=seed, waves=waves)
    ref, iters, conv, ref_hist = oracle.rak(off, idx, w, tol, max_iter, "async", strict=strict,
                                            seed=seed, waves=waves)
    assert r.iterations == iters and bool(r.converged) == conv
    assert np.array_equal(hist, ref_hist)
    mism = np.nonzero(labels != ref)[0]
    assert mism.size == 0, f"{mism.size} labels differ, first at vertex {mism[:5]}"
    assert abs(q - oracle.modularity(off, idx, w, ref)) <= Q_SYNC_TOL
    return labels, r, q


def assert_async_quality(lp, off, idx, w, waves=31, tol=0.05, max_iter=20, strict=True, seed=0):
    """Converged, with modularity within 1e-2 of the oracle's plain in-place
    ascending-order run (every vertex its own wave)."""
    labels, r, hist, q = gpu_run(lp, off, idx, w, tolerance=tol, max_iter=max_iter,
                                 mode="async", strict=strict, seed=seed, waves=waves)
    n = off.shape[0] - 1
    assert labels.min() >= 0 and labels.max() < n
    ref, iters, conv, _ = oracle.rak(off, idx, w, tol, max_iter, "async", strict=strict, seed=seed)
    q_ref = oracle.modularity(off, idx, w, ref)
    assert abs(q - oracle.modularity(off, idx, w, labels)) <= Q_SYNC_TOL
    assert conv and r.converged, (r.as_dict(), iters)
    assert abs(q - q_ref) <= Q_ASYNC_TOL, (q, q_ref)
    return q, q_ref


# ---------------------------------------------------------------- hand-derived traces
def test_golden_traces_sync(lp, golden_traces):
    for case in golden_traces:
        if case["mode"] != "sync":
            continue
        off, idx, w = csr_from_adj(case["adj"], case.get("w"))
        with lp.Graph(off, idx, w) as G:
            r = G.rak(tolerance=case["tolerance"], max_iter=case["max_iter"], mode="sync",
                      init_labels=case.get("init") and np.array(case["init"], np.int32))
            assert G.labels().tolist() == case["labels"], case["name"]
            assert r.iterations == case["iterations"], case["name"]
            assert bool(r.converged) == case["converged"], case["name"]
            assert G.history().tolist() == case["changed"], case["name"]
            if "modularity" in case:
                assert abs(G.modularity() - case["modularity"]) <= 1e-15


def test_golden_traces_async(lp, golden_traces):
    for case in golden_traces:
        if case["mode"] != "async":
            continue
        off, idx, w = csr_from_adj(case["adj"], case.get("w"))
        # waves 0 in a trace = every vertex its own wave: any W >= n
        waves = case.get("waves", 0) or 4096
        with lp.Graph(off, idx, w) as G:
            r = G.rak(tolerance=case["tolerance"], max_iter=case["max_iter"], mode="async",
                      waves=waves)
            assert G.labels().tolist() == case["labels"], case["name"]
            assert r.iterations == case["iterations"], case["name"]
            assert bool(r.converged) == case["converged"], case["name"]
            assert G.history().tolist() == case["changed"], case["name"]


# ---------------------------------------------------------------- every degree bucket
def hub_graph(seed, n=40_000, hubs=3, hub_deg=12_000, p_extra=0.0002, sorted_rows=False):
    """A sparse random graph plus `hubs` vertices of degree ~hub_deg, so hub
    rows are longer than 4096 entries (swept by CTA clusters).  Rows are
    shuffled unless sorted_rows (sorted rows enable the identity first
    sweep)."""
    rng = np.random.default_rng(seed)
    m_rand = int(p_extra * n * n / 2)
    u = rng.integers(0, n, m_rand)
    v = rng.integers(0, n, m_rand)
    hu = [np.full(hub_deg, h) for h in range(hubs)]
    hv = [rng.choice(np.arange(hubs, n), hub_deg, replace=False) for _ in range(hubs)]
    u = np.concatenate([u] + hu)
    v = np.concatenate([v] + hv)
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.unique(np.stack([np.minimum(u, v), np.maximum(u, v)], 1), axis=0)
    src = np.concatenate([a[:, 0], a[:, 1]])
    dst = np.concatenate([a[:, 1], a[:, 0]])
    perm = rng.permutation(src.size)  # shuffled rows: adjacency order matters
    src, dst = src[perm], dst[perm]
    if sorted_rows:
        order = np.lexsort((dst, src))
        src, dst = src[order], dst[order]
    order = np.argsort(src, kind="stable")
    src, dst = src[order], dst[order]
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off).astype(np.int32)
    pair_w = (a[:, 0] * 7919 + a[:, 1] * 104729) % 5 + 1
    wmap = dict(zip(map(tuple, a.tolist()), pair_w.tolist()))
    w = np.array([wmap[(min(x, y), max(x, y))] for x, y in zip(src.tolist(), dst.tolist())],
                 np.int32)
    return off, dst.astype(np.int32), w


@pytest.mark.parametrize("strict", [True, False])
@pytest.mark.parametrize("shape", ["small", "warp", "cta", "cta2", "hub", "mixed"])
def test_sync_parity_per_bucket(lp, shape, strict):
    if shape == "small":
        off, idx, w = random_graph(3000, 6 / 3000, 1, wmax=3)
    elif shape == "warp":
        off, idx, w = random_graph(1500, 70 / 1500, 2, wmax=1)
    elif shape == "cta":
        off, idx, w = random_graph(2500, 400 / 2500, 3, wmax=4)
    elif shape == "cta2":
        off, idx, w = random_graph(2000, 800 / 2000, 13, wmax=4)
    elif shape == "hub":
        off, idx, w = hub_graph(4)
    else:
        g = gg.rmat(15, seed=5)
        off, idx, w = g.offsets, g.indices, g.weights
    deg = np.diff(off)
    assert deg.max() > {"small": 8, "warp": 33, "cta": 129, "cta2": 513, "hub": 8192,
                        "mixed": 1024}[shape]
    assert_sync_parity(lp, off, idx, w, strict=strict, seed=11)


@pytest.mark.parametrize("strict", [True, False])
def test_tiny_rows_with_ties(lp, strict):
    """Rows of at most 8 entries take one lane each: unit weights make most
    label totals tie, and the degrees straddle the 8-entry boundary."""
    off, idx, w = random_graph(4000, 4 / 4000, 21)
    deg = np.diff(off)
    assert (deg == 1).any() and (deg == 8).any() and (deg > 8).any()
    assert_sync_parity(lp, off, idx, w, strict=strict, seed=4)
    assert_async_parity(lp, off, idx, w, 3, strict=strict, seed=4)


def test_batch_of_tiny_row_graphs(lp):
    """Graph sets of road grids and k-mer paths (every row has at most 8
    entries): per-graph change counts and labels as run one by one."""
    graphs = [gg.grid_road(48 + 16 * i, seed=i) for i in range(5)]
    graphs += [gg.kmer_like(3000 + 1000 * i, seed=i) for i in range(5)]
    assert all(np.diff(g.offsets).max() <= 8 for g in graphs)
    triples = [(g.offsets, g.indices, g.weights) for g in graphs]
    h = lp.lp_batch_create(triples)
    try:
        for mode, waves, strict in (("sync", None, True), ("sync", None, False),
                                    ("async", 3, True), ("async", 3, False)):
            kw = {} if waves is None else {"waves": waves}
            res = lp.lp_batch_run(h, len(graphs), tolerance=0.05, max_iter=20, mode=mode,
                                  strict=strict, seed=6, **kw)
            for i, g in enumerate(graphs):
                lab = lp.lp_batch_labels_get(h, i, g.n)
                ref, iters, conv, hist = oracle.rak(g.offsets, g.indices, g.weights, 0.05, 20,
                                                    mode, strict=strict, seed=6, **kw)
                assert res[i].iterations == iters and bool(res[i].converged) == conv, i
                assert res[i].last_changed == hist[-1], i
                assert np.array_equal(lab, ref), (mode, strict, i)
    finally:
        lp.lp_batch_destroy(h)


@pytest.mark.parametrize("strict", [True, False])
def test_identity_first_sweep_cluster_rows(lp, strict):
    """Sorted rows without repeats: the first sweep takes the identity path,
    including rows swept by CTA clusters; sync and 2-wave async stay exact."""
    off, idx, w = hub_graph(9, n=30_000, hubs=4, hub_deg=13_000, sorted_rows=True)
    assert np.all(np.diff(idx)[np.diff(np.repeat(np.arange(off.size - 1), np.diff(off))) == 0] > 0)
    assert_sync_parity(lp, off, idx, w, strict=strict, seed=4)
    assert_async_parity(lp, off, idx, w, 2, strict=strict, seed=4)


@pytest.mark.parametrize("strict", [True, False])
@pytest.mark.parametrize("mode", ["sync", "async"])
def test_cluster_rows_overflow_tables(lp, strict, mode):
    """Rows longer than 4096 entries are swept by CTA clusters.  From distinct
    shuffled labels, two rows of 150k entries hold more distinct labels than
    the cluster's shared tables keep within their probe windows, so part of
    them go through the rows' global overflow tables.  Labels and changed
    counts match the oracle for three sweeps (2-wave async in async mode)."""
    off, idx, w = hub_graph(21, n=200_000, hubs=2, hub_deg=150_000, p_extra=2e-5)
    n = off.shape[0] - 1
    init = np.random.default_rng(5).permutation(n).astype(np.int32)
    waves = 2 if mode == "async" else 0
    kw = dict(waves=waves) if waves else {}
    with lp.Graph(off, idx, w) as G:
        r = G.rak(tolerance=0.0, max_iter=3, mode=mode, strict=strict, seed=5, init_labels=init,
                  **kw)
        labels, hist = G.labels(), G.history()
    ref, iters, conv, ref_hist = oracle.rak(off, idx, w, 0.0, 3, mode, strict=strict, seed=5,
                                            init_labels=init, waves=waves)
    assert r.iterations == iters == 3
    assert np.array_equal(hist, ref_hist)
    mism = np.nonzero(labels != ref)[0]
    assert mism.size == 0, f"{mism.size} labels differ, first at vertex {mism[:5]}"


@pytest.mark.parametrize("waves", [2, 7, 31, 4096])
@pytest.mark.parametrize("shape", ["small", "cta", "cta2", "hub", "mixed"])
def test_async_parity_per_bucket(lp, shape, waves):
    if shape == "small":
        off, idx, w = random_graph(3000, 6 / 3000, 5, wmax=3)
    elif shape == "cta":
        off, idx, w = random_graph(2500, 300 / 2500, 6, wmax=4)
    elif shape == "cta2":
        off, idx, w = random_graph(2000, 700 / 2000, 14, wmax=4)
    elif shape == "hub":
        off, idx, w = hub_graph(7, n=20_000, hub_deg=9_000)
    else:
        g = gg.rmat(14, seed=8)
        off, idx, w = g.offsets, g.indices, g.weights
    for strict in (True, False):
        assert_async_parity(lp, off, idx, w, waves, strict=strict, seed=3)


def test_async_one_wave_is_sync(lp):
    g = gg.rmat(13, seed=9)
    a = gpu_run(lp, g.offsets, g.indices, g.weights, mode="async", waves=1, tolerance=0.0,
                max_iter=6)
    b = gpu_run(lp, g.offsets, g.indices, g.weights, mode="sync", tolerance=0.0, max_iter=6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])


def test_sync_parity_unit_weights_and_tolerances(lp):
    g = gg.sbm_planted(5000, 25, 0.01, 0.001, seed=3)
    for tol in (0.0, 0.01, 0.05, 0.3, 1.0):
        assert_sync_parity(lp, g.offsets, g.indices, g.weights, tol=tol, max_iter=30)


# ---------------------------------------------------------------- configuration shapes
def test_sbm10k_config(lp):
    g = gg.workload("sbm10k")
    r = assert_sync_parity(lp, g.offsets, g.indices, g.weights, strict=True)
    assert r.converged
    assert_sync_parity(lp, g.offsets, g.indices, g.weights, strict=False, seed=1)
    assert_async_parity(lp, g.offsets, g.indices, g.weights, 31)


def test_rmat_and_road_small(lp):
    g = gg.rmat(16, seed=2)
    assert_sync_parity(lp, g.offsets, g.indices, g.weights)
    assert_async_parity(lp, g.offsets, g.indices, g.weights, 31)
    assert_async_parity(lp, g.offsets, g.indices, g.weights, 2)
    assert_async_quality(lp, g.offsets, g.indices, g.weights, waves=2)
    g = gg.grid_road(512, seed=2)
    assert_sync_parity(lp, g.offsets, g.indices, g.weights)
    assert_async_parity(lp, g.offsets, g.indices, g.weights, 31)
    assert_async_quality(lp, g.offsets, g.indices, g.weights, waves=31)
    g = gg.kmer_like(200_000, seed=2)
    assert_sync_parity(lp, g.offsets, g.indices, g.weights)


@pytest.mark.parametrize("waves", [8, 127])
def test_all_waves_launch_parity(lp, waves):
    """Asynchronous runs of 8 or more waves over rows of at most 32 entries
    sweep every wave of an iteration in one cooperative launch with grid
    barriers (rows of at most 8 entries: the kernel that loads the next
    wave's rows before each barrier): labels bit-exact with the oracle, also
    when resumed."""
    g = gg.kmer_like(120_000, seed=4)
    for strict in (True, False):
        labels, r, q = assert_async_parity(lp, g.offsets, g.indices, g.weights, waves,
                                           strict=strict, seed=3)
    g = gg.sbm_mixing(20_000, 40, 14.0, 0.3, seed=6, wmin=1, wmax=4)  # rows of up to 32 entries
    assert 8 < int(np.diff(g.offsets).max()) <= 32
    for strict in (True, False):
        assert_async_parity(lp, g.offsets, g.indices, g.weights, waves, strict=strict, seed=5)
    g = gg.grid_road(256, seed=5)
    assert_async_parity(lp, g.offsets, g.indices, g.weights, waves, strict=False, seed=2)
    # two iterations, then a resumed run from those labels
    ref1, _, _, _ = oracle.rak(g.offsets, g.indices, g.weights, 0.0, 2, "async", seed=2,
                               waves=waves)
    ref2, _, _, _ = oracle.rak(g.offsets, g.indices, g.weights, 0.0, 2, "async", seed=2,
                               waves=waves, iter_offset=2, init_labels=ref1)
    lab, r, _, _ = gpu_run(lp, g.offsets, g.indices, g.weights, tolerance=0.0, max_iter=2,
                           mode="async", seed=2, waves=waves, iter_offset=2, init_labels=ref1)
    assert np.array_equal(lab, ref2)


def test_grid_barrier_wait_is_bounded(lp):
    """The all-waves sweep's grid barrier gives up after its poll limit: a
    barrier that waits for a CTA that does not exist reports the timeout, and
    the context keeps working afterwards."""
    assert lp.lp_selftest_barrier_timeout()
    g = gg.kmer_like(20_000, seed=1)
    assert_async_parity(lp, g.offsets, g.indices, g.weights, 16)


def test_self_loop_variant_parity(lp):
    """Graphs with a self-loop on every vertex (the paper's inputs, Sec. 3.1)
    through the same path: labels bit-exact with the oracle."""
    g = gg.with_self_loops(gg.rmat(13, seed=6))
    assert_sync_parity(lp, g.offsets, g.indices, g.weights, strict=False, seed=2)
    assert_async_parity(lp, g.offsets, g.indices, g.weights, 2)
    g = gg.with_self_loops(gg.grid_road(128, seed=3), weight=3)
    assert_async_parity(lp, g.offsets, g.indices, g.weights, 16)


def test_async_wave_counts_of_the_benchmarks(lp):
    """The wave counts the benchmarks use keep modularity within 1e-2 of the
    sequential in-place order: 3 waves on the road grid (coprime with its
    power-of-two width, so vertical neighbours update in different waves) and
    127 waves on the k-mer paths (random neighbour ids)."""
    g = gg.grid_road(1024, seed=2)
    assert_async_quality(lp, g.offsets, g.indices, g.weights, waves=3)
    g = gg.kmer_like(1 << 20, seed=2)
    assert_async_quality(lp, g.offsets, g.indices, g.weights, waves=127)


# ---------------------------------------------------------------- modularity
@pytest.mark.parametrize("seed", range(4))
def test_modularity_parity(lp, seed):
    rng = np.random.default_rng(seed)
    off, idx, w = random_graph(int(rng.integers(50, 3000)), 0.02, seed, wmax=7,
                               self_loops=bool(seed % 2))
    n = off.shape[0] - 1
    with lp.Graph(off, idx, w) as G:
        for k in (1, 3, n // 7 + 1, n):
            lab = rng.integers(0, k, n).astype(np.int32)
            q = G.modularity(lab)
            assert abs(q - oracle.modularity(off, idx, w, lab)) <= Q_SYNC_TOL


def test_modularity_large_exact(lp):
    g = gg.rmat(18, seed=9)
    rng = np.random.default_rng(1)
    lab = rng.integers(0, 1000, g.n).astype(np.int32)
    with lp.Graph(g.offsets, g.indices, g.weights) as G:
        assert G.modularity(lab) == oracle.modularity(g.offsets, g.indices, g.weights, lab)


# ---------------------------------------------------------------- edge cases and resume
def test_edge_cases(lp):
    # empty graph
    off = np.zeros(1, np.int32)
    labels, r, hist, q = gpu_run(lp, off, np.zeros(0, np.int32), None)
    assert labels.size == 0 and r.iterations == 1 and r.converged and q == 0.0
    # vertices without edges
    off = np.zeros(6, np.int32)
    labels, r, hist, q = gpu_run(lp, off, np.zeros(0, np.int32), None)
    assert labels.tolist() == [0, 1, 2, 3, 4] and r.iterations == 1 and hist.tolist() == [0]
    # a self-loop only
    off, idx, w = csr_from_adj([[0], []], [[3], []])
    labels, r, hist, q = gpu_run(lp, off, idx, w)
    assert labels.tolist() == [0, 1] and q == 0.0
    # duplicates, self-loops, maximum-degree row of 32 / 33 / 128 / 129 / 1024 / 1025
    for d in (31, 32, 33, 128, 129, 1024, 1025):
        rows = [[(v + k) % (d + 1) for k in range(1, d + 1)] for v in range(d + 1)]
        rows[0] = rows[0] + [0, 1, 1]
        off, idx, _ = csr_from_adj(rows)
        assert_sync_parity(lp, off, idx, None, max_iter=5)


@pytest.mark.parametrize("mode_strict", [("sync", True), ("sync", False)])
def test_resume_is_bit_exact(lp, mode_strict):
    mode, strict = mode_strict
    g = gg.rmat(14, seed=4)
    with lp.Graph(g.offsets, g.indices, g.weights) as G:
        G.rak(tolerance=0.0, max_iter=6, mode=mode, strict=strict, seed=5)
        full = G.labels().copy()
        G.rak(tolerance=0.0, max_iter=3, mode=mode, strict=strict, seed=5)
        mid = G.labels().copy()
        G.rak(tolerance=0.0, max_iter=3, mode=mode, strict=strict, seed=5, iter_offset=3,
              init_labels=mid)
        assert np.array_equal(G.labels(), full)


def test_invalid_inputs_are_rejected(lp):
    off, idx, w = csr_from_adj([[1], [0]])
    bad = [
        (np.array([1, 1, 2], np.int32), idx, None, "offsets\\[0\\]"),
        (np.array([0, 2, 1], np.int32), idx[:1], None, "non-decreasing"),
        (np.array([0, 1, 3], np.int32), np.array([1, 0, 0], np.int32)[:2], None, "offsets\\[n\\]"),
        (off, np.array([1, 2], np.int32), None, "column index"),
        (off, np.array([1, -1], np.int32), None, "column index"),
        (off, idx, np.array([1, 0], np.int32), "weight"),
    ]
    for o, i, ww, msg in bad:
        with pytest.raises(lp.LPError, match=msg):
            lp.Graph(o, i, ww)
    with pytest.raises(lp.LPError, match="symmetric"):
        lp.Graph(*csr_from_adj([[1], []]), check_symmetric=True)
    big = np.array([0, 2, 4], np.int32)
    with pytest.raises(lp.LPError, match="2\\^31"):
        lp.Graph(big, np.array([1, 1, 0, 0], np.int32),
                 np.array([2**30, 2**30, 1, 1], np.int32))
    with lp.Graph(off, idx, None) as G:
        with pytest.raises(lp.LPError, match="label"):
            G.modularity(np.array([0, 2], np.int32))
        with pytest.raises(lp.LPError, match="label"):
            G.rak(init_labels=np.array([5, 0], np.int32))
        with pytest.raises(lp.LPError, match="tolerance"):
            G.rak(tolerance=1.5)
        with pytest.raises(lp.LPError, match="max_iter"):
            G.rak(max_iter=0)
        r = G.rak()  # still usable
        assert r.iterations >= 1


def test_device_pointers_and_borrow(lp):
    import torch

    g = gg.rmat(14, seed=6)
    ref, iters, _, _ = oracle.rak(g.offsets, g.indices, g.weights, 0.05, 20, "sync")
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (g.offsets, g.indices, g.weights)]
    for borrow in (False, True):
        with lp.Graph(*t, borrow=borrow) as G:
            r = G.rak()
            out = torch.empty(g.n, dtype=torch.int32, device=dev)
            G.labels(out)
            assert np.array_equal(out.cpu().numpy(), ref) and r.iterations == iters
            q = G.modularity(out)
            assert abs(q - oracle.modularity(g.offsets, g.indices, g.weights, ref)) <= Q_SYNC_TOL


# ---------------------------------------------------------------- batches
def test_batch_matches_single_graph_runs(lp):
    params = gg.batch_sbm_params(count=40, seed=77, n_lo=200, n_hi=6000)
    graphs = gg.batch_sbm(params)
    graphs[3] = gg.rmat(12, seed=3)          # a weighted graph with hubs in the mix
    graphs[5] = gg.CSR(np.zeros(1, np.int32), np.zeros(0, np.int32), None)  # empty
    triples = [(g.offsets, g.indices, g.weights) for g in graphs]
    h = lp.lp_batch_create(triples)
    try:
        for strict in (True, False):
            res = lp.lp_batch_run(h, len(graphs), tolerance=0.05, max_iter=20, mode="sync",
                                  strict=strict, seed=2)
            for i, g in enumerate(graphs):
                lab = lp.lp_batch_labels_get(h, i, g.n)
                ref, iters, conv, hist = oracle.rak(g.offsets, g.indices, g.weights, 0.05, 20,
                                                    "sync", strict=strict, seed=2)
                assert res[i].iterations == iters and bool(res[i].converged) == conv, i
                assert res[i].last_changed == hist[-1]
                assert np.array_equal(lab, ref), i
                q = lp.lp_batch_modularity(h, i)
                assert abs(q - oracle.modularity(g.offsets, g.indices, g.weights, ref)) <= Q_SYNC_TOL
    finally:
        lp.lp_batch_destroy(h)


def test_batch_majority_policy_per_graph(lp):
    """Graph sets where the majority pre-pass runs for some graphs and not for
    others in the same launch: the pre-pass and the CTA kernels must agree on
    each graph's policy (a synchronous SBM oscillates, changing nearly every
    label, while the graphs with long rows settle)."""
    off, idx, w = hub_graph(9, n=20_000, hubs=2, hub_deg=6_000)
    graphs = [gg.CSR(off, idx, w)]
    off, idx, w = random_graph(2000, 800 / 2000, 14, wmax=4)       # cta2 rows
    graphs.append(gg.CSR(off, idx, w))
    off, idx, w = random_graph(2500, 300 / 2500, 15, wmax=3)       # cta rows
    graphs.append(gg.CSR(off, idx, w))
    graphs.append(gg.sbm_planted(3000, 6, 0.02, 0.0005, seed=3))     # oscillates in sync
    graphs.append(gg.rmat(13, seed=8))
    triples = [(g.offsets, g.indices, g.weights) for g in graphs]
    h = lp.lp_batch_create(triples)
    try:
        for mode, waves in (("sync", None), ("async", 2)):
            kw = {} if waves is None else {"waves": waves}
            res = lp.lp_batch_run(h, len(graphs), tolerance=0.0, max_iter=6, mode=mode,
                                  strict=True, seed=1, **kw)
            for i, g in enumerate(graphs):
                lab = lp.lp_batch_labels_get(h, i, g.n)
                ref, iters, conv, hist = oracle.rak(g.offsets, g.indices, g.weights, 0.0, 6,
                                                    mode, strict=True, seed=1, **kw)
                assert res[i].iterations == iters and res[i].last_changed == hist[-1], (mode, i)
                assert np.array_equal(lab, ref), (mode, i)
    finally:
        lp.lp_batch_destroy(h)


def test_graph_launch_and_host_loop_agree(lp):
    """A run that repeats the previous run's parameters is one CUDA graph
    launch (a conditional node per iteration, the tolerance test on the
    device); other runs, and every run while per-launch profiling is on, are
    driven by the host iteration by iteration.  Both give identical results,
    for a batch and for single graphs, also when a captured graph is replayed
    and when it is rebuilt for other parameters."""
    params = gg.batch_sbm_params(count=12, seed=91, n_lo=300, n_hi=4000)
    graphs = gg.batch_sbm(params)
    graphs[2] = gg.rmat(11, seed=4)
    triples = [(g.offsets, g.indices, g.weights) for g in graphs]

    def batch_run(mode, waves):
        h = lp.lp_batch_create(triples)
        try:
            out = []
            for rep in range(2):  # the second call reuses the captured graph
                res = lp.lp_batch_run(h, len(graphs), tolerance=0.02, max_iter=15, mode=mode,
                                      waves=waves, strict=False, seed=5)
                out.append([(r.iterations, r.converged, r.last_changed) for r in res] +
                           [lp.lp_batch_labels_get(h, i, g.n).tolist()
                            for i, g in enumerate(graphs)])
            assert out[0] == out[1]
            return out[0]
        finally:
            lp.lp_batch_destroy(h)

    for mode, waves in (("sync", 31), ("async", 3)):
        graph_mode = batch_run(mode, waves)
        lp.lp_profile_enable(True)
        try:
            host_loop = batch_run(mode, waves)
        finally:
            lp.lp_profile_enable(False)
        assert graph_mode == host_loop

    # single graph: a run repeating the previous run's parameters is captured
    # (first repeat) and replayed (later repeats); profiled runs are host-driven
    g = gg.rmat(13, seed=6)
    with lp.Graph(g.offsets, g.indices, g.weights) as G:
        for kw in (dict(mode="sync"), dict(mode="async", waves=2),
                   dict(mode="sync", tolerance=0.0, max_iter=4), dict(mode="sync")):
            runs = []
            for prof in (False, False, False, True):
                lp.lp_profile_enable(prof)
                try:
                    r = G.rak(**kw)
                finally:
                    lp.lp_profile_enable(False)
                runs.append((r.iterations, r.converged, r.last_changed, G.history().tolist(),
                             G.labels().tolist()))
            assert all(x == runs[0] for x in runs), kw

    # many waves over small rows: repeated runs stay on the host-launched
    # all-waves sweep (no captured graph) and repeat the oracle's result
    g = gg.kmer_like(60_000, seed=9)
    ref, iters, _, hist = oracle.rak(g.offsets, g.indices, g.weights, 0.05, 20, "async",
                                     seed=4, waves=31)
    with lp.Graph(g.offsets, g.indices, g.weights) as G:
        for _ in range(3):
            r = G.rak(tolerance=0.05, max_iter=20, mode="async", waves=31, seed=4)
            assert r.iterations == iters and np.array_equal(G.history(), hist)
            assert np.array_equal(G.labels(), ref)


@pytest.mark.parametrize("bounds", [(8, 64, 256, 1024), (16, 128, 512, 1024), (1, 1, 1, 1),
                                    (32, 32, 129, 513)])
def test_bucket_bounds_keep_parity(lp, bounds):
    """Any bucket bounds within the kernels' capacities give the oracle's
    labels (sync and 2-wave async), for a single graph and a batch."""
    g = gg.rmat(14, seed=17)
    with lp.Graph(g.offsets, g.indices, g.weights) as G:
        G.set_buckets(bounds)
        for mode, waves in (("sync", 0), ("async", 2)):
            kw = dict(waves=waves) if waves else {}
            r = G.rak(tolerance=0.05, max_iter=20, mode=mode, strict=False, seed=3, **kw)
            ref, iters, conv, hist = oracle.rak(g.offsets, g.indices, g.weights, 0.05, 20, mode,
                                                strict=False, seed=3, waves=waves)
            assert r.iterations == iters and np.array_equal(G.history(), hist)
            assert np.array_equal(G.labels(), ref)
    graphs = gg.batch_sbm(gg.batch_sbm_params(count=10, seed=55, n_lo=300, n_hi=3000))
    graphs[1] = gg.rmat(10, seed=8)
    h = lp.lp_batch_create([(x.offsets, x.indices, x.weights) for x in graphs])
    try:
        lp.lp_batch_set_buckets(h, bounds)
        res = lp.lp_batch_run(h, len(graphs), tolerance=0.05, max_iter=20, mode="sync")
        for i, x in enumerate(graphs):
            ref, iters, conv, _ = oracle.rak(x.offsets, x.indices, x.weights, 0.05, 20, "sync")
            assert res[i].iterations == iters
            assert np.array_equal(lp.lp_batch_labels_get(h, i, x.n), ref), i
    finally:
        lp.lp_batch_destroy(h)


def test_bucket_bounds_are_checked(lp):
    g = gg.rmat(8, seed=1)
    with lp.Graph(g.offsets, g.indices, g.weights) as G:
        for bad in ((0, 64, 256, 1024), (33, 64, 256, 1024), (16, 8, 256, 1024),
                    (16, 129, 256, 1024), (16, 64, 513, 1024), (16, 64, 256, 1025)):
            with pytest.raises(lp.LPError):
                G.set_buckets(bad)


def test_autotune_then_run_matches_oracle(lp):
    """The autotuner times 16 bucket choices and keeps the fastest; runs
    after it still give the oracle's results."""
    graphs = gg.batch_sbm(gg.batch_sbm_params(count=16, seed=66, n_lo=500, n_hi=5000))
    h = lp.lp_batch_create([(x.offsets, x.indices, x.weights) for x in graphs])
    try:
        t = lp.lp_batch_autotune(h, sweeps=3, mode="sync")
        assert t.candidates == 16 and t.best_ms <= t.default_ms
        assert 1 <= t.small_max <= 32 and t.small_max <= t.warp_max <= 128
        assert t.warp_max <= t.cta_max <= 512 and t.cta_max <= t.cta2_max <= 1024
        res = lp.lp_batch_run(h, len(graphs), tolerance=0.05, max_iter=20, mode="sync")
        for i, x in enumerate(graphs):
            ref, iters, conv, _ = oracle.rak(x.offsets, x.indices, x.weights, 0.05, 20, "sync")
            assert res[i].iterations == iters
            assert np.array_equal(lp.lp_batch_labels_get(h, i, x.n), ref), i
    finally:
        lp.lp_batch_destroy(h)
    g = gg.rmat(13, seed=23)
    with lp.Graph(g.offsets, g.indices, g.weights) as G:
        t = G.autotune(sweeps=3, mode="async", waves=2)
        assert t.candidates == 16
        G.rak(tolerance=0.05, max_iter=20, mode="async", waves=2)
        ref, _, _, _ = oracle.rak(g.offsets, g.indices, g.weights, 0.05, 20, "async", waves=2)
        assert np.array_equal(G.labels(), ref)


# ---------------------------------------------------------------- full-size workloads
# (synchronous parity and asynchronous quality at full size: test_fullsize_gpu.py)
@pytest.fixture(scope="module")
def rmat22():
    return gg.workload("rmat22")


@pytest.fixture(scope="module")
def road4096():
    return gg.workload("road4096")


# ------------------------------------------------- splitting disconnected communities
def split_check(lp, g, mode, waves=None, strict=True, max_iter=20, init=None, tol=0.05):
    kw = {} if waves is None else {"waves": waves}
    ref, _, _, _ = oracle.rak(g.offsets, g.indices, g.weights, tol, max_iter, mode,
                              strict=strict, seed=4, init_labels=init, **kw)
    ref_split, k_ref = oracle.split(g.offsets, g.indices, ref)
    with lp.Graph(g.offsets, g.indices, g.weights) as G:
        G.rak(tolerance=tol, max_iter=max_iter, mode=mode, strict=strict, seed=4,
              init_labels=init, **kw)
        assert np.array_equal(G.labels(), ref)
        k = G.split()
        assert k == k_ref
        assert np.array_equal(G.labels(), ref_split)
        q = G.modularity()
        assert abs(q - oracle.modularity(g.offsets, g.indices, g.weights, ref_split)) <= Q_SYNC_TOL


def test_split_parity(lp):
    """Communities split into connected components on the GPU equal the
    oracle's split of the oracle's labels (each component named by its
    smallest vertex), on every bucket's rows."""
    split_check(lp, gg.rmat(14, seed=3), "sync", strict=False)
    split_check(lp, gg.rmat(14, seed=3), "async", waves=2)
    off, idx, w = hub_graph(5, n=20_000, hub_deg=9_000)
    split_check(lp, gg.CSR(off, idx, w), "sync")
    split_check(lp, gg.grid_road(256, seed=2), "async", waves=3)
    split_check(lp, gg.sbm_planted(3000, 6, 0.02, 0.0005, seed=2), "sync", strict=False)


def test_split_of_scattered_labels(lp):
    """Labels v mod 3 after one sweep leave most communities in many pieces."""
    g = gg.rmat(12, seed=9)
    init = (np.arange(g.n) % 3).astype(np.int32)
    split_check(lp, g, "sync", max_iter=1, init=init, tol=1.0)
    g = gg.grid_road(64, seed=9)
    init = (np.arange(g.n) % 3).astype(np.int32)
    split_check(lp, g, "sync", max_iter=1, init=init, tol=1.0)


def test_split_before_any_run_and_edge_cases(lp):
    off, idx, w = csr_from_adj([[1], [0], [], [4], [3]])
    with lp.Graph(off, idx, w) as G:
        assert G.split() == 5  # unique labels: every vertex alone
        assert G.labels().tolist() == [0, 1, 2, 3, 4]
        G.rak(tolerance=0.0, max_iter=5, mode="async", waves=2)
        assert G.split() == 3
        assert G.labels().tolist() == [0, 0, 2, 3, 3]
    empty = gg.CSR(np.zeros(1, np.int32), np.zeros(0, np.int32), None)
    with lp.Graph(empty.offsets, empty.indices, None) as G:
        assert G.split() == 0


@pytest.mark.slow
def test_split_full_size(lp, road4096, rmat22):
    split_check(lp, road4096, "async", waves=3)
    split_check(lp, rmat22, "async", waves=2)
