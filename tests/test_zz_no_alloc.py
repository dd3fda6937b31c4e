"""lp_rak_sweep_noalloc: one synchronous sweep that allocates no memory.

It serves callers whose device memory is fully reserved by another allocator
(a framework's caching allocator, a pool sized once under a fixed budget), so
they cannot let a library call cudaMalloc.  Its only scratch is a static
device array of the library.  These tests check, through the C ABI, that two
calls in a row give exactly the labels and changed counts of the existing
entry point (lp_rak_run, one synchronous iteration from the same labels) and
of the CPU oracle's single sweep; that labels crowding one region of a hub's
shared table spill into the array's overflow table and come out right, and
leave it clean for the next call; that calls allocate no device memory; and
that rows longer than the array's limit are rejected.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lp():
    import torch

    import __graft_entry__

    assert torch.cuda.is_available()
    __graft_entry__.build()
    import paper_2301_09125_gb300 as lp

    return lp


def hub_csr(n=12_000, hub_deg=4_000, seed=3):
    """Sparse random graph plus one vertex with hub_deg neighbours (row limit
    4096), rows shuffled, weights 1-3."""
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n, 3 * n)
    v = rng.integers(0, n, 3 * n)
    hv = rng.choice(np.arange(1, n), hub_deg, replace=False)
    u = np.concatenate([u, np.zeros(hub_deg, np.int64)])
    v = np.concatenate([v, hv])
    keep = u != v
    a = np.unique(np.stack([np.minimum(u[keep], v[keep]), np.maximum(u[keep], v[keep])], 1), axis=0)
    src = np.concatenate([a[:, 0], a[:, 1]])
    dst = np.concatenate([a[:, 1], a[:, 0]])
    wpair = (a[:, 0] * 31 + a[:, 1] * 17) % 3 + 1
    w = np.concatenate([wpair, wpair])
    perm = rng.permutation(src.size)
    order = np.argsort(src[perm], kind="stable")
    src, dst, w = src[perm][order], dst[perm][order], w[perm][order]
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, src + 1, 1)
    return np.cumsum(off).astype(np.int32), dst.astype(np.int32), w.astype(np.int32)


@pytest.mark.parametrize("strict", [True, False])
@pytest.mark.parametrize("graph", ["rmat", "hub"])
def test_two_calls_match_lp_rak_run(lp, graph, strict):
    import torch

    if graph == "rmat":
        g = gg.rmat(14, seed=12)
        off, idx, w = g.offsets, g.indices, g.weights
    else:
        off, idx, w = hub_csr()
    n = off.shape[0] - 1
    assert np.diff(off).max() <= 4096
    dev = torch.device("cuda")
    t_off, t_idx, t_w = (torch.from_numpy(a).to(dev) for a in (off, idx, w))
    lab0 = torch.arange(n, dtype=torch.int32, device=dev)
    lab1 = torch.empty(n, dtype=torch.int32, device=dev)
    lab2 = torch.empty(n, dtype=torch.int32, device=dev)
    seed = 41
    c1 = lp.lp_rak_sweep_noalloc(t_off, t_idx, t_w, lab0, lab1, strict=strict, seed=seed,
                                 iteration=0)
    c2 = lp.lp_rak_sweep_noalloc(t_off, t_idx, t_w, lab1, lab2, strict=strict, seed=seed,
                                 iteration=1)
    torch.cuda.synchronize()
    with lp.Graph(off, idx, w) as G:
        G.rak(mode="sync", tolerance=0.0, max_iter=1, strict=strict, seed=seed)
        ref1 = G.labels().copy()
        h1 = G.history()
        G.rak(mode="sync", tolerance=0.0, max_iter=1, strict=strict, seed=seed, iter_offset=1,
              init_labels=ref1)
        ref2 = G.labels().copy()
        h2 = G.history()
    assert np.array_equal(lab1.cpu().numpy(), ref1)
    assert np.array_equal(lab2.cpu().numpy(), ref2)
    assert c1 == h1[0] and c2 == h2[0]
    verts = np.arange(n, dtype=np.int32)
    o1 = oracle.choose_many(off, idx, w, np.arange(n, dtype=np.int32), verts, strict=strict,
                            seed=seed, t=0)
    o2 = oracle.choose_many(off, idx, w, o1, verts, strict=strict, seed=seed, t=1)
    assert np.array_equal(lab1.cpu().numpy(), o1)
    assert np.array_equal(lab2.cpu().numpy(), o2)


def crowded_labels(n, hub_nbrs, lg=13):
    """Labels for the hub's neighbours that all share one Fibonacci hash (top
    lg bits of label * 0x9E3779B1) in the hub's 2^lg-slot table: more than the
    32 labels its probe window holds, so the rest must spill to the overflow
    table whatever the insertion order."""
    cand = np.arange(n, dtype=np.uint64)
    h = ((cand * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)) >> np.uint64(32 - lg)
    h0 = int(np.bincount(h.astype(np.int64), minlength=1 << lg).argmax())
    pick = cand[h == h0].astype(np.int32)
    assert pick.size > 40
    lab = np.arange(n, dtype=np.int32)
    lab[hub_nbrs] = pick[np.arange(hub_nbrs.size) % pick.size]
    return lab


@pytest.mark.parametrize("strict", [True, False])
def test_overflow_table_spills_and_stays_clean(lp, strict):
    import torch

    off, idx, w = hub_csr(n=600_000, hub_deg=4_000, seed=5)  # ~73 labels per hash value
    n = off.shape[0] - 1
    hub = int(np.argmax(np.diff(off)))
    assert np.diff(off)[hub] > 2048  # the hub's table has 2^13 slots
    lab_in = crowded_labels(n, idx[off[hub]:off[hub + 1]])
    dev = torch.device("cuda")
    t_off, t_idx, t_w = (torch.from_numpy(a).to(dev) for a in (off, idx, w))
    t_in = torch.from_numpy(lab_in).to(dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    c = lp.lp_rak_sweep_noalloc(t_off, t_idx, t_w, t_in, out, strict=strict, seed=9, iteration=4)
    verts = np.arange(n, dtype=np.int32)
    ref = oracle.choose_many(off, idx, w, lab_in, verts, strict=strict, seed=9, t=4)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert c == int(np.sum(ref != lab_in))
    with lp.Graph(off, idx, w) as G:
        G.rak(mode="sync", tolerance=0.0, max_iter=1, strict=strict, seed=9, iter_offset=4,
              init_labels=lab_in)
        assert np.array_equal(G.labels(), ref)
    # a call without spills afterwards: the overflow tables came back clean
    g = gg.rmat(13, seed=21)
    t = [torch.from_numpy(a).to(dev) for a in (g.offsets, g.indices, g.weights)]
    lab0 = torch.arange(g.n, dtype=torch.int32, device=dev)
    lab1 = torch.empty(g.n, dtype=torch.int32, device=dev)
    lp.lp_rak_sweep_noalloc(*t, lab0, lab1, strict=strict, seed=9, iteration=0)
    ref = oracle.choose_many(g.offsets, g.indices, g.weights, np.arange(g.n, dtype=np.int32),
                             np.arange(g.n, dtype=np.int32), strict=strict, seed=9, t=0)
    assert np.array_equal(lab1.cpu().numpy(), ref)


def test_calls_allocate_no_device_memory(lp):
    import torch

    g = gg.rmat(14, seed=30)
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (g.offsets, g.indices, g.weights)]
    lab0 = torch.arange(g.n, dtype=torch.int32, device=dev)
    lab1 = torch.empty(g.n, dtype=torch.int32, device=dev)
    lp.lp_rak_sweep_noalloc(*t, lab0, lab1)  # one-time set-up and module load
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats().get("allocated_bytes.all.current", 0)
    for it in range(2):
        lp.lp_rak_sweep_noalloc(*t, lab0 if it == 0 else lab1, lab1 if it == 0 else lab0,
                                iteration=it)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_stats().get("allocated_bytes.all.current", 0) == stats0


def test_rejects_rows_beyond_the_limit(lp):
    import torch

    off, idx, w = hub_csr(n=9_000, hub_deg=5_000)
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (off, idx, w)]
    n = off.shape[0] - 1
    lab0 = torch.arange(n, dtype=torch.int32, device=dev)
    lab1 = torch.empty(n, dtype=torch.int32, device=dev)
    with pytest.raises(lp.LPError, match="4096"):
        lp.lp_rak_sweep_noalloc(*t, lab0, lab1)
    with pytest.raises(lp.LPError, match="differ"):
        lp.lp_rak_sweep_noalloc(*t, lab0, lab0)
