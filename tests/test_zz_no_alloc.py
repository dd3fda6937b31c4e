"""lp_rak_sweep_noalloc: one synchronous sweep that allocates no memory.

It serves callers whose device memory is fully reserved by another allocator
(a framework's caching allocator, a pool sized once under a fixed budget), so
they cannot let a library call cudaMalloc.  Its only scratch is a static
device array of the library.  These tests check, through the C ABI, that two
calls in a row give exactly the labels and changed counts of the existing
entry point (lp_rak_run, one synchronous iteration from the same labels), and
that rows longer than the array's limit are rejected.
"""
import numpy as np
import pytest

import graphgen as gg

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
