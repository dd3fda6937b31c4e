"""Pins of the COPRA oracle (Sec. 3.3) against what the paper and the
mathematics fix, independent of its own code:

* one label per vertex (max_labels = 1) is RAK: the threshold keeps a label
  only when it holds all the weight, else the best label alone, so labels,
  iteration counts and changed counts equal the RAK oracle's in every mode;
* the first iteration from singletons has a closed form (each neighbour u of
  v carries its own label with belonging 1), restated here with numpy;
* a bridge vertex between two cliques joins both with belonging 1/2 (by hand);
* disjoint cliques end as one community each with belonging 1;
* invariants: belongings sum to exactly 2^16, sets are sorted, hold at most
  max_labels pairs and only vertex ids;
* a second, independent restatement (plain Python dictionaries) on tiny
  random graphs, set by set, synchronous and sequential asynchronous.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from conftest import csr_from_adj, random_graph

S = oracle.COPRA_ONE


@pytest.mark.parametrize("mode,waves,strict", [("sync", 0, True), ("sync", 0, False),
                                               ("async", 2, True), ("async", 0, False)])
def test_one_label_is_rak(mode, waves, strict):
    graphs = [gg.rmat(11, seed=4), gg.sbm_planted(800, 8, 0.05, 0.002, seed=2),
              gg.CSR(*random_graph(300, 0.05, 7, wmax=4))]
    for g in graphs:
        lab, iters, conv, hist = oracle.rak(g.offsets, g.indices, g.weights, 0.05, 20, mode,
                                            strict=strict, seed=9, waves=waves)
        c_lab, _, c_b, c_it, c_conv, c_hist = oracle.copra(
            g.offsets, g.indices, g.weights, max_labels=1, tolerance=0.05, max_iter=20,
            mode=mode, waves=waves, strict=strict, seed=9)
        assert np.array_equal(lab, c_lab)
        assert iters == c_it and conv == c_conv and np.array_equal(hist, c_hist)
        assert np.all(c_b[:, 0] == S)


def first_iteration(off, idx, w, L):
    """Closed form of the first COPRA iteration from singletons (strict ties,
    rows without repeated neighbours): neighbour u carries label u with
    weight w_vu; kept iff L * w_vu >= W; none kept: the heaviest alone (first
    in row order); b = floor(w_u * S / sum of kept w), the remainder to the
    heaviest kept (first in row order); stored by b desc, then row order."""
    n = off.shape[0] - 1
    out = []
    for v in range(n):
        row = idx[off[v]:off[v + 1]]
        ww = np.ones(row.size, np.int64) if w is None else w[off[v]:off[v + 1]].astype(np.int64)
        if row.size == 0:
            out.append([(v, S)])
            continue
        W = int(ww.sum())
        keep = [i for i in range(row.size) if L * ww[i] >= W]
        if not keep:
            keep = [int(np.argmax(ww))]  # first maximum
        tot = int(ww[keep].sum())
        b = {i: int(ww[i]) * S // tot for i in keep}
        best = max(keep, key=lambda i: (ww[i], -i))
        b[best] += S - sum(b.values())
        out.append([(int(row[i]), b[i]) for i in sorted(keep, key=lambda i: (-b[i], i))])
    return out


@pytest.mark.parametrize("L", [1, 2, 3, 8])
def test_first_iteration_closed_form(L):
    for seed in range(4):
        off, idx, w = random_graph(120, 0.06, 40 + seed, wmax=5)
        _, sl, sb, _, _, _ = oracle.copra(off, idx, w, max_labels=L, tolerance=0.0, max_iter=1)
        ref = first_iteration(off, idx, w, L)
        for v in range(off.shape[0] - 1):
            got = [(int(sl[v, s]), int(sb[v, s])) for s in range(L) if sb[v, s] > 0]
            assert got == ref[v], (L, seed, v)


def test_bridge_vertex_by_hand():
    # two K4 (0-3, 5-8) and vertex 4 adjacent to 3 and 5
    adj = [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2, 4], [3, 5],
           [4, 6, 7, 8], [5, 7, 8], [5, 6, 8], [5, 6, 7]]
    off, idx, w = csr_from_adj(adj)
    _, sl, sb, _, _, _ = oracle.copra(off, idx, w, max_labels=2, tolerance=0.0, max_iter=1)
    # vertex 4 hears labels 3 and 5 with equal weight: both kept at 1/2, 3 first
    assert (sl[4, 0], sb[4, 0], sl[4, 1], sb[4, 1]) == (3, S // 2, 5, S // 2)
    # vertex 0 hears 1, 2, 3 with weight 1 each: none reaches 1/2, so the first alone
    assert (sl[0, 0], sb[0, 0], sb[0, 1]) == (1, S, 0)


def test_disjoint_cliques_one_community_each():
    k, size = 5, 6
    adj = [[c * size + j for j in range(size) if j != i] for c in range(k) for i in range(size)]
    off, idx, w = csr_from_adj(adj)
    for L in (1, 2, 4):
        lab, _, sb, it, conv, _ = oracle.copra(off, idx, w, max_labels=L, tolerance=0.0,
                                               max_iter=30, mode="async", waves=0)
        assert conv
        for c in range(k):
            assert np.unique(lab[c * size:(c + 1) * size]).size == 1
        assert np.unique(lab).size == k
        assert np.all(sb[:, 0] == S)


def test_invariants():
    g = gg.rmat(12, seed=8)
    for L in (2, 5, 16):
        lab, sl, sb, it, conv, hist = oracle.copra(g.offsets, g.indices, g.weights, max_labels=L,
                                                   tolerance=0.01, max_iter=15, mode="async",
                                                   waves=2, strict=False, seed=3)
        assert np.all(sb.sum(axis=1, dtype=np.int64) == S)
        nz = sb > 0
        assert np.all(nz[:, 0]) and np.all(nz[:, :-1] >= nz[:, 1:])  # sets are prefixes
        assert np.all(np.diff(sb.astype(np.int64), axis=1)[nz[:, 1:]] <= 0)  # b descending
        assert np.all((sl[nz] >= 0) & (sl[nz] < g.n))
        assert np.array_equal(lab, sl[:, 0])
        assert len(hist) == it


def brute_copra(adj, w, L, iters, waves, strict, seed):
    """Independent restatement with dictionaries (tiny graphs): waves = 1 is
    synchronous, waves = n the plain ascending in-place order."""
    n = len(adj)
    sets = [[(v, S)] for v in range(n)]
    for t in range(iters):
        new = [None] * n
        for k in range(waves):
            for v in range(k, n, waves):
                if not adj[v]:
                    new[v] = [(v, S)]
                    continue
                tot, first, order = {}, {}, 0
                for u, wt in zip(adj[v], w[v]):
                    src = new[u] if (u % waves) < k else sets[u]
                    for lab, b in src:
                        if lab not in tot:
                            tot[lab], first[lab] = 0, order
                        tot[lab] += wt * b
                        order += 1
                W = sum(w[v])

                def key(lab):
                    h = 0 if strict else oracle.tie_hash(seed, t, v, lab)
                    return (-tot[lab], h, first[lab])

                kept = [lab for lab in tot if L * tot[lab] >= W * S]
                if not kept:
                    kept = [min(tot, key=key)]
                tk = sum(tot[lab] for lab in kept)
                b = {lab: tot[lab] * S // tk for lab in kept}
                b[min(kept, key=key)] += S - sum(b.values())
                new[v] = sorted(((lab, b[lab]) for lab in kept),
                                key=lambda x: (-x[1], first[x[0]]))
        sets = new
    return sets


@pytest.mark.parametrize("strict", [True, False])
def test_brute_force_tiny_graphs(strict):
    rng = np.random.default_rng(5)
    for trial in range(30):
        n = int(rng.integers(2, 11))
        off, idx, w = random_graph(n, float(rng.uniform(0.2, 0.8)), 100 + trial, wmax=4)
        w = np.ones(idx.size, np.int32) if w is None else w
        adj = [idx[off[v]:off[v + 1]].tolist() for v in range(n)]
        ww = [w[off[v]:off[v + 1]].tolist() for v in range(n)]
        L = int(rng.integers(1, 6))
        iters = int(rng.integers(1, 5))
        for mode, waves in (("sync", 1), ("async", n)):
            _, sl, sb, it, _, _ = oracle.copra(off, idx, w, max_labels=L, tolerance=0.0,
                                               max_iter=iters, mode=mode,
                                               waves=0 if mode == "async" else 0, strict=strict,
                                               seed=11)
            ref = brute_copra(adj, ww, L, it, waves, strict, 11)
            for v in range(n):
                got = [(int(sl[v, s]), int(sb[v, s])) for s in range(L) if sb[v, s] > 0]
                assert got == ref[v], (trial, mode, v, got, ref[v])
