"""Pins of the CPU oracle against things other than itself.

* hand-derived traces of Sec. 3.2's rule (tests/golden/rak_traces.json);
* published SplitMix64 outputs (tests/golden/splitmix64.json);
* modularity against the O(n^2) double sum of its definition (Sec. 1) and
  against closed forms;
* special cases that reduce to a library routine (first RAK step with unique
  labels = per-row numpy argmax, which returns the first maximum);
* invariants: fixed point after convergence, non-increasing label count,
  labels are vertex ids, resume equals an uninterrupted run, strict equals
  non-strict when no two labels can tie, uniform choice among ties.
"""
import itertools

import numpy as np
import pytest

import oracle
from conftest import csr_from_adj, load_golden, random_graph


# ---------------------------------------------------------------- golden traces
def test_golden_traces(golden_traces):
    assert len(golden_traces) >= 15
    for case in golden_traces:
        off, idx, w = csr_from_adj(case["adj"], case.get("w"))
        labels, iters, conv, hist = oracle.rak(
            off, idx, w, tolerance=case["tolerance"], max_iter=case["max_iter"],
            mode=case["mode"], strict=True, init_labels=case.get("init"),
            waves=case.get("waves", 0))
        assert labels.tolist() == case["labels"], case["name"]
        assert iters == case["iterations"], case["name"]
        assert conv == case["converged"], case["name"]
        assert hist.tolist() == case["changed"], case["name"]
        if "modularity" in case:
            assert oracle.modularity(off, idx, w, labels) == pytest.approx(
                case["modularity"], abs=1e-15), case["name"]


def test_splitmix64_published_outputs():
    g = load_golden("splitmix64.json")
    gamma = int(g["gamma"], 16)
    for k, expect in enumerate(g["outputs"], start=1):
        assert oracle.mix64((k * gamma) % 2**64) == int(expect, 16)


def test_tie_hash_is_counter_mode_splitmix():
    # tie_hash(seed, t, v, l) = mix(k_tv + (l+1) gamma), k_tv = mix(k_t + (v+1) gamma),
    # k_t = mix(seed + (t+1) gamma): the SplitMix64 stream keyed three times.
    gamma = 0x9E3779B97F4A7C15
    m = 2**64
    for seed, t, v, l in [(0, 0, 0, 0), (1, 3, 17, 5), (2**63 + 7, 19, 4_000_000, 123_456)]:
        kt = oracle.mix64((seed + (t + 1) * gamma) % m)
        ktv = oracle.mix64((kt + (v + 1) * gamma) % m)
        assert oracle.tie_hash(seed, t, v, l) == oracle.mix64((ktv + (l + 1) * gamma) % m)


# ---------------------------------------------------------------- modularity
def brute_modularity(off, idx, w, labels):
    """(1/2m) sum_{v,u} [A_vu - k_v k_u / 2m] delta(c_v, c_u), dense, float64."""
    n = off.shape[0] - 1
    a = np.zeros((n, n))
    for v in range(n):
        for e in range(off[v], off[v + 1]):
            a[v, idx[e]] += 1.0 if w is None else float(w[e])
    k = a.sum(axis=1)
    two_m = k.sum()
    if two_m == 0:
        return 0.0
    same = labels[:, None] == labels[None, :]
    return float(((a - np.outer(k, k) / two_m) * same).sum() / two_m)


@pytest.mark.parametrize("seed", range(12))
def test_modularity_matches_double_sum(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 60))
    off, idx, w = random_graph(n, float(rng.uniform(0.05, 0.6)), seed,
                               wmax=int(rng.integers(1, 9)), self_loops=bool(seed % 2))
    labels = rng.integers(0, max(1, n // int(rng.integers(1, 6))), size=n).astype(np.int32)
    q = oracle.modularity(off, idx, w, labels)
    assert q == pytest.approx(brute_modularity(off, idx, w, labels), abs=1e-12)
    assert -0.5 - 1e-12 <= q <= 1.0


def test_modularity_closed_forms():
    # one community -> 0
    off, idx, w = random_graph(30, 0.3, 1, wmax=5)
    assert oracle.modularity(off, idx, w, np.zeros(30, np.int32)) == pytest.approx(0, abs=1e-15)
    # k equal disjoint cliques, one label each -> 1 - 1/k
    for k, s in [(2, 4), (3, 5), (7, 6)]:
        rows = [[b * s + j for j in range(s) if j != i] for b in range(k) for i in range(s)]
        off, idx, _ = csr_from_adj(rows)
        lab = np.repeat(np.arange(k) * s, s).astype(np.int32)
        assert oracle.modularity(off, idx, None, lab) == pytest.approx(1 - 1 / k, abs=1e-15)
    # singletons -> sum_i A_ii / 2m - sum_i (k_i / 2m)^2
    off, idx, w = random_graph(25, 0.4, 3, wmax=4, self_loops=True)
    n = 25
    k = np.array([w[off[v]:off[v + 1]].sum() for v in range(n)], dtype=np.float64)
    diag = np.array([w[off[v]:off[v + 1]][idx[off[v]:off[v + 1]] == v].sum() for v in range(n)])
    two_m = k.sum()
    expect = diag.sum() / two_m - ((k / two_m) ** 2).sum()
    got = oracle.modularity(off, idx, w, np.arange(n, dtype=np.int32))
    assert got == pytest.approx(expect, abs=1e-15)
    # a single edge split in two: the lower bound -1/2
    off, idx, _ = csr_from_adj([[1], [0]])
    assert oracle.modularity(off, idx, None, np.array([0, 1], np.int32)) == -0.5


def test_modularity_exact_integers():
    off, idx, w = random_graph(40, 0.3, 7, wmax=6)
    lab = np.random.default_rng(7).integers(0, 5, 40).astype(np.int32)
    q, l_in, two_m, s = oracle.modularity(off, idx, w, lab, exact=True)
    assert two_m == int(w.sum())
    src = np.repeat(np.arange(40), np.diff(off))
    assert l_in == int(w[lab[src] == lab[idx]].sum())
    kv = np.bincount(src, weights=w, minlength=40).astype(np.int64)
    kc = np.bincount(lab, weights=kv, minlength=40).astype(np.int64)
    assert s == sum(int(x) ** 2 for x in kc)


# ---------------------------------------------------------------- RAK special cases
@pytest.mark.parametrize("seed", range(6))
def test_first_step_is_rowwise_argmax(seed):
    """With unique labels and no duplicate entries, the label weights of v are
    its edge weights, so the first synchronous strict step takes the neighbour
    behind the row's first maximum weight (numpy.argmax returns the first)."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 200))
    off, idx, w = random_graph(n, float(rng.uniform(0.02, 0.3)), 100 + seed, wmax=4)
    labels, iters, _, _ = oracle.rak(off, idx, w, tolerance=0.0, max_iter=1, mode="sync")
    for v in range(n):
        row = slice(off[v], off[v + 1])
        if off[v] == off[v + 1]:
            assert labels[v] == v
        else:
            assert labels[v] == idx[row][np.argmax(w[row])]
    # non-strict: same maximum weight, possibly another neighbour
    labels_ns, _, _, _ = oracle.rak(off, idx, w, tolerance=0.0, max_iter=1, mode="sync",
                                    strict=False, seed=seed)
    for v in range(n):
        row = slice(off[v], off[v + 1])
        if off[v] != off[v + 1]:
            wv = dict(zip(idx[row].tolist(), w[row].tolist()))
            assert wv[int(labels_ns[v])] == w[row].max()


def label_weights(off, idx, w, labels, v):
    acc = {}
    for e in range(off[v], off[v + 1]):
        lab = int(labels[idx[e]])
        acc[lab] = acc.get(lab, 0) + (1 if w is None else int(w[e]))
    return acc


@pytest.mark.parametrize("mode", ["sync", "async"])
def test_fixed_point_after_convergence(mode):
    for seed in range(8):
        off, idx, w = random_graph(80, 0.08, 200 + seed, wmax=3)
        labels, iters, conv, hist = oracle.rak(off, idx, w, tolerance=0.0, max_iter=200,
                                               mode=mode)
        if not conv:
            continue  # sync runs may oscillate; nothing to check then
        assert hist[-1] == 0
        again = oracle.choose_many(off, idx, w, labels, np.arange(80), strict=True, t=iters)
        assert np.array_equal(again, labels)
        for v in range(80):
            acc = label_weights(off, idx, w, labels, v)
            if acc:
                assert acc[int(labels[v])] == max(acc.values())


@pytest.mark.parametrize("mode,strict", list(itertools.product(["sync", "async"], [True, False])))
def test_labels_shrink_and_are_vertex_ids(mode, strict):
    off, idx, w = random_graph(120, 0.05, 11, wmax=3)
    cur = np.arange(120, dtype=np.int32)
    prev_count = 120
    for it in range(8):
        nxt, iters, _, _ = oracle.rak(off, idx, w, tolerance=0.0, max_iter=1, mode=mode,
                                      strict=strict, seed=5, iter_offset=it, init_labels=cur)
        assert set(nxt.tolist()) <= set(cur.tolist())
        assert 0 <= nxt.min() and nxt.max() < 120
        count = len(np.unique(nxt))
        assert count <= prev_count
        prev_count = count
        cur = nxt


@pytest.mark.parametrize("mode,strict", list(itertools.product(["sync", "async"], [True, False])))
def test_resume_equals_uninterrupted_run(mode, strict):
    off, idx, w = random_graph(150, 0.04, 21, wmax=5)
    full, iters, conv, hist = oracle.rak(off, idx, w, tolerance=0.0, max_iter=7, mode=mode,
                                         strict=strict, seed=9)
    cur = None
    for it in range(iters):
        cur, k, _, h = oracle.rak(off, idx, w, tolerance=0.0, max_iter=1, mode=mode,
                                  strict=strict, seed=9, iter_offset=it, init_labels=cur)
        assert h[0] == hist[it]
    assert np.array_equal(cur, full)


def test_strict_equals_nonstrict_without_ties():
    """Distinct powers of two as edge weights make every label sum of a vertex
    distinct, so the tie rule never applies."""
    rng = np.random.default_rng(5)
    for trial in range(10):
        n = 12
        pairs = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < 0.35][:30]
        rows = [[] for _ in range(n)]
        ws = [[] for _ in range(n)]
        for j, (u, v) in enumerate(pairs):
            rows[u].append(v)
            ws[u].append(1 << j)
            rows[v].append(u)
            ws[v].append(1 << j)
        off, idx, w = csr_from_adj(rows, ws)
        for mode in ("sync", "async"):
            a = oracle.rak(off, idx, w, tolerance=0.0, max_iter=10, mode=mode, strict=True)
            b = oracle.rak(off, idx, w, tolerance=0.0, max_iter=10, mode=mode, strict=False,
                           seed=trial)
            assert np.array_equal(a[0], b[0]) and a[1] == b[1]


def test_nonstrict_picks_uniformly_among_ties():
    """Star centre with k unique, equally weighted neighbour labels: the
    non-strict choice must be uniform over them (chi-square, k-1 dof)."""
    k = 8
    off, idx, _ = csr_from_adj([list(range(1, k + 1))] + [[0]] * k)
    cur = np.arange(k + 1, dtype=np.int32)
    counts = np.zeros(k + 1)
    trials = 8000
    for t in range(trials):
        c = oracle.choose_many(off, idx, None, cur, np.array([0]), strict=False, seed=3, t=t)
        counts[c[0]] += 1
    assert counts[0] == 0
    exp = trials / k
    chi2 = float(((counts[1:] - exp) ** 2 / exp).sum())
    assert chi2 < 24.3  # 0.999 quantile of chi-square with 7 dof
    # strict always takes the first neighbour in adjacency order
    c = oracle.choose_many(off, idx, None, cur, np.array([0]), strict=True, t=0)
    assert c[0] == 1


def test_disjoint_cliques_converge_to_one_label_each():
    rng = np.random.default_rng(8)
    sizes = rng.integers(4, 15, size=12)
    n = int(sizes.sum())
    perm = rng.permutation(n)
    rows = [[] for _ in range(n)]
    start = 0
    members = []
    for s in sizes:
        vs = perm[start:start + s]
        members.append(vs)
        for a in vs:
            rows[a] = sorted(int(b) for b in vs if b != a)
        start += s
    off, idx, _ = csr_from_adj(rows)
    for mode in ("sync", "async"):
        labels, iters, conv, _ = oracle.rak(off, idx, None, tolerance=0.0, max_iter=50,
                                            mode=mode)
        assert conv
        for vs in members:
            assert len(set(labels[vs].tolist())) == 1
            assert int(labels[vs[0]]) in set(vs.tolist())
        assert len(np.unique(labels)) == len(sizes)


@pytest.mark.parametrize("strict", [True, False])
def test_async_waves_limits(strict):
    """One wave is the synchronous rule; n or more waves (or 0) is the plain
    in-place update in ascending order; waves in between are neither."""
    for seed in range(6):
        off, idx, w = random_graph(90, 0.06, 300 + seed, wmax=3)
        sync = oracle.rak(off, idx, w, tolerance=0.0, max_iter=12, mode="sync", strict=strict,
                          seed=seed)
        one = oracle.rak(off, idx, w, tolerance=0.0, max_iter=12, mode="async", strict=strict,
                         seed=seed, waves=1)
        assert np.array_equal(sync[0], one[0]) and sync[1] == one[1]
        assert np.array_equal(sync[3], one[3])
        seq = oracle.rak(off, idx, w, tolerance=0.0, max_iter=12, mode="async", strict=strict,
                         seed=seed, waves=0)
        for big in (90, 91, 1000):
            b = oracle.rak(off, idx, w, tolerance=0.0, max_iter=12, mode="async", strict=strict,
                           seed=seed, waves=big)
            assert np.array_equal(seq[0], b[0]) and np.array_equal(seq[3], b[3])


def test_async_wave_visibility():
    """A vertex of wave k sees new labels exactly for neighbours in waves < k:
    on a path 0-1-2 with W = 3 the sweep reads left to right like the
    sequential order, with W = 2 vertex 1 (wave 1) sees vertex 2 (wave 0) new."""
    off, idx, w = csr_from_adj([[1], [0, 2], [1]], [[1], [1, 5], [5]])
    # unique labels; v0 -> 1, v2 -> 1 (heavy edge), v1 -> 2 (heavy edge)
    lab3, _, _, h3 = oracle.rak(off, idx, w, tolerance=0.0, max_iter=1, mode="async", waves=3)
    # W=3: v0 -> 1; v1 sees new v0 = 1 (w1) and old v2 = 2 (w5) -> 2; v2 sees new v1 = 2 -> 2
    assert lab3.tolist() == [1, 2, 2] and h3.tolist() == [2]
    lab2, _, _, h2 = oracle.rak(off, idx, w, tolerance=0.0, max_iter=1, mode="async", waves=2)
    # W=2: waves {0,2} then {1}: v0 -> 1, v2 sees old v1 = 1 -> 1; v1 sees 1 (w1) and 1 (w5) -> 1
    assert lab2.tolist() == [1, 1, 1] and h2.tolist() == [2]


def test_rejects_bad_arguments():
    off, idx, _ = csr_from_adj([[1], [0]])
    with pytest.raises(ValueError):
        oracle.rak(off, idx, None, tolerance=1.5)
    with pytest.raises(ValueError):
        oracle.rak(off, idx, None, max_iter=0)
    with pytest.raises(ValueError):
        oracle.rak(off, np.array([1, 5], np.int32), None)
    with pytest.raises(ValueError):
        oracle.rak(off, idx, None, mode="async", waves=-1)


# ------------------------------------------------- splitting disconnected communities
def test_split_hand_example():
    # path 0-1-2 and edge 3-4 share label 7, vertex 5 is isolated, and the
    # edge 2-6 joins two different labels
    off, idx, _ = csr_from_adj([[1], [0, 2], [1, 6], [4], [3], [], [2]])
    labels = np.array([7, 7, 7, 7, 7, 5, 1], np.int32)
    out, k = oracle.split(off, idx, labels)
    assert out.tolist() == [0, 0, 0, 3, 3, 5, 6] and k == 4


@pytest.mark.parametrize("seed", range(4))
def test_split_matches_library_components(seed):
    """The split equals scipy's connected components of the graph that keeps
    only the edges whose two ends share a label, each component named by its
    smallest vertex."""
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    off, idx, _ = random_graph(400, 0.01, seed)
    rng = np.random.default_rng(seed)
    labels = rng.integers(0, 6, 400).astype(np.int32)
    rows = np.repeat(np.arange(400), np.diff(off))
    keep = labels[rows] == labels[idx]
    a = sp.csr_matrix((np.ones(int(keep.sum())), (rows[keep], idx[keep])), shape=(400, 400))
    k_ref, comp = csg.connected_components(a, directed=False)
    first = np.full(k_ref, 400)
    np.minimum.at(first, comp, np.arange(400))
    out, k = oracle.split(off, idx, labels)
    assert k == k_ref
    assert np.array_equal(out, first[comp])


def test_split_refines_and_is_idempotent():
    off, idx, _ = random_graph(300, 0.02, 9)
    labels, _, _, _ = oracle.rak(off, idx, None, 0.05, 20, "sync", strict=False, seed=3)
    out, k = oracle.split(off, idx, labels)
    # same component => same community; every component is named by a member
    for c in np.unique(out):
        assert len(np.unique(labels[out == c])) == 1 and out[c] == c
    again, k2 = oracle.split(off, idx, out)
    assert np.array_equal(again, out) and k2 == k
    assert k >= len(np.unique(labels))


# ------------------------------------------------------------------------- SLPA
def test_slpa_memory_of_one_slot_is_identity():
    off, idx, w = random_graph(50, 0.1, 1)
    lab, mem, it, conv, hist = oracle.slpa(off, idx, w, memory_size=1)
    assert it == 0 and np.array_equal(lab, np.arange(50)) and mem.shape == (1, 50)


@pytest.mark.parametrize("strict", [True, False])
def test_slpa_first_iteration_is_a_rak_step(strict):
    """In the first iteration every speaker can only speak its own id, so the
    listener's choice is one synchronous RAK step from unique labels (the tie
    hash of iteration index 1 on both sides)."""
    off, idx, w = random_graph(300, 0.03, 5, wmax=3)
    _, mem, it, _, _ = oracle.slpa(off, idx, w, memory_size=2, tolerance=0.0, strict=strict,
                                   seed=7)
    ref, _, _, _ = oracle.rak(off, idx, w, 0.0, 1, "sync", strict=strict, seed=7, iter_offset=1)
    assert it == 1 and np.array_equal(mem[1], ref)


def test_slpa_star_first_iteration_by_hand():
    # centre 0 hears leaves 1..4 (one each, first is 1); every leaf hears 0
    off, idx, w = csr_from_adj([[1, 2, 3, 4], [0], [0], [0], [0]])
    _, mem, _, _, _ = oracle.slpa(off, idx, w, memory_size=2, tolerance=0.0)
    assert mem[1].tolist() == [1, 0, 0, 0, 0]


def test_slpa_slots_are_uniform():
    t = 5
    slots = np.array([oracle.slpa_slot(3, t, v, p) for v in range(400) for p in range(10)])
    assert slots.min() >= 0 and slots.max() < t
    counts = np.bincount(slots, minlength=t)
    expected = slots.size / t
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 20.5  # 4 degrees of freedom, p ~ 0.0004


def test_slpa_memories_are_valid_and_stay_in_components():
    """Every stored label was in some neighbour's memory before that
    iteration; labels never cross components; isolated vertices repeat
    themselves; the community is the label stored most often."""
    off_a, idx_a, _ = random_graph(60, 0.2, 8)
    off_b, idx_b, _ = random_graph(40, 0.25, 9)
    off = np.concatenate([off_a, off_b[1:] + off_a[-1], [off_a[-1] + off_b[-1]]]).astype(np.int32)
    idx = np.concatenate([idx_a, idx_b + 60]).astype(np.int32)  # vertex 100 isolated
    lab, mem, it, _, _ = oracle.slpa(off, idx, None, memory_size=8, tolerance=0.0, seed=2)
    assert it == 7
    comp = np.where(np.arange(101) < 60, 0, np.where(np.arange(101) < 100, 1, 2))
    for t in range(1, it + 1):
        for v in range(101):
            row = idx[off[v]:off[v + 1]]
            if row.size == 0:
                assert mem[t, v] == mem[t - 1, v]
                continue
            assert mem[t, v] in set(mem[:t, row].ravel().tolist())
            assert comp[mem[t, v]] == comp[v]
    for v in range(101):
        vals, first, counts = np.unique(mem[:, v], return_index=True, return_counts=True)
        top = counts.max()
        assert lab[v] == vals[first == first[counts == top].min()][0]
