"""Serving with continuous batching: requests submitted while others run are
admitted as slots and budget free up, those queued together as one cohort
(one batch arena, one launch per bucket per iteration); every result equals
the same graph run alone through lp_rak_run (bit-exact labels, iterations
and modularity), whether it ran alone or in a cohort."""
import time

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


def pool():
    graphs = [gg.sbm_mixing(20_000, 40, 16.0, 0.3, seed=1, wmin=1, wmax=8),
              gg.rmat(15, edge_factor=8, seed=2, wmin=1, wmax=8),
              gg.grid_road(200, seed=3, wmin=1, wmax=8),
              gg.sbm_mixing(3_000, 10, 12.0, 0.3, seed=4, wmin=1, wmax=8),
              gg.rmat(12, edge_factor=8, seed=5, wmin=1, wmax=8)]
    return graphs


@pytest.mark.parametrize("mode,max_cohort", [("sync", 16), ("async", 16), ("sync", 1)])
def test_results_alone_and_in_the_mix(lp, mode, max_cohort):
    graphs = pool()
    kw = dict(tolerance=0.05, max_iter=20, mode=mode, strict=True, waves=7)
    alone = []
    for g in graphs:
        with lp.Graph(g.offsets, g.indices, g.weights) as G:
            r = G.rak(**kw)
            alone.append((G.labels().copy(), r.iterations, G.modularity()))
    cfg = lp.lp_server_config_default()
    cfg.max_active = 3          # fewer slots than requests: later ones queue
    cfg.streams = 2
    cfg.max_cohort = max_cohort
    srv = lp.lp_server_create(cfg, **kw)
    try:
        order = [i % len(graphs) for i in range(12)]
        outs = [np.full(graphs[i].n, -1, np.int32) for i in order]
        for rid, (i, out) in enumerate(zip(order, outs)):
            g = graphs[i]
            lp.lp_server_submit(srv, rid, g.offsets, g.indices, g.weights, out)
            if rid % 4 == 3:
                time.sleep(0.01)  # later requests arrive while earlier ones run
        lp.lp_server_drain(srv)
        res = {r.request_id: r for r in lp.lp_server_poll(srv, capacity=64)}
        stats = lp.lp_server_stats(srv)
    finally:
        lp.lp_server_destroy(srv)
    assert sorted(res) == list(range(12))
    assert stats["largest_cohort"] <= min(max_cohort, cfg.max_active)
    if max_cohort == 1:
        assert stats["cohorts"] == 12 and stats["batched_requests"] == 0
    for rid, i in enumerate(order):
        r = res[rid]
        lab, iters, q = alone[i]
        assert r.status == 0, r.as_dict()
        assert r.iterations == iters
        assert np.array_equal(outs[rid], lab)
        assert abs(r.modularity - q) <= 1e-9
        assert r.latency_ms >= r.queued_ms >= 0


def test_budget_and_errors(lp):
    g = gg.rmat(12, seed=1)
    cfg = lp.lp_server_config_default()
    cfg.hbm_budget = 1 << 20  # smaller than one request
    srv = lp.lp_server_create(cfg)
    try:
        with pytest.raises(lp.LPError, match="budget"):
            lp.lp_server_submit(srv, 0, g.offsets, g.indices, g.weights)
    finally:
        lp.lp_server_destroy(srv)
    cfg = lp.lp_server_config_default()
    srv = lp.lp_server_create(cfg)
    bad_idx = g.indices.copy()
    bad_idx[5] = g.n + 3
    try:
        lp.lp_server_submit(srv, 7, g.offsets, bad_idx, g.weights)
        lp.lp_server_submit(srv, 8, g.offsets, g.indices, g.weights)
        lp.lp_server_drain(srv)
        res = {r.request_id: r for r in lp.lp_server_poll(srv)}
    finally:
        lp.lp_server_destroy(srv)
    assert res[7].status == lp.LP_EINVAL and res[8].status == 0
    assert lp.lp_server_poll.__name__  # the server stays usable after a bad request


def test_cohorts_form_under_load(lp):
    """A burst queued behind a long request is admitted in cohorts of several
    requests; every result still equals the graph run alone."""
    graphs = pool()
    kw = dict(tolerance=0.05, max_iter=20, mode="sync", strict=True)
    alone = []
    for g in graphs:
        with lp.Graph(g.offsets, g.indices, g.weights) as G:
            r = G.rak(**kw)
            alone.append((G.labels().copy(), r.iterations, G.modularity()))
    cfg = lp.lp_server_config_default()
    cfg.max_active = 8
    cfg.streams = 2
    cfg.max_cohort = 4
    srv = lp.lp_server_create(cfg, **kw)
    try:
        order = [i % len(graphs) for i in range(40)]
        outs = [np.full(graphs[i].n, -1, np.int32) for i in order]
        for rid, (i, out) in enumerate(zip(order, outs)):
            g = graphs[i]
            lp.lp_server_submit(srv, rid, g.offsets, g.indices, g.weights, out)
        lp.lp_server_drain(srv)
        res = {r.request_id: r for r in lp.lp_server_poll(srv, capacity=64)}
        stats = lp.lp_server_stats(srv)
    finally:
        lp.lp_server_destroy(srv)
    assert sorted(res) == list(range(40))
    assert stats["batched_requests"] > 0 and 2 <= stats["largest_cohort"] <= 4, stats
    for rid, i in enumerate(order):
        lab, iters, q = alone[i]
        assert res[rid].status == 0 and res[rid].iterations == iters
        assert np.array_equal(outs[rid], lab)
        assert abs(res[rid].modularity - q) <= 1e-9


def test_invalid_request_inside_a_cohort_fails_alone(lp):
    """A burst with one invalid graph: whether it was queued with others (its
    cohort's batch then fails to ingest and the requests are admitted one by
    one) or alone, only that request fails."""
    g = gg.rmat(12, seed=1)
    bad_idx = g.indices.copy()
    bad_idx[5] = g.n + 3
    ref = None
    with lp.Graph(g.offsets, g.indices, g.weights) as G:
        G.rak()
        ref = G.labels().copy()
    cfg = lp.lp_server_config_default()
    cfg.max_active = 16
    srv = lp.lp_server_create(cfg)
    outs = {}
    try:
        for rid in range(12):
            outs[rid] = np.full(g.n, -1, np.int32)
            idx = bad_idx if rid == 6 else g.indices
            lp.lp_server_submit(srv, rid, g.offsets, idx, g.weights, outs[rid])
        lp.lp_server_drain(srv)
        res = {r.request_id: r for r in lp.lp_server_poll(srv, capacity=64)}
    finally:
        lp.lp_server_destroy(srv)
    assert res[6].status == lp.LP_EINVAL
    for rid in range(12):
        if rid != 6:
            assert res[rid].status == 0 and np.array_equal(outs[rid], ref), rid
