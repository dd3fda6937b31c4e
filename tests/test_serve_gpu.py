"""Serving with continuous batching: requests submitted while others run are
admitted as slots and budget free up; every result equals the same graph run
alone through lp_rak_run (synchronous mode: bit-exact labels, iterations and
modularity)."""
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


@pytest.mark.parametrize("mode", ["sync", "async"])
def test_results_alone_and_in_the_mix(lp, mode):
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
    finally:
        lp.lp_server_destroy(srv)
    assert sorted(res) == list(range(12))
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
