"""Serving loop: queries answered in a continuously batched mix give exactly what they give alone, and what the
CPU oracle's Algorithm 1 gives for the same graph and parameters."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import graphs

import paper_2105_04023_gb300 as im

pytestmark = pytest.mark.gpu

IC, WC = 0, 1


@pytest.fixture(scope="module")
def ctx():
    from paper_2105_04023_gb300 import build

    build.build()
    c = im.Context(0)
    yield c
    c.close()


POOL = [(graphs.rmat(10, 12, seed=71), WC, 0.0), (graphs.rmat(11, 8, seed=72), IC, 0.05),
        (graphs.erdos_renyi(700, 5000, seed=73), IC, 0.1), (graphs.star_hub(800, seed=74), WC, 0.0)]
# (graph, K, R, seed, literal blocking)
QUERIES = [(i % 4, 3 + (i * 5) % 9, (64, 256, 128)[i % 3], 100 + i, i % 5 == 4) for i in range(14)]


def _graph(i):
    g, model, p = POOL[i]
    return im.Graph.from_synth(g, model, p)


def _prm(K, R, seed, literal=False):
    return im.params(R=R, K=K, eps_g=0.01, eps_l=0.3, seed=seed,
                     blocking=im.IM_BLOCK_LITERAL if literal else im.IM_BLOCK_RESIDUAL)


def _alone(ctx, gid, K, R, seed, literal=False):
    return ctx.im_select_seeds(_graph(gid), _prm(K, R, seed, literal), trace=False)


def _oracle(gid, K, R, seed, literal=False):
    g, model, p = POOL[gid]
    return oracle.select_seeds(g.n, g.xadj, g.adj, model, p, R, K, 0.01, 0.3, 0.0, seed, literal=literal)


def _check(res, q, ctx):
    """A served result equals the same query alone on the GPU and the oracle's selection."""
    alone = _alone(ctx, *q)
    assert res["seeds"].tolist() == alone["seeds"].tolist(), q
    assert res["sigma_final"] == alone["sigma_final"]
    assert res["rebuilds"] == alone["rebuilds"]
    ref = _oracle(*q)
    assert res["seeds"].tolist() == ref["seeds"].tolist(), q
    assert res["sigma_final"] == float(ref["sigma"][-1])
    assert res["rebuilds"] == int(ref["rebuilt"].sum())


def _drain(srv, tickets, max_steps=100000):
    out = {}
    for _ in range(max_steps):
        active, queued = srv.im_server_step()
        for t in list(tickets):
            r = srv.im_server_poll(t)
            if r is not None:
                out[t] = r
                tickets.remove(t)
        if not tickets and active == 0 and queued == 0:
            return out
    raise AssertionError("server did not finish")


def test_mix_equals_alone_with_late_arrivals(ctx):
    srv = im.Server(ctx, hbm_budget_bytes=8 << 30, max_active=64)
    gids = [srv.im_server_add_graph(_graph(i)) for i in range(len(POOL))]
    tickets = {}
    first = QUERIES[: len(QUERIES) // 2]
    for q in first:
        tickets[srv.im_server_submit(gids[q[0]], _prm(*q[1:]))] = q
    # a few ticks with the first half running, then the rest arrive and join the batch
    for _ in range(5):
        srv.im_server_step()
    for q in QUERIES[len(QUERIES) // 2:]:
        tickets[srv.im_server_submit(gids[q[0]], _prm(*q[1:]))] = q
    res = _drain(srv, set(tickets))
    for t, q in tickets.items():
        _check(res[t], q, ctx)
    srv.close()


def test_budget_limits_admission(ctx):
    probe = im.Server(ctx, hbm_budget_bytes=1 << 30, max_active=1)
    one = probe.im_server_footprint(probe.im_server_add_graph(_graph(0)), im.params(R=256, K=4, eps_g=0.01))
    probe.close()
    # room for one query of this size at a time, not two
    srv = im.Server(ctx, hbm_budget_bytes=one * 3 // 2, max_active=16)
    gid = srv.im_server_add_graph(_graph(0))
    tickets = {srv.im_server_submit(gid, im.params(R=256, K=4, eps_g=0.01, seed=s)): s for s in (1, 2, 3)}
    seen_active = []
    pending = set(tickets)
    res = {}
    for _ in range(100000):
        active, queued = srv.im_server_step()
        seen_active.append(active)
        for t in list(pending):
            r = srv.im_server_poll(t)
            if r is not None:
                res[t] = r
                pending.remove(t)
        if not pending:
            break
    assert max(seen_active) == 1
    for t, s in tickets.items():
        _check(res[t], (0, 4, 256, s), ctx)
    srv.close()


def test_cancel_and_over_budget(ctx):
    srv = im.Server(ctx, hbm_budget_bytes=8 << 20, max_active=1)
    gid = srv.im_server_add_graph(_graph(1))
    t1 = srv.im_server_submit(gid, im.params(R=64, K=3, eps_g=0.01, seed=5))
    t2 = srv.im_server_submit(gid, im.params(R=64, K=3, eps_g=0.01, seed=6))
    t3 = srv.im_server_submit(gid, im.params(R=64, K=3, eps_g=0.01, seed=7))
    srv.im_server_cancel(t2)  # still queued
    res = _drain(srv, {t1, t3})
    _check(res[t1], (1, 3, 64, 5), ctx)
    _check(res[t3], (1, 3, 64, 7), ctx)
    with pytest.raises(im.ImError) as ei:
        srv.im_server_poll(t2)
    assert ei.value.status == im._lib.IM_ECANCELED
    big = srv.im_server_add_graph(im.Graph.from_synth(graphs.rmat(14, 16, seed=75), WC))
    with pytest.raises(im.ImError) as ei:
        srv.im_server_submit(big, im.params(R=1024, K=5, eps_g=0.01))
    assert ei.value.status == im._lib.IM_ENOMEM
    srv.close()


def test_cancel_running_query_frees_its_slot(ctx):
    srv = im.Server(ctx, hbm_budget_bytes=1 << 30, max_active=1)
    gid = srv.im_server_add_graph(_graph(0))
    t1 = srv.im_server_submit(gid, im.params(R=256, K=20, eps_g=0.0, seed=9))
    t2 = srv.im_server_submit(gid, im.params(R=64, K=2, eps_g=0.01, seed=10))
    active, queued = srv.im_server_step()
    assert active == 1 and queued == 1
    srv.im_server_cancel(t1)
    res = _drain(srv, {t2})
    _check(res[t2], (0, 2, 64, 10), ctx)
    srv.close()


def test_repeated_first_diffusions_are_reused(ctx):
    # queries that share (graph, R, seed) start from the kept first diffusion and still answer exactly what they
    # answer alone; a different seed or R does not hit
    srv = im.Server(ctx, hbm_budget_bytes=8 << 30, max_active=4)
    gids = [srv.im_server_add_graph(_graph(i)) for i in range(2)]
    first = [(0, 6, 256, 31, False), (1, 4, 64, 32, False)]
    rest = [(0, 9, 256, 31, False), (0, 3, 256, 31, True), (1, 7, 64, 32, False), (0, 5, 128, 31, False),
            (1, 2, 64, 33, False), (0, 8, 256, 31, False)]
    res, tickets = {}, {}
    for batch in (first, rest):
        ts = {srv.im_server_submit(gids[q[0]], _prm(*q[1:])): q for q in batch}
        res.update(_drain(srv, set(ts)))
        tickets.update(ts)
    info = srv.im_server_info()
    assert info["build_hits"] == 4, info  # the four later queries with the keys of the first two
    assert info["kept_builds"] == 4, info  # one per distinct (graph, R, seed)
    assert info["used_bytes"] > 0
    for t, q in tickets.items():
        _check(res[t], q, ctx)
    srv.close()
