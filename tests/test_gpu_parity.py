"""Parity of the CUDA library with the CPU oracle, element by element, on seeded synthetic graphs.

Registers, sweep counts, edge-simulation visits and frontier sizes must be bit-exact; seed sets, register sums and
rebuild decisions exact; sigma exact (an integer count over R) and the estimate within 1e-12 relative (both sides
form it from the same integer in double).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from gpu_common import assert_build_parity, assert_select_parity, gpu_build
from synth import graphs, workloads

import paper_2105_04023_gb300 as im

pytestmark = pytest.mark.gpu

IC, WC, PER_EDGE = 0, 1, 2


@pytest.fixture(scope="module")
def ctx():
    from paper_2105_04023_gb300 import build

    build.build()
    c = im.Context(0)
    yield c
    c.close()


SMALL = {
    "er300": graphs.erdos_renyi(300, 2400, seed=3),
    "rmat10": graphs.rmat(10, 8, seed=4),
    "hub1500": graphs.star_hub(1500, seed=5),
    "ragged97": graphs.random_small(97, 700, seed=6),
    "chain200": graphs.chain(200),
}


@pytest.mark.parametrize("R", [64, 128, 256, 512, 1024])
@pytest.mark.parametrize("gname,model,p", [("er300", IC, 0.05), ("rmat10", WC, 0.0), ("hub1500", IC, 0.3),
                                           ("ragged97", PER_EDGE, 0.0), ("chain200", IC, 0.9)])
def test_registers_bit_exact(ctx, R, gname, model, p):
    g = SMALL[gname]
    pe = np.linspace(0.0, 0.6, g.m, dtype=np.float32) if model == PER_EDGE else None
    assert_build_parity(ctx, g, model, p, R, seed=7 + R, p_edge=pe)


def test_registers_er2000_workload(ctx):
    w = workloads.er_2k()
    assert_build_parity(ctx, w.graph, w.model, w.p, w.R, w.seed)


@pytest.mark.parametrize("scale,ef,model,p,R", [(13, 16, WC, 0.0, 256), (12, 8, IC, 0.05, 128), (14, 16, IC, 0.01, 512)])
def test_registers_rmat_several_tiles(ctx, scale, ef, model, p, R):
    g = graphs.rmat(scale, ef, seed=100 + scale)
    assert_build_parity(ctx, g, model, p, R, seed=scale)


def test_registers_device_and_host_memory_agree(ctx):
    g = graphs.rmat(11, 12, seed=9)
    _, Mh, sh, vh, _ = gpu_build(ctx, g, WC, 0.0, 256, 3)
    _, Md, sd, vd, _ = gpu_build(ctx, g, WC, 0.0, 256, 3, device="cuda")
    assert np.array_equal(Mh, Md) and sh == sd and vh == vd


@pytest.mark.parametrize("eps_c", [0.02, 0.2])
def test_early_exit_matches_oracle(ctx, eps_c):
    g = graphs.rmat(11, 16, seed=11)
    assert_build_parity(ctx, g, WC, 0.0, 128, 5, eps_c=eps_c)


def test_select_er2000_workload(ctx):
    w = workloads.er_2k()
    assert_select_parity(ctx, w.graph, w.model, w.p, w.R, w.K, w.eps_g, w.eps_l, seed=w.seed)


@pytest.mark.parametrize("eps", [(0.0, 0.0), (math.inf, math.inf), (0.01, 0.3), (0.1, 0.5)],
                         ids=["always", "never", "paper", "loose"])
@pytest.mark.parametrize("gname,model,p,R", [("rmat10", WC, 0.0, 64), ("er300", IC, 0.05, 256),
                                             ("hub1500", IC, 0.1, 128), ("er300", IC, 0.05, 512),
                                             ("rmat10", WC, 0.0, 1024)])
def test_select_variants(ctx, eps, gname, model, p, R):
    g = SMALL[gname]
    assert_select_parity(ctx, g, model, p, R, K=8, eps_g=eps[0], eps_l=eps[1], seed=21)


def test_select_per_edge_model(ctx):
    g = graphs.rmat(10, 10, seed=31)
    pe = (np.arange(g.m) % 7 / 20.0).astype(np.float32)
    assert_select_parity(ctx, g, PER_EDGE, 0.0, 128, K=6, eps_g=0.01, p_edge=pe, seed=2)


def test_select_rmat_scale13_wc(ctx):
    g = graphs.rmat(13, 16, seed=41)
    assert_select_parity(ctx, g, WC, 0.0, 256, K=12, eps_g=0.01, seed=2, device="cuda")


@pytest.mark.parametrize("gname,model,p,R", [("rmat10", WC, 0.0, 64), ("er300", IC, 0.05, 128),
                                             ("hub1500", IC, 0.3, 256), ("ragged97", IC, 0.2, 512)])
def test_lazy_argmax_equals_full_scan(monkeypatch, gname, model, p, R):
    """The lazy argmax of the steps that keep the sketch (bounds from earlier scans, exact evaluation of the
    candidates whose bound beats the best exact gain) picks the full scan's seed every step, ties to the smallest
    id included; eps = +inf keeps the sketch for every step after the first."""
    g = SMALL[gname]
    K = min(20, g.n)
    graph = im.Graph.from_synth(g, model, p)
    prm = im.params(R=R, K=K, eps_g=math.inf, eps_l=math.inf, seed=13)
    monkeypatch.setenv("IM_CELF", "0")
    c0 = im.Context(0)
    monkeypatch.delenv("IM_CELF")
    try:
        full = c0.im_select_seeds(graph, prm)
    finally:
        c0.close()
    c1 = im.Context(0)
    try:
        lazy = c1.im_select_seeds(graph, prm)
    finally:
        c1.close()
    for k in ("seeds", "gsum", "rebuilt", "sigma"):
        assert lazy[k].tolist() == full[k].tolist(), k
    ref = oracle.select_seeds(g.n, g.xadj, g.adj, model, p, R, K, math.inf, math.inf, 0.0, 13)
    assert lazy["seeds"].tolist() == ref["seeds"].tolist()


@pytest.mark.parametrize("gname,p,R", [("er2000", 0.03, 512), ("rmat12", 0.02, 256), ("rmat12", 0.01, 1024)])
def test_streamed_push_equals_vertex_push(monkeypatch, gname, p, R):
    """Push sweeps over a large L stream every in-pair when the sampled graph has no dense edges (small p, large R);
    registers, sweeps, visits, frontiers and a whole selection equal the vertex-by-vertex push and the oracle."""
    g = graphs.erdos_renyi(2000, 24000, seed=57) if gname == "er2000" else graphs.rmat(12, 16, seed=58)
    graph = im.Graph.from_synth(g, IC, p)
    outs = []
    for env in ("0", "1"):
        monkeypatch.setenv("IM_STREAM", env)
        c = im.Context(0)
        monkeypatch.delenv("IM_STREAM")
        try:
            sk = c.im_build_sketches(graph, im.params(R=R, seed=4))
            info = sk.im_sketch_info()
            outs.append((sk.im_sketch_registers(), info[0], info[1], info[2].tolist(),
                         c.im_select_seeds(graph, im.params(R=R, K=6, eps_g=0.01, seed=4))))
            sk.close()
        finally:
            c.close()
    (M0, s0, v0, l0, sel0), (M1, s1, v1, l1, sel1) = outs
    assert np.array_equal(M0, M1) and (s0, v0, l0) == (s1, v1, l1)
    for k in ("seeds", "gsum", "rebuilt", "sigma"):
        assert sel0[k].tolist() == sel1[k].tolist(), k
    Mo, so, vo, lo = oracle.build_sketch(g.n, g.xadj, g.adj, IC, p, R, 4)
    assert np.array_equal(M1, Mo) and (s1, v1) == (so, vo)


@pytest.mark.parametrize("pulls,gname,model,p,R", [(2, "rmat10", WC, 0.0, 256), (3, "er300", IC, 0.05, 64),
                                                   (2, "hub1500", IC, 0.3, 512)])
def test_pulled_later_sweeps_equal_the_oracle(monkeypatch, pulls, gname, model, p, R):
    """With IM_PULL_SWEEPS the first sweeps after the first also pull into every row (they read the out-pairs'
    targets and simulations, kept only then); registers, sweeps, visits and a selection with rebuilds still equal the
    oracle's."""
    g = SMALL[gname]
    graph = im.Graph.from_synth(g, model, p)
    monkeypatch.setenv("IM_PULL_SWEEPS", str(pulls))
    c = im.Context(0)
    monkeypatch.delenv("IM_PULL_SWEEPS")
    try:
        sk = c.im_build_sketches(graph, im.params(R=R, seed=8))
        M, sweeps, visits = sk.im_sketch_registers(), *sk.im_sketch_info()[:2]
        sk.close()
        K = min(8, g.n)
        sel = c.im_select_seeds(graph, im.params(R=R, K=K, eps_g=0.0, eps_l=0.0, seed=8))
    finally:
        c.close()
    Mo, so, vo, _ = oracle.build_sketch(g.n, g.xadj, g.adj, model, p, R, 8)
    assert np.array_equal(M, Mo) and (sweeps, visits) == (so, vo)
    ref = oracle.select_seeds(g.n, g.xadj, g.adj, model, p, R, K, 0.0, 0.0, 0.0, 8)
    assert sel["seeds"].tolist() == ref["seeds"].tolist()
    assert sel["gsum"].tolist() == ref["gsum"].tolist()


@pytest.mark.parametrize("env,gname,model,p,R,literal",
                         [({}, "rmat10", WC, 0.0, 64, False), ({}, "hub1500", IC, 0.3, 1024, False),
                          ({"IM_PULL_SWEEPS": "2"}, "er300", IC, 0.05, 256, False),
                          ({"IM_STREAM": "0"}, "ragged97", IC, 0.2, 512, False),
                          ({}, "er300", IC, 0.05, 128, True)])
def test_kept_row_sums_equal_the_registers(monkeypatch, env, gname, model, p, R, literal):
    """The sweeps keep every row's register sum (the first sweep and pulling sweeps store it, the copies after a push
    sweep add what the sweep raised), and the first greedy step after each build starts its argmax from those sums.
    Under IM_TEST_CHECK_SUMS that step scans every row instead and raises a fault if a kept sum differs from the
    row's registers: none may, and the selection equals the oracle's, rebuilds included."""
    g = SMALL[gname]
    K = min(10, g.n)
    graph = im.Graph.from_synth(g, model, p)
    blocking = im.IM_BLOCK_LITERAL if literal else im.IM_BLOCK_RESIDUAL
    prm = im.params(R=R, K=K, eps_g=0.0, eps_l=0.0, seed=17, blocking=blocking)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    monkeypatch.setenv("IM_TEST_CHECK_SUMS", "1")
    c = im.Context(0)
    for k in list(env) + ["IM_TEST_CHECK_SUMS"]:
        monkeypatch.delenv(k)
    try:
        checked = c.im_select_seeds(graph, prm)
    finally:
        c.close()
    ref = oracle.select_seeds(g.n, g.xadj, g.adj, model, p, R, K, 0.0, 0.0, 0.0, 17, literal=literal)
    assert checked["seeds"].tolist() == ref["seeds"].tolist()
    assert checked["gsum"].tolist() == ref["gsum"].tolist()
    assert int(np.sum(checked["rebuilt"])) >= 2


@pytest.mark.parametrize("model,p,R", [(IC, 0.02, 256), (WC, 0.0, 128)])
def test_autotuned_shapes_give_the_same_selection(model, p, R):
    """The autotuner times every candidate launch shape on the first diffusion (it checks they agree) and keeps the
    fastest for the graph's class; a selection under the chosen shape equals the oracle's."""
    g = graphs.rmat(12, 16, seed=59)
    graph = im.Graph.from_synth(g, model, p)
    c = im.Context(0)
    try:
        t = c.im_autotune(graph, im.params(R=R, seed=4))
        assert t["first_sweep_blocks"] in (3, 4, 6) and t["candidates"] >= 3
        assert 0 < t["best_ms"] <= t["default_ms"]
        out = c.im_select_seeds(graph, im.params(R=R, K=6, eps_g=0.01, seed=4))
    finally:
        c.close()
    ref = oracle.select_seeds(g.n, g.xadj, g.adj, model, p, R, 6, 0.01, 0.3, 0.0, 4)
    assert out["seeds"].tolist() == ref["seeds"].tolist()
    assert out["sigma"].tolist() == ref["sigma"].tolist()


# --- literal blocking and undirected inputs ----------------------------------------------------------------------

@pytest.mark.parametrize("eps", [(0.0, 0.0), (0.01, 0.3)], ids=["always", "paper"])
@pytest.mark.parametrize("gname,model,p,R", [("er300", IC, 0.05, 256), ("rmat10", WC, 0.0, 128),
                                             ("hub1500", IC, 0.3, 64), ("er300", IC, 0.05, 512)])
def test_select_literal_blocking(ctx, eps, gname, model, p, R):
    """Algorithms 1 and 2 as printed: blocked registers keep their rank and are never updated (reading R17)."""
    g = SMALL[gname]
    assert_select_parity(ctx, g, model, p, R, K=8, eps_g=eps[0], eps_l=eps[1], seed=21, literal=True)


def test_select_literal_heavy_rows(ctx):
    g = graphs.rmat(12, 16, seed=43)
    assert_select_parity(ctx, g, WC, 0.0, 256, K=10, eps_g=0.0, eps_l=0.0, seed=4, literal=True, device="cuda")


UNDIRECTED = {
    "rmat11s": graphs.symmetrized(graphs.rmat(11, 8, seed=51)),
    "er500s": graphs.symmetrized(graphs.erdos_renyi(500, 2000, seed=52)),
    "hub1500s": graphs.symmetrized(graphs.star_hub(1500, seed=5)),
}


@pytest.mark.parametrize("R", [64, 256, 512])
@pytest.mark.parametrize("gname,model,p", [("rmat11s", IC, 0.05), ("er500s", IC, 0.2), ("hub1500s", WC, 0.0)])
def test_registers_undirected(ctx, R, gname, model, p):
    """Undirected inputs: both directions share the hash key (min, max) (reading R16)."""
    assert_build_parity(ctx, UNDIRECTED[gname], model, p, R, seed=9 + R, undirected=True)


@pytest.mark.parametrize("gname,model,p,R", [("rmat11s", IC, 0.05, 128), ("er500s", IC, 0.1, 256),
                                             ("hub1500s", WC, 0.0, 64)])
def test_select_undirected(ctx, gname, model, p, R):
    assert_select_parity(ctx, UNDIRECTED[gname], model, p, R, K=8, eps_g=0.01, seed=3, undirected=True)


def test_undirected_input_must_be_symmetric(ctx):
    g = graphs.rmat(9, 8, seed=53)  # directed: some (u, v) has no (v, u)
    with pytest.raises(im.ImError) as err:
        ctx.im_build_sketches(im.Graph.from_synth(g, IC, 0.1, undirected=True), im.params(R=64))
    assert err.value.status == 1 and "(v, u)" in str(err.value)


# --- edge cases -------------------------------------------------------------------------------------------------

def test_single_vertex(ctx):
    g = graphs.csr_from_edges(1, np.zeros(0, np.int64), np.zeros(0, np.int64))
    assert_build_parity(ctx, g, IC, 0.5, 64, 1)
    assert_select_parity(ctx, g, IC, 0.5, 64, K=1, eps_g=0.01)


def test_no_edges(ctx):
    g = graphs.csr_from_edges(70, np.zeros(0, np.int64), np.zeros(0, np.int64))
    assert_build_parity(ctx, g, WC, 0.0, 128, 1)
    assert_select_parity(ctx, g, WC, 0.0, 128, K=5, eps_g=0.01)


def test_probability_zero_and_one(ctx):
    g = graphs.rmat(9, 8, seed=51)
    assert_build_parity(ctx, g, IC, 0.0, 64, 2)
    assert_build_parity(ctx, g, IC, 1.0, 64, 2)
    assert_select_parity(ctx, g, IC, 1.0, 64, K=4, eps_g=0.01)


def test_k_equals_n(ctx):
    g = graphs.random_small(24, 60, seed=52)
    assert_select_parity(ctx, g, IC, 0.4, 64, K=24, eps_g=0.01)


def test_long_chain_many_sweeps(ctx):
    g = graphs.chain(3000)
    assert_build_parity(ctx, g, IC, 1.0, 64, 3)


def test_sweep_limit_reports_timeout(ctx):
    g = graphs.chain(500)
    graph = im.Graph.from_synth(g, IC, 1.0)
    with pytest.raises(im.ImError) as ei:
        ctx.im_build_sketches(graph, im.params(R=64, seed=1, max_sweeps=5))
    assert ei.value.status == im._lib.IM_ETIMEOUT


@pytest.mark.parametrize("case", ["decreasing_xadj", "target_out_of_range", "bad_end", "bad_R", "bad_K", "bad_p"])
def test_invalid_arguments(ctx, case):
    g = graphs.random_small(20, 60, seed=53)
    xadj, adj = g.xadj.copy(), g.adj.copy()
    prm = im.params(R=64, K=3)
    p = 0.1
    if case == "decreasing_xadj":
        xadj[5], xadj[6] = xadj[6] + 1, xadj[5]
    elif case == "target_out_of_range":
        adj[3] = 20
    elif case == "bad_end":
        xadj[-1] -= 1
    elif case == "bad_R":
        prm = im.params(R=100, K=3)
    elif case == "bad_K":
        prm = im.params(R=64, K=0)
    elif case == "bad_p":
        p = 1.5
    for device in (None, "cuda"):
        gg = im.Graph.from_synth(graphs.Graph(g.n, xadj, adj), IC, p, device=device)
        with pytest.raises(im.ImError) as ei:
            ctx.im_select_seeds(gg, prm)
        assert ei.value.status == im._lib.IM_EINVAL
    # the context stays usable after a rejected call
    assert_build_parity(ctx, g, IC, 0.1, 64, 1)


# --- estimate ---------------------------------------------------------------------------------------------------

def test_estimate_and_exact_sigma(ctx):
    g = graphs.rmat(12, 12, seed=61)
    R = 256
    sk, Mo = assert_build_parity(ctx, g, WC, 0.0, R, 8)
    probe = oracle.RegisterProbe(g.n, g.xadj, g.adj, WC, 0.0, R, 8)
    for S in ([0], [5, 77, 1000], list(range(0, 4000, 97)), [3, 3, 9]):
        e, sigma = sk.im_estimate(S, exact=True)
        e_ref, _ = oracle.estimate_set(Mo, S)
        assert e == pytest.approx(e_ref, rel=1e-12)
        assert sigma * R == probe.reach_total(sorted(set(S)))
        e2, none = sk.im_estimate(S)
        assert e2 == e and none is None


# --- batch ------------------------------------------------------------------------------------------------------

def test_persistent_search_matches_stepped(monkeypatch):
    """Whole reachability searches in one cooperative launch (IM_PERSISTENT=1) give the stepped launches' result."""
    probs = [workloads.batch_problem(i, max_scale=13) for i in (3, 7, 12)]
    gs = [im.Graph.from_synth(p.graph, p.model, p.p, device="cuda") for p in probs]
    prms = [im.params(R=p.R, K=p.K, eps_g=p.eps_g, eps_l=p.eps_l, seed=p.seed) for p in probs]
    monkeypatch.setenv("IM_PERSISTENT", "1")
    c1 = im.Context(0)
    pers = c1.im_select_seeds_batch(gs, prms)
    c1.close()
    monkeypatch.delenv("IM_PERSISTENT")
    c0 = im.Context(0)
    step = c0.im_select_seeds_batch(gs, prms)
    c0.close()
    for a, b in zip(pers, step):
        assert a["seeds"].tolist() == b["seeds"].tolist() and a["sigma_final"] == b["sigma_final"]


def test_batch_same_R_problems_out_of_phase(ctx):
    """Problems of one R in different phases share every launch: while one pulls the first sweep of a (re)build,
    another pushes, and one tile may serve units of both in the same launch."""
    probs = [workloads.batch_problem(i, max_scale=16) for i in (226, 228, 227, 231, 235)]  # all R = 64
    assert {p.R for p in probs} == {64}
    gs = [im.Graph.from_synth(p.graph, p.model, p.p, device="cuda") for p in probs]
    prms = [im.params(R=p.R, K=p.K, eps_g=p.eps_g, eps_l=p.eps_l, seed=p.seed) for p in probs]
    batch = ctx.im_select_seeds_batch(gs, prms)
    for g, prm, b in zip(gs, prms, batch):
        single = ctx.im_select_seeds(g, prm, trace=False)
        assert b["seeds"].tolist() == single["seeds"].tolist()
        assert b["sigma_final"] == single["sigma_final"] and b["rebuilds"] == single["rebuilds"]
    p = probs[3]  # the smallest: also against the oracle
    ref = oracle.select_seeds(p.graph.n, p.graph.xadj, p.graph.adj, p.model, p.p, p.R, p.K, p.eps_g, p.eps_l, 0.0,
                              p.seed)
    assert batch[3]["seeds"].tolist() == ref["seeds"].tolist()


def test_batch_equals_individual_and_oracle(ctx):
    probs = [workloads.batch_problem(i, max_scale=11) for i in range(10)]
    gs = [im.Graph.from_synth(p.graph, p.model, p.p) for p in probs]
    prms = [im.params(R=p.R, K=p.K, eps_g=p.eps_g, eps_l=p.eps_l, seed=p.seed) for p in probs]
    batch = ctx.im_select_seeds_batch(gs, prms)
    for p, g, prm, b in zip(probs, gs, prms, batch):
        single = ctx.im_select_seeds(g, prm)
        assert b["seeds"].tolist() == single["seeds"].tolist()
        assert b["sigma_final"] == single["sigma_final"] and b["rebuilds"] == single["rebuilds"]
        ref = oracle.select_seeds(p.graph.n, p.graph.xadj, p.graph.adj, p.model, p.p, p.R, p.K, p.eps_g, p.eps_l,
                                  0.0, p.seed)
        assert b["seeds"].tolist() == ref["seeds"].tolist()
        assert b["sigma_final"] == ref["sigma"][-1]
