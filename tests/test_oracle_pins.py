"""Pins for the CPU oracle: published test vectors, exact closed forms, brute force on tiny graphs and invariants.

Each test ties one oracle function to something other than the oracle itself, so that a dropped term, a wrong sign,
a swapped operand or a wrong index in it fails here.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import bruteforce as bf
from synth import graphs

IC, WC, PER_EDGE = 0, 1, 2


# --- hash primitives -------------------------------------------------------------------------------------------

def test_fmix32_published_vectors(orc):
    # MurmurHash3_x86_32 of the empty key with seed s reduces to fmix32(s); the published values for seeds 0, 1 and
    # 0xFFFFFFFF are 0, 0x514E28B7 and 0x81F16F39.
    assert orc.fmix32(0) == 0
    assert orc.fmix32(1) == 0x514E28B7
    assert orc.fmix32(0xFFFFFFFF) == 0x81F16F39


def test_fmix32_is_a_bijection_on_a_sample(orc):
    xs = np.random.PCG64(7).random_raw(20000) & 0xFFFFFFFF
    ys = {orc.fmix32(int(x)) for x in xs}
    assert len(ys) == len(set(int(x) for x in xs))


def test_splitmix64_published_vector(orc):
    # The reference sequence of splitmix64 (Steele, Lea & Flood 2014; Vigna's splitmix64.c) from seed 1234567.
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431, 16408922859458223821]
    assert [orc.splitmix64(1234567, i) for i in range(5)] == ref


def test_sim_words_take_alternate_outputs(orc):
    # X_r is the high half of output 2r, Y_r of output 2r+1 (reading R3), checked on the published sequence.
    X, Y = orc.sim_words(1234567, 2)
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431]
    assert [int(X[0]), int(Y[0]), int(X[1]), int(Y[1])] == [r >> 32 for r in ref]


def test_clz32_matches_bit_length(orc):
    xs = [0, 1, 2, 3, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF] + [int(x) for x in
                                                               np.random.PCG64(3).random_raw(2000) >> np.uint64(
                                                                   np.random.PCG64(4).random_raw(1)[0] % 32 + 32)]
    for x in xs:
        x &= 0xFFFFFFFF
        assert orc.clz32(x) == 32 - x.bit_length()


def test_edge_hash_is_fmix32_of_small_keys(orc):
    # Where u*n+v fits in 32 bits the edge hash is exactly fmix32(u*n+v), the form named for the 2000-vertex graph.
    n = 2000
    for u, v in [(0, 1), (1, 0), (5, 1999), (1999, 1998), (1234, 567)]:
        assert orc.edge_hash(u, v, n) == orc.fmix32(u * n + v)


def test_edge_hash_keeps_high_key_bits(orc):
    # For n = 2^20, (u, v) and (u + 4096, v) agree in the low 32 bits of u*n+v; their hashes must still differ.
    n = 1 << 20
    same = sum(orc.edge_hash(u, v, n) == orc.edge_hash(u + 4096, v, n) for u in range(0, 4096, 97) for v in (0, 77))
    assert same == 0


def test_init_rank_is_clz_of_vertex_hash_xor_word(orc):
    for v in [0, 1, 2, 1999, 1 << 20, (1 << 22) - 1]:
        for y in [0, 1, 0xDEADBEEF, 0xFFFFFFFF]:
            hv = orc.fmix32((v ^ 0x9E3779B9) & 0xFFFFFFFF)
            assert orc.init_rank(v, y) == 32 - (hv ^ y).bit_length()


# --- sampling test (Eq. 4-5) -----------------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1e-9, 2.3283064365386963e-10, 0.005, 0.01, 0.05, 0.1, 1 / 3, 0.5, 0.999999, 1.0,
                               0.123456789])
def test_threshold_gives_smallest_grid_probability_not_below_p(orc, p):
    # Live iff (h ^ X) <= T, so P(live) = (T+1)/2^32 over uniform X; that must be the least multiple of 2^-32
    # that is >= p (Eq. 5 with h_max = 2^32: P < w).
    ok, T = orc.threshold_from_p(p)
    assert ok == 1
    q = Fraction(p)
    assert Fraction(T + 1, 1 << 32) >= q
    assert Fraction(T, 1 << 32) < q


def test_threshold_of_the_2000_vertex_workload(orc):
    assert orc.threshold_from_p(0.05) == (1, 214748364)


@pytest.mark.parametrize("p", [0.0, -0.5])
def test_nonpositive_probability_never_samples(orc, p):
    ok, _ = orc.threshold_from_p(p)
    assert ok == 0
    assert not orc.is_live(0, 0, 0xFFFFFFFF, 0)


def test_live_compare_direction_and_bound(orc):
    # Feeding X = h ^ t makes (h ^ X) = t, so the test must accept exactly t <= T.
    h = 0x12345678
    for T in [0, 1, 214748364, 0x7FFFFFFF, 0xFFFFFFFE, 0xFFFFFFFF]:
        for t in {0, max(T - 1, 0), T, min(T + 1, 0xFFFFFFFF), 0xFFFFFFFF}:
            assert orc.is_live(h, h ^ t, T, 1) == (t <= T)


def test_weighted_cascade_threshold_is_one_over_indegree(orc):
    # WC uses p(u,v) = 1/indeg(v) (Section 2.1); the threshold must satisfy the same exact property with q = 1/d.
    g = graphs.random_small(40, 400, seed=11)
    T, ok = orc.edge_thresholds(g.n, g.xadj, g.adj, WC)
    indeg = np.bincount(g.adj, minlength=g.n)
    for e in range(g.m):
        d = int(indeg[g.adj[e]])
        assert ok[e] == 1
        assert Fraction(int(T[e]) + 1, 1 << 32) >= Fraction(1, d) > Fraction(int(T[e]), 1 << 32)


def test_per_edge_thresholds(orc):
    g = graphs.random_small(20, 100, seed=12)
    pe = np.linspace(0.0, 1.0, g.m, dtype=np.float32)
    T, ok = orc.edge_thresholds(g.n, g.xadj, g.adj, PER_EDGE, p_edge=pe)
    for e in range(g.m):
        ok1, t1 = orc.threshold_from_p(float(pe[e]))
        assert ok[e] == ok1 and (not ok1 or T[e] == t1)


def test_live_fraction_matches_probability(orc):
    # Section 3.1 (Fig. 3-4) argues the hash-based draws behave like uniform ones: over ~2.6M (edge, simulation)
    # pairs the live fraction must sit within 5 standard deviations of (T+1)/2^32, and per-simulation counts must
    # pass a chi-square test.
    g = graphs.erdos_renyi(2000, 20000, seed=1)
    X, _ = orc.sim_words(99, 128)
    p = 0.05
    _, T = orc.threshold_from_p(p)
    q = (T + 1) / 2 ** 32
    src, dst = g.edges()
    h = np.array([orc.edge_hash(int(u), int(v), g.n) for u, v in zip(src, dst)], dtype=np.uint32)
    live = (h[:, None] ^ X[None, :]) <= np.uint32(T)  # the oracle's live test is checked pointwise below
    for e in range(0, g.m, 997):
        for j in range(0, 128, 13):
            assert live[e, j] == orc.is_live(int(h[e]), int(X[j]), T, 1)
    N = live.size
    sd = math.sqrt(N * q * (1 - q))
    assert abs(live.sum() - N * q) < 5 * sd
    per_sim = live.sum(axis=0)
    exp = g.m * q
    chi2 = float(((per_sim - exp) ** 2 / (exp * (1 - q))).sum())
    # 127 degrees of freedom: the 1e-6 upper tail is about 230
    assert chi2 < 230


# --- diffusion (Algorithm 2) -----------------------------------------------------------------------------------

def _problem(orc, g, model, p, R, seed, p_edge=None):
    T, ok = orc.edge_thresholds(g.n, g.xadj, g.adj, model, p=p, p_edge=p_edge)
    X, Y = orc.sim_words(seed, R)
    return T, ok, X, Y


CASES = [
    ("ic0.05", graphs.random_small(48, 300, 21), IC, 0.05, None),
    ("ic0.3", graphs.random_small(40, 160, 22), IC, 0.3, None),
    ("ic0.7", graphs.random_small(33, 90, 23), IC, 0.7, None),
    ("wc", graphs.random_small(64, 400, 24), WC, 0.0, None),
    ("per_edge", graphs.random_small(30, 120, 25), PER_EDGE, 0.0, "ramp"),
    ("chainish", graphs.chain(20), IC, 0.9, None),
]


@pytest.mark.parametrize("name,g,model,p,pe", CASES, ids=[c[0] for c in CASES])
def test_registers_equal_bruteforce_reach_maxima(orc, name, g, model, p, pe):
    p_edge = np.linspace(0.0, 0.9, g.m, dtype=np.float32) if pe == "ramp" else None
    R = 64
    T, ok, X, Y = _problem(orc, g, model, p, R, seed=5, p_edge=p_edge)
    M, sweeps, visits, log = orc.build_sketch(g.n, g.xadj, g.adj, model, p, R, seed=5, p_edge=p_edge)
    live = bf.live_matrix(orc, g.n, g.xadj, g.adj, T, ok, X)
    ref = bf.registers(orc, g.n, g.xadj, g.adj, live, Y)
    assert np.array_equal(M, ref)
    assert log[0] == g.n and visits >= g.m * R


def test_blocked_registers_equal_residual_reach_maxima(orc):
    g = graphs.random_small(40, 200, 31)
    R = 64
    T, ok, X, Y = _problem(orc, g, IC, 0.3, R, seed=8)
    live = bf.live_matrix(orc, g.n, g.xadj, g.adj, T, ok, X)
    reached = np.zeros((g.n, R), np.uint8)
    for s in (3, 17):
        orc.reach_add(g.n, g.xadj, g.adj, T, ok, R, X, s, reached)
    assert np.array_equal(reached, bf.reached_by(g.n, g.xadj, g.adj, live, [3, 17], R))
    M = orc.init_registers(g.n, R, Y, blocked=reached)
    orc.simulate(g.n, g.xadj, g.adj, T, ok, R, X, M, blocked=reached)
    ref = bf.registers(orc, g.n, g.xadj, g.adj, live, Y, blocked=reached.astype(bool))
    assert np.array_equal(M, ref)


def test_probability_zero_leaves_initial_ranks(orc):
    g = graphs.random_small(50, 300, 41)
    R = 64
    M, sweeps, visits, log = orc.build_sketch(g.n, g.xadj, g.adj, IC, 0.0, R, seed=3)
    _, Y = orc.sim_words(3, R)
    ref = np.array([[32 - (orc.fmix32(v ^ 0x9E3779B9) ^ int(Y[j])).bit_length() for j in range(R)]
                    for v in range(g.n)], dtype=np.uint8)
    assert np.array_equal(M, ref)
    assert sweeps == 1 and visits == g.m * R


def test_probability_one_gives_transitive_closure_maxima(orc):
    # With every edge live, M_v[j] is the max initial rank over everything v reaches (scipy's traversal, not ours).
    g = graphs.random_small(60, 150, 42)
    R = 64
    M, *_ = orc.build_sketch(g.n, g.xadj, g.adj, IC, 1.0, R, seed=4)
    _, Y = orc.sim_words(4, R)
    A = sp.csr_matrix((np.ones(g.m), g.adj, g.xadj), shape=(g.n, g.n))
    rank = np.array([[orc.init_rank(v, int(Y[j])) for j in range(R)] for v in range(g.n)])
    for v in range(g.n):
        reach = csg.breadth_first_order(A, v, directed=True, return_predecessors=False)
        assert np.array_equal(M[v], rank[reach].max(axis=0))


@pytest.mark.parametrize("reverse", [False, True], ids=["forward", "reverse"])
def test_chain_sweep_count_is_the_longest_propagation_distance(orc, reverse):
    # On a path with every edge live, Jacobi sweep t sets M_u to the max over the t vertices downstream of u; the
    # last change happens at t* = max over (u, j) of the distance from u to the first downstream maximum, and one
    # more sweep finds nothing, so sweeps = t* + 1.  Visits: sweep t processes u iff its successor changed in sweep
    # t-1.  The reversed path (edges i -> i-1) makes in-place updates in id order finish early, so it tells Jacobi
    # sweeps apart from Gauss-Seidel ones.
    L = 40
    if reverse:
        g = graphs.csr_from_edges(L, np.arange(1, L), np.arange(L - 1))
        succ = lambda u: u - 1 if u > 0 else None  # noqa: E731
        order = lambda u: list(range(u, -1, -1))  # noqa: E731
    else:
        g = graphs.chain(L)
        succ = lambda u: u + 1 if u < L - 1 else None  # noqa: E731
        order = lambda u: list(range(u, L))  # noqa: E731
    R = 64
    M, sweeps, visits, log = orc.build_sketch(g.n, g.xadj, g.adj, IC, 1.0, R, seed=6)
    _, Y = orc.sim_words(6, R)
    rank = np.array([[orc.init_rank(v, int(Y[j])) for j in range(R)] for v in range(L)])
    tstar = 0
    for j in range(R):
        for u in range(L):
            downstream = rank[order(u), j]
            tstar = max(tstar, int(np.argmax(downstream)))
    assert sweeps == tstar + 1
    cur = rank.copy()
    changed = np.ones(L, bool)
    total = 0
    for _ in range(sweeps):
        nxt = cur.copy()
        for u in range(L):
            v = succ(u)
            if v is not None and changed[v]:
                total += R
                nxt[u] = np.maximum(nxt[u], cur[v])
        changed = (nxt != cur).any(axis=1)
        cur = nxt
    assert visits == total
    assert np.array_equal(M, cur)


def test_blocked_registers_never_update_even_if_the_set_is_not_closed(orc):
    # Algorithm 2 skips the update of a blocked (u, j) outright.  With the reach set of a seed set as the blocked
    # set that check can never fire (a blocked vertex only reaches blocked ones), so an arbitrary mask is used here:
    # a blocked register stays 0 and relays nothing.
    g = graphs.random_small(40, 220, 33)
    R = 64
    T, ok, X, Y = _problem(orc, g, IC, 0.5, R, seed=12)
    live = bf.live_matrix(orc, g.n, g.xadj, g.adj, T, ok, X)
    blocked = (np.random.PCG64(5).random_raw(g.n * R).reshape(g.n, R) % 5 == 0).astype(np.uint8)
    M = orc.init_registers(g.n, R, Y, blocked=blocked)
    orc.simulate(g.n, g.xadj, g.adj, T, ok, R, X, M, blocked=blocked)
    ref = bf.registers(orc, g.n, g.xadj, g.adj, live, Y, blocked=blocked.astype(bool))
    assert np.array_equal(M, ref)


def test_converged_registers_are_a_fixpoint(orc):
    g = graphs.random_small(64, 500, 51)
    R = 128
    T, ok, X, Y = _problem(orc, g, WC, 0.0, R, seed=9)
    M, *_ = orc.build_sketch(g.n, g.xadj, g.adj, WC, 0.0, R, seed=9)
    M2 = M.copy()
    sweeps, visits, log = orc.simulate(g.n, g.xadj, g.adj, T, ok, R, X, M2)
    assert sweeps == 1 and np.array_equal(M, M2)


def test_result_is_schedule_independent(orc):
    # In-place (Gauss-Seidel) updates in a random vertex order reach the same least fixpoint.
    g = graphs.random_small(50, 260, 52)
    R = 64
    T, ok, X, Y = _problem(orc, g, IC, 0.4, R, seed=10)
    live = bf.live_matrix(orc, g.n, g.xadj, g.adj, T, ok, X)
    M, *_ = orc.build_sketch(g.n, g.xadj, g.adj, IC, 0.4, R, seed=10)
    G = np.array([[orc.init_rank(v, int(Y[j])) for j in range(R)] for v in range(g.n)], dtype=np.uint8)
    order = np.random.default_rng(0).permutation(g.n)
    changed = True
    while changed:
        changed = False
        for u in order:
            for e in range(g.xadj[u], g.xadj[u + 1]):
                v = g.adj[e]
                new = np.where(live[e], np.maximum(G[u], G[v]), G[u])
                if (new != G[u]).any():
                    G[u] = new
                    changed = True
    assert np.array_equal(M, G)


def test_early_exit_stops_at_first_small_frontier(orc):
    g = graphs.random_small(64, 400, 53)
    R = 64
    _, s_full, _, log_full = orc.build_sketch(g.n, g.xadj, g.adj, IC, 0.5, R, seed=11)
    eps_c = 0.1
    _, s_cut, _, log_cut = orc.build_sketch(g.n, g.xadj, g.adj, IC, 0.5, R, seed=11, eps_c=eps_c)
    sizes = list(log_full[1:]) + [0]  # |L'| after each sweep of the full run
    first = next(i for i, x in enumerate(sizes) if x <= eps_c * g.n)
    assert s_cut == first + 1
    assert np.array_equal(log_cut, log_full[: s_cut])


# --- greedy loop (Algorithm 1) ---------------------------------------------------------------------------------

def _greedy_case(orc, g, model, p, R, K, eps_g, eps_l, seed):
    T, ok, X, Y = _problem(orc, g, model, p, R, seed)
    live = bf.live_matrix(orc, g.n, g.xadj, g.adj, T, ok, X)
    ref = bf.greedy(orc, g.n, g.xadj, g.adj, live, Y, K, eps_g, eps_l)
    out = orc.select_seeds(g.n, g.xadj, g.adj, model, p, R, K, eps_g, eps_l, seed=seed)
    assert out["seeds"].tolist() == ref["seeds"]
    assert out["gsum"].tolist() == ref["gsum"]
    assert out["rebuilt"].tolist() == ref["rebuilt"]
    assert np.array_equal(out["sigma"], np.array(ref["sigma"]))
    assert np.array_equal(out["est"], np.array(ref["est"]))
    return out


@pytest.mark.parametrize("eps", [(0.0, 0.0), (math.inf, math.inf), (0.01, 0.3), (0.2, 0.9)],
                         ids=["always", "never", "paper", "loose"])
@pytest.mark.parametrize("gseed", [61, 62, 63])
def test_greedy_equals_bruteforce_on_tiny_graphs(orc, eps, gseed):
    g = graphs.random_small(12, 30, gseed)
    _greedy_case(orc, g, IC, 0.5, 64, 3, eps[0], eps[1], seed=gseed)


def test_greedy_bruteforce_weighted_cascade_longer(orc):
    g = graphs.random_small(24, 80, 64)
    out = _greedy_case(orc, g, WC, 0.0, 64, 6, 0.01, 0.3, seed=3)
    assert len(set(out["seeds"].tolist())) == 6


@pytest.mark.parametrize("eps", [(0.0, 0.0), (math.inf, math.inf), (0.01, 0.3)], ids=["always", "never", "paper"])
def test_greedy_bruteforce_every_vertex_a_seed(orc, eps):
    # K = n: once the remaining gains all tie the argmax must still skip S (reading R9) and end with every vertex
    g = graphs.random_small(9, 14, 66)
    out = _greedy_case(orc, g, IC, 0.5, 64, g.n, eps[0], eps[1], seed=5)
    assert sorted(out["seeds"].tolist()) == list(range(g.n))


def test_greedy_bruteforce_step_that_reaches_nothing_new(orc):
    # A star with p = 1: the hub reaches every leaf in every sample.  With thresholds near 0 the first step rebuilds
    # (sigma becomes the reference), so the second seed, a leaf, has delta = 0: err_l is +infinity (reading R8) and
    # err_g = e / sigma is far above the threshold, so that step rebuilds too.
    g = graphs.csr_from_edges(10, np.zeros(9, np.int64), np.arange(1, 10))
    out = _greedy_case(orc, g, IC, 1.0, 64, 3, 1e-9, 1e-9, seed=4)
    assert out["seeds"].tolist()[0] == 0 and out["sigma"].tolist() == [10.0, 10.0, 10.0]
    assert out["rebuilt"].tolist() == [1, 1, 1]


def test_simulate_stops_at_the_sweep_limit(orc):
    # a 40-vertex chain with every edge live needs a sweep per hop; a limit of 7 stops after exactly 7 sweeps
    g = graphs.chain(40)
    T, ok, X, Y = _problem(orc, g, IC, 1.0, 64, 3)
    full = orc.simulate(g.n, g.xadj, g.adj, T, ok, 64, X, orc.init_registers(g.n, 64, Y))[0]
    assert full >= 39
    assert orc.simulate(g.n, g.xadj, g.adj, T, ok, 64, X, orc.init_registers(g.n, 64, Y), max_sweeps=7)[0] == 7


def test_simulate_empty_graph(orc):
    sweeps, visits, log = orc.simulate(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint32),
                                       np.zeros(0, np.uint8), 64, np.zeros(64, np.uint32), np.zeros((0, 64), np.uint8))
    assert (sweeps, visits, len(log)) == (0, 0, 0)


@pytest.mark.parametrize("K,R", [(0, 64), (13, 64), (3, 0)])
def test_select_seeds_rejects_bad_arguments(orc, K, R):
    g = graphs.random_small(12, 30, 61)
    with pytest.raises(RuntimeError):
        orc.select_seeds(g.n, g.xadj, g.adj, IC, 0.5, R, K, 0.01, 0.3, seed=1)


def test_never_rebuild_runs_one_diffusion_and_always_rebuild_runs_k(orc):
    g = graphs.random_small(30, 120, 65)
    never = orc.select_seeds(g.n, g.xadj, g.adj, IC, 0.3, 64, 5, math.inf, math.inf, seed=2)
    always = orc.select_seeds(g.n, g.xadj, g.adj, IC, 0.3, 64, 5, 0.0, 0.0, seed=2)
    assert never["builds"] == 1 and never["rebuilt"].sum() == 0
    assert always["builds"] == 5 and always["rebuilt"].sum() == 5  # the K-th rebuild is decided, not run


def test_estimate_is_eq2(orc):
    for g_sum, R in [(0, 64), (64, 64), (149, 64), (1000, 256), (16384, 512)]:
        assert orc.estimate_from_sum(g_sum, R) == pytest.approx(2.0 ** (g_sum / R) / 0.77351, rel=1e-15)
    M = np.array([[1, 5, 0, 2], [3, 0, 0, 7], [0, 0, 4, 0]], np.uint8)
    e, gsum = orc.estimate_set(M, [0, 1])
    assert gsum == 3 + 5 + 0 + 7
    assert e == pytest.approx(2.0 ** (15 / 4) / 0.77351, rel=1e-15)


def test_register_probe_equals_bruteforce(orc):
    g = graphs.random_small(40, 200, 71)
    R = 64
    T, ok, X, Y = _problem(orc, g, WC, 0.0, R, seed=13)
    live = bf.live_matrix(orc, g.n, g.xadj, g.adj, T, ok, X)
    ref = bf.registers(orc, g.n, g.xadj, g.adj, live, Y)
    probe = orc.RegisterProbe(g.n, g.xadj, g.adj, WC, 0.0, R, 13)
    for v in range(g.n):
        for j in range(0, R, 7):
            assert probe(v, j) == ref[v, j]
    assert probe.reach_total([1, 5]) == int(bf.reached_by(g.n, g.xadj, g.adj, live, [1, 5], R).sum())


# --- influence scoring: mt19937 sample-then-diffuse (Section 4's separate influence oracle, reading R15) ---------

def test_mt19937_value_fixed_by_the_cpp_standard(orc):
    # [rand.predef]: the 10000th consecutive output of a default-constructed std::mt19937 (seed 5489) is 4123659995.
    assert int(orc.mt_outputs(5489, 10000)[-1]) == 4123659995


@pytest.mark.parametrize("seed", [1, 5489, 0xDEADBEEF, 0xFFFFFFFF])
def test_mt19937_matches_numpy(orc, seed):
    # numpy's RandomState seeds its own MT19937 with init_genrand for an integer seed; a full-range uint32 draw is
    # one raw output.  2000 outputs span four twists of the state.
    ref = np.random.RandomState(seed).randint(0, 2 ** 32, size=2000, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(orc.mt_outputs(seed, 2000), ref)


def _reach_count(g, live, seeds):
    """Vertices reached from `seeds` over the edges flagged in `live` (scipy breadth-first order per seed)."""
    src = np.repeat(np.arange(g.n), np.diff(g.xadj))
    keep = live.astype(bool)
    A = sp.csr_matrix((np.ones(int(keep.sum())), (src[keep], g.adj[keep])), shape=(g.n, g.n))
    seen = np.zeros(g.n, bool)
    for s in set(int(x) for x in seeds):
        seen[csg.breadth_first_order(A, s, directed=True, return_predecessors=False)] = True
    return int(seen.sum())


def test_influence_mc_equals_a_search_over_numpy_drawn_edges(orc):
    # 20000+ edges: three generator streams per sample, so the per-chunk reseeding and the in-chunk output index
    # are both exercised.  Edges are drawn here with numpy's MT19937 and the stream seeds of reading R15 (the high
    # half of splitmix64 output s * nchunks + chunk), then searched with scipy.
    g = graphs.erdos_renyi(3000, 21000, seed=41)
    m = g.adj.shape[0]
    assert m > 2 * orc.MC_CHUNK
    nchunks = -(-m // orc.MC_CHUNK)
    for model, p in ((IC, 0.12), (WC, 0.0)):
        T, ok = orc.edge_thresholds(g.n, g.xadj, g.adj, model, p)
        seeds = [7, 100, 7, 2999]
        total, reach = orc.influence_mc(g.n, g.xadj, g.adj, model, p, seeds, 6, seed=99)
        for s in range(6):
            draws = np.concatenate([
                np.random.RandomState(orc.splitmix64(99, s * nchunks + c) >> 32).randint(
                    0, 2 ** 32, size=min(orc.MC_CHUNK, m - c * orc.MC_CHUNK), dtype=np.uint64)
                for c in range(nchunks)])
            live = ok.astype(bool) & (draws <= T)
            assert reach[s] == _reach_count(g, live, seeds), (model, s)
        assert total == int(reach.sum())


def test_influence_mc_closed_forms(orc):
    g = graphs.random_small(60, 240, seed=5)
    seeds = [3, 3, 17]
    # p = 0: nothing is live, every sample reaches exactly the distinct seeds
    _, r0 = orc.influence_mc(g.n, g.xadj, g.adj, IC, 0.0, seeds, 64, seed=1)
    assert (r0 == 2).all()
    # p = 1: every edge is live, every sample reaches the seeds' reachability set in G
    _, r1 = orc.influence_mc(g.n, g.xadj, g.adj, IC, 1.0, seeds, 64, seed=1)
    assert (r1 == _reach_count(g, np.ones(g.adj.shape[0], np.uint8), seeds)).all()


def test_influence_mc_draw_equal_to_threshold_is_live(orc):
    # Reading R4's bound in the scorer: an edge whose draw equals its threshold is live.  On a star, every edge whose
    # sample-0 draw d is below 2^24 gets p = (d + 1) / 2^32 (exact in float32, so T = ceil(p 2^32) - 1 = d); every
    # other edge gets p = 0.  The hub then reaches exactly those leaves in sample 0.
    L = 6000
    g = graphs.csr_from_edges(L + 1, np.zeros(L, np.int64), np.arange(1, L + 1))
    draws = orc.mt_outputs(orc.mc_stream_seed(31, 0, 0, 1), L)
    hit = draws < (1 << 24)
    pe = np.zeros(L, np.float32)
    pe[hit] = ((draws[hit].astype(np.float64) + 1.0) / 2.0 ** 32).astype(np.float32)
    assert np.array_equal(pe[hit].astype(np.float64) * 2.0 ** 32 - 1.0, draws[hit].astype(np.float64))
    assert hit.sum() >= 5
    T, ok = orc.edge_thresholds(g.n, g.xadj, g.adj, PER_EDGE, 0.0, pe)
    assert np.array_equal(T[hit], draws[hit])
    _, reach = orc.influence_mc(g.n, g.xadj, g.adj, PER_EDGE, 0.0, [0], 1, 31, p_edge=pe)
    assert int(reach[0]) == 1 + int(hit.sum())


def test_influence_mc_star_expectation(orc):
    # A star: the hub reaches each of its L leaves with probability p, so the mean reach is 1 + L p with standard
    # error sqrt(L p (1 - p) / N); the mean over N = 4000 samples lies within 5 standard errors.
    L, p, N = 200, 0.3, 4000
    g = graphs.csr_from_edges(L + 1, np.zeros(L, np.int64), np.arange(1, L + 1))
    total, reach = orc.influence_mc(g.n, g.xadj, g.adj, IC, p, [0], N, seed=2024)
    assert abs(total / N - (1 + L * p)) < 5 * math.sqrt(L * p * (1 - p) / N)
    assert reach.min() >= 1 and reach.max() <= L + 1
    # a leaf as the only seed reaches itself alone
    assert orc.influence_mc(g.n, g.xadj, g.adj, IC, p, [5], 64, seed=3)[0] == 64


# --- literal blocking (reading R17) and undirected inputs (reading R16) ------------------------------------------

@pytest.mark.parametrize("eps", [(0.0, 0.0), (0.01, 0.3), (0.2, 0.9)], ids=["always", "paper", "loose"])
@pytest.mark.parametrize("gseed", [61, 63])
def test_literal_blocking_greedy_equals_bruteforce(orc, eps, gseed):
    # Algorithms 1 and 2 as printed: a rebuild re-initialises every register and Simulate skips only the blocked
    # (u, j), so a blocked vertex keeps its rank and still passes it to unblocked in-neighbours
    g = graphs.random_small(12, 30, gseed)
    T, ok, X, Y = _problem(orc, g, IC, 0.5, 64, gseed)
    live = bf.live_matrix(orc, g.n, g.xadj, g.adj, T, ok, X)
    ref = bf.greedy(orc, g.n, g.xadj, g.adj, live, Y, 4, eps[0], eps[1], literal=True)
    out = orc.select_seeds(g.n, g.xadj, g.adj, IC, 0.5, 64, 4, eps[0], eps[1], seed=gseed, literal=True)
    assert out["seeds"].tolist() == ref["seeds"]
    assert out["gsum"].tolist() == ref["gsum"]
    assert out["rebuilt"].tolist() == ref["rebuilt"]
    assert np.array_equal(out["sigma"], np.array(ref["sigma"]))


def test_literal_blocking_registers_keep_their_rank(orc):
    # after blocking, a literal rebuild's blocked registers are exactly the initial ranks, the residual ones 0
    g = graphs.random_small(30, 120, 67)
    R = 64
    T, ok, X, Y = _problem(orc, g, IC, 0.4, R, 9)
    live = bf.live_matrix(orc, g.n, g.xadj, g.adj, T, ok, X)
    blocked = bf.reached_by(g.n, g.xadj, g.adj, live, [0, 5], R).astype(bool)
    assert blocked.any() and not blocked.all()
    init = orc.init_registers(g.n, R, Y)
    lit = init.copy()
    orc.simulate(g.n, g.xadj, g.adj, T, ok, R, X, lit, blocked=blocked.astype(np.uint8))
    assert np.array_equal(lit[blocked], init[blocked])
    assert np.array_equal(lit, bf.registers(orc, g.n, g.xadj, g.adj, live, Y, blocked=blocked, literal=True))
    res = orc.init_registers(g.n, R, Y, blocked=blocked.astype(np.uint8))
    orc.simulate(g.n, g.xadj, g.adj, T, ok, R, X, res, blocked=blocked.astype(np.uint8))
    assert np.array_equal(res, bf.registers(orc, g.n, g.xadj, g.adj, live, Y, blocked=blocked))
    assert not np.array_equal(lit, res)


def _symmetric(n, m, seed):
    g = graphs.random_small(n, m, seed)
    src, dst = g.edges()
    return graphs.csr_from_edges(n, np.concatenate([src, dst]), np.concatenate([dst, src]))


def test_undirected_edge_key_is_symmetric(orc):
    n = 1000
    for u, v in [(0, 1), (3, 999), (512, 17), (998, 999)]:
        h = orc.edge_hash(min(u, v), max(u, v), n)
        assert orc.edge_hash_dir(u, v, n, True) == h == orc.edge_hash_dir(v, u, n, True)
        assert orc.edge_hash_dir(u, v, n, False) == orc.edge_hash(u, v, n)


def test_undirected_weighted_cascade_equals_bruteforce(orc):
    # weighted cascade keeps a threshold per direction (1 / indeg of the target), so the shared key couples the two
    # directions without making them equal; registers are still the brute-force reach-set maxima
    g = _symmetric(40, 60, 82)
    M, _, _, _ = orc.build_sketch(g.n, g.xadj, g.adj, WC, 0.0, 64, seed=5, undirected=True)
    T, ok, X, Y = _problem(orc, g, WC, 0.0, 64, 5)
    live = bf.live_matrix(orc, g.n, g.xadj, g.adj, T, ok, X, undirected=True)
    assert np.array_equal(M, bf.registers(orc, g.n, g.xadj, g.adj, live, Y))


@pytest.mark.parametrize("model,p", [(IC, 0.25), (IC, 0.6)])
def test_undirected_registers_are_component_maxima(orc, model, p):
    # with one probability for both directions, an edge is live in both directions together, so the reach set of v
    # in a sample is its connected component: every register is the largest rank over the component (scipy's
    # components, independent of the oracle)
    g = _symmetric(40, 60, 81)
    R = 64
    M, sweeps, visits, _ = orc.build_sketch(g.n, g.xadj, g.adj, model, p, R, seed=5, undirected=True)
    T, ok, X, Y = _problem(orc, g, model, p, R, 5)
    live = bf.live_matrix(orc, g.n, g.xadj, g.adj, T, ok, X, undirected=True)
    src = np.repeat(np.arange(g.n), np.diff(g.xadj))
    rank = np.array([[orc.init_rank(v, int(Y[j])) for j in range(R)] for v in range(g.n)])
    for j in range(R):
        e = live[:, j]
        A = sp.coo_matrix((np.ones(int(e.sum())), (src[e], g.adj[e])), shape=(g.n, g.n)).tocsr()
        assert (A != A.T).nnz == 0  # the live sample is symmetric
        _, comp = csg.connected_components(A, directed=False)
        for c in np.unique(comp):
            members = comp == c
            assert np.all(M[members, j] == rank[members, j].max())
    assert np.array_equal(M, bf.registers(orc, g.n, g.xadj, g.adj, live, Y))


def test_undirected_greedy_equals_bruteforce(orc):
    g = _symmetric(14, 20, 83)
    T, ok, X, Y = _problem(orc, g, IC, 0.4, 64, 6)
    live = bf.live_matrix(orc, g.n, g.xadj, g.adj, T, ok, X, undirected=True)
    ref = bf.greedy(orc, g.n, g.xadj, g.adj, live, Y, 4, 0.01, 0.3)
    out = orc.select_seeds(g.n, g.xadj, g.adj, IC, 0.4, 64, 4, 0.01, 0.3, seed=6, undirected=True)
    assert out["seeds"].tolist() == ref["seeds"]
    assert out["gsum"].tolist() == ref["gsum"]
    assert np.array_equal(out["sigma"], np.array(ref["sigma"]))
