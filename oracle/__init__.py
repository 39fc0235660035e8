"""CPU oracle for HyperFuseR (arXiv 2105.04023): ctypes front end to ``oracle.c``.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
this package; the CUDA library never imports, links or calls it.  The C source states which passage of the paper
each function follows and the readings taken where the paper is silent.

Parity status per function (what pins each one is listed in ``tests/test_oracle_pins.py``):
  fmix32, splitmix64 ........ pinned to published test vectors
  thresholds, live test ..... pinned to the exact-probability property of Eq. 5 and to boundary cases
  init ranks ................ pinned to clz on independently formed values
  simulate (registers) ...... pinned to brute-force breadth-first search per (vertex, simulation)
  reach / sigma ............. pinned to brute-force breadth-first search per simulation
  select_seeds .............. pinned to brute-force greedy on tiny graphs (always-rebuild, never-rebuild, mixed)
  estimate .................. pinned to Eq. 2 on hand-built sketches
  mt19937 ................... pinned to the value the C++ standard fixes (10000th output of the default seed) and
                              to numpy's independent implementation
  influence_mc .............. pinned to reachability closed forms (p = 0, p = 1), to a per-sample search over edges
                              drawn with numpy's generator, and to the expected reach of a star
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

IC, WC, PER_EDGE = 0, 1, 2

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_dbl = ctypes.c_double
_ptr = ctypes.c_void_p


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file to a shared library (plain gcc, -O2, no fused multiply-add contraction)."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile liboracle.so from oracle.c.  ORACLE_LIBRARY names another build to load instead: the mutation
    tests point it at an oracle with one planted mistake, to show that a pin catches it."""
    other = os.environ.get("ORACLE_LIBRARY")
    if other:
        return other
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        sig = {
            "or_fmix32": (_u32, [_u32]),
            "or_splitmix64": (_u64, [_u64, _u64]),
            "or_sim_words": (None, [_u64, _i32, _ptr, _ptr]),
            "or_edge_hash": (_u32, [_i64, _i64, _i64]),
            "or_edge_hash_dir": (_u32, [_i64, _i64, _i64, _i32]),
            "or_clz32": (_i32, [_u32]),
            "or_init_rank": (_i32, [_i64, _u32]),
            "or_threshold_from_p": (_i32, [_dbl, _ptr]),
            "or_is_live": (_i32, [_u32, _u32, _u32, _i32]),
            "or_edge_thresholds": (_i32, [_i64, _i64, _ptr, _ptr, _i32, _dbl, _ptr, _ptr, _ptr]),
            "or_init_registers": (None, [_i64, _i32, _ptr, _ptr, _ptr]),
            "or_simulate": (_i32, [_i64, _ptr, _ptr, _ptr, _ptr, _i32, _ptr, _ptr, _ptr, _dbl, _i64, _ptr, _ptr,
                                   _ptr, _i64, _i32]),
            "or_reach_add": (_i64, [_i64, _ptr, _ptr, _ptr, _ptr, _i32, _ptr, _i64, _ptr, _i32]),
            "or_estimate_from_sum": (_dbl, [_u64, _i32]),
            "or_build": (_i32, [_i64, _i64, _ptr, _ptr, _i32, _dbl, _ptr, _i32, _u64, _dbl, _ptr, _ptr, _ptr, _ptr,
                                _i64, _i32]),
            "or_select_seeds": (_i32, [_i64, _i64, _ptr, _ptr, _i32, _dbl, _ptr, _i32, _i32, _dbl, _dbl, _dbl, _u64,
                                       _ptr, _ptr, _ptr, _ptr, _ptr, _ptr, _ptr, _ptr, _i32, _i32]),
            "or_estimate_set": (_dbl, [_i64, _i32, _ptr, _ptr, _i32, _ptr]),
            "or_register_at": (_i32, [_i64, _ptr, _ptr, _ptr, _ptr, _ptr, _ptr, _i64, _i32, _ptr, _ptr, _i32]),
            "or_mt_outputs": (None, [_u32, _i64, _ptr]),
            "or_mc_stream_seed": (_u32, [_u64, _i64, _i64, _i64]),
            "or_mc_live": (_i32, [_i64, _ptr, _ptr, _u64, _i64, _ptr]),
            "or_influence_mc": (_i64, [_i64, _i64, _ptr, _ptr, _i32, _dbl, _ptr, _ptr, _i32, _i64, _i64, _u64, _ptr]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(xadj, adj):
    return np.ascontiguousarray(xadj, dtype=np.int64), np.ascontiguousarray(adj, dtype=np.int32)


def fmix32(x: int) -> int:
    return int(lib().or_fmix32(x))


def splitmix64(seed: int, i: int) -> int:
    return int(lib().or_splitmix64(seed, i))


def sim_words(seed: int, R: int) -> tuple[np.ndarray, np.ndarray]:
    X = np.zeros(R, np.uint32)
    Y = np.zeros(R, np.uint32)
    lib().or_sim_words(seed, R, _p(X), _p(Y))
    return X, Y


def edge_hash(u: int, v: int, n: int) -> int:
    return int(lib().or_edge_hash(u, v, n))


def edge_hash_dir(u: int, v: int, n: int, undirected: bool) -> int:
    """Reading R16: an undirected input's edge hashes by its ordered key, the same in both directions."""
    return int(lib().or_edge_hash_dir(u, v, n, 1 if undirected else 0))


def clz32(x: int) -> int:
    return int(lib().or_clz32(x))


def init_rank(v: int, y: int) -> int:
    return int(lib().or_init_rank(v, y))


def threshold_from_p(p: float) -> tuple[int, int]:
    t = np.zeros(1, np.uint32)
    ok = lib().or_threshold_from_p(p, _p(t))
    return int(ok), int(t[0])


def is_live(h: int, x: int, T: int, possible: int = 1) -> bool:
    return bool(lib().or_is_live(h, x, T, possible))


def edge_thresholds(n, xadj, adj, model, p=0.0, p_edge=None):
    xadj, adj = _csr(xadj, adj)
    m = adj.shape[0]
    T = np.zeros(max(m, 1), np.uint32)
    ok = np.zeros(max(m, 1), np.uint8)
    pe = None if p_edge is None else np.ascontiguousarray(p_edge, dtype=np.float32)
    rc = lib().or_edge_thresholds(n, m, _p(xadj), _p(adj), model, p, _p(pe), _p(T), _p(ok))
    if rc != 0:
        raise ValueError(f"or_edge_thresholds rc={rc}")
    return T[:m], ok[:m]


def init_registers(n, R, Y, blocked=None):
    M = np.zeros((n, R), np.uint8)
    Y = np.ascontiguousarray(Y, dtype=np.uint32)
    b = None if blocked is None else np.ascontiguousarray(blocked, dtype=np.uint8)
    lib().or_init_registers(n, R, _p(Y), _p(b), _p(M))
    return M


def simulate(n, xadj, adj, T, possible, R, X, M, blocked=None, eps_c=0.0, max_sweeps=0, log_cap=4096,
             undirected=False):
    """Runs Algorithm 2 in place on M; returns (sweeps, visits, frontier sizes at the start of each sweep)."""
    xadj, adj = _csr(xadj, adj)
    assert M.flags.c_contiguous and M.dtype == np.uint8
    T = np.ascontiguousarray(T, dtype=np.uint32)
    possible = np.ascontiguousarray(possible, dtype=np.uint8)
    X = np.ascontiguousarray(X, dtype=np.uint32)
    b = None if blocked is None else np.ascontiguousarray(blocked, dtype=np.uint8)
    sw = np.zeros(1, np.int64)
    vi = np.zeros(1, np.uint64)
    log = np.zeros(log_cap, np.int64)
    rc = lib().or_simulate(n, _p(xadj), _p(adj), _p(T), _p(possible), R, _p(X), _p(b), _p(M), eps_c, max_sweeps,
                           _p(sw), _p(vi), _p(log), log_cap, 1 if undirected else 0)
    if rc != 0:
        raise RuntimeError(f"or_simulate rc={rc}")
    s = int(sw[0])
    return s, int(vi[0]), log[: min(s, log_cap)].copy()


def reach_add(n, xadj, adj, T, possible, R, X, s, reached, undirected=False):
    xadj, adj = _csr(xadj, adj)
    T = np.ascontiguousarray(T, dtype=np.uint32)
    possible = np.ascontiguousarray(possible, dtype=np.uint8)
    X = np.ascontiguousarray(X, dtype=np.uint32)
    assert reached.flags.c_contiguous and reached.dtype == np.uint8
    r = lib().or_reach_add(n, _p(xadj), _p(adj), _p(T), _p(possible), R, _p(X), s, _p(reached),
                           1 if undirected else 0)
    if r < 0:
        raise MemoryError
    return int(r)


def estimate_from_sum(g: int, R: int) -> float:
    return float(lib().or_estimate_from_sum(g, R))


def build_sketch(n, xadj, adj, model, p, R, seed, p_edge=None, eps_c=0.0, log_cap=4096, undirected=False):
    """Registers after a fresh build; returns (M[n, R], sweeps, visits, frontier log)."""
    xadj, adj = _csr(xadj, adj)
    M = np.zeros((n, R), np.uint8)
    pe = None if p_edge is None else np.ascontiguousarray(p_edge, dtype=np.float32)
    sw = np.zeros(1, np.int64)
    vi = np.zeros(1, np.uint64)
    log = np.zeros(log_cap, np.int64)
    rc = lib().or_build(n, adj.shape[0], _p(xadj), _p(adj), model, p, _p(pe), R, seed, eps_c, _p(M), _p(sw), _p(vi),
                        _p(log), log_cap, 1 if undirected else 0)
    if rc != 0:
        raise RuntimeError(f"or_build rc={rc}")
    s = int(sw[0])
    return M, s, int(vi[0]), log[: min(s, log_cap)].copy()


def select_seeds(n, xadj, adj, model, p, R, K, eps_g, eps_l=0.3, eps_c=0.0, seed=1, p_edge=None, literal=False,
                 undirected=False):
    """Algorithm 1; returns a dict of per-step arrays and run totals.  literal: blocked registers as Algorithms 1 and
    2 print them (reading R17); undirected: reading R16."""
    xadj, adj = _csr(xadj, adj)
    pe = None if p_edge is None else np.ascontiguousarray(p_edge, dtype=np.float32)
    seeds = np.zeros(K, np.int32)
    sigma = np.zeros(K, np.float64)
    est = np.zeros(K, np.float64)
    gsum = np.zeros(K, np.uint64)
    rebuilt = np.zeros(K, np.uint8)
    vis = np.zeros(1, np.uint64)
    sw = np.zeros(1, np.int64)
    nb = np.zeros(1, np.int32)
    rc = lib().or_select_seeds(n, adj.shape[0], _p(xadj), _p(adj), model, p, _p(pe), R, K, eps_g, eps_l, eps_c, seed,
                               _p(seeds), _p(sigma), _p(est), _p(gsum), _p(rebuilt), _p(vis), _p(sw), _p(nb),
                               1 if literal else 0, 1 if undirected else 0)
    if rc != 0:
        raise RuntimeError(f"or_select_seeds rc={rc}")
    return dict(seeds=seeds, sigma=sigma, est=est, gsum=gsum, rebuilt=rebuilt, visits=int(vis[0]), sweeps=int(sw[0]),
                builds=int(nb[0]))


def estimate_set(M: np.ndarray, S) -> tuple[float, int]:
    M = np.ascontiguousarray(M, dtype=np.uint8)
    S = np.ascontiguousarray(S, dtype=np.int32)
    g = np.zeros(1, np.uint64)
    e = lib().or_estimate_set(M.shape[0], M.shape[1], _p(M), _p(S), S.shape[0], _p(g))
    return float(e), int(g[0])


class RegisterProbe:
    """Evaluates single registers M_v[j] by breadth-first search (for sampled checks on large graphs)."""

    def __init__(self, n, xadj, adj, model, p, R, seed, p_edge=None, undirected=False):
        self.n = n
        self.undirected = 1 if undirected else 0
        self.xadj, self.adj = _csr(xadj, adj)
        self.T, self.ok = edge_thresholds(n, self.xadj, self.adj, model, p=p, p_edge=p_edge)
        self.X, self.Y = sim_words(seed, R)
        self.seen = np.zeros(max(n, 1), np.uint8)
        self.queue = np.zeros(max(n, 1), np.int64)

    def __call__(self, v: int, j: int) -> int:
        return int(lib().or_register_at(self.n, _p(self.xadj), _p(self.adj), _p(self.T), _p(self.ok), _p(self.X),
                                        _p(self.Y), v, j, _p(self.seen), _p(self.queue), self.undirected))

    def reach_total(self, seeds) -> int:
        """|{(v, j): v reachable from the seed set in sample j}| summed over the R samples."""
        R = self.X.shape[0]
        reached = np.zeros((self.n, R), np.uint8)
        total = 0
        for s in seeds:
            total += reach_add(self.n, self.xadj, self.adj, self.T, self.ok, R, self.X, int(s), reached,
                               self.undirected)
        return total


MC_CHUNK = 8192  # edges per generator stream of the influence oracle (reading R15)


def mt_outputs(seed: int, count: int) -> np.ndarray:
    """The first `count` outputs of mt19937 seeded with init_genrand(seed)."""
    out = np.zeros(max(count, 1), np.uint32)
    lib().or_mt_outputs(seed & 0xFFFFFFFF, count, _p(out))
    return out[:count]


def mc_stream_seed(seed: int, s: int, c: int, nchunks: int) -> int:
    return int(lib().or_mc_stream_seed(seed, s, c, nchunks))


def mc_live(n, xadj, adj, model, p, seed, s, p_edge=None) -> np.ndarray:
    """Reading R15: the live edges (one byte per out-CSR edge) of sample s."""
    T, ok = edge_thresholds(n, xadj, adj, model, p, p_edge)
    m = T.shape[0]
    live = np.zeros(max(m, 1), np.uint8)
    lib().or_mc_live(m, _p(np.ascontiguousarray(T)), _p(np.ascontiguousarray(ok)), seed, s, _p(live))
    return live[:m]


def influence_mc(n, xadj, adj, model, p, seeds, N, seed, p_edge=None, first=0):
    """Sample-then-diffuse influence of `seeds` over samples first .. first + N - 1 (Section 4's oracle, reading
    R15).  Returns (total reached over those samples, per-sample reach counts)."""
    xadj, adj = _csr(xadj, adj)
    S = np.ascontiguousarray(seeds, dtype=np.int32)
    pe = None if p_edge is None else np.ascontiguousarray(p_edge, dtype=np.float32)
    reach = np.zeros(max(N, 1), np.int64)
    t = lib().or_influence_mc(n, adj.shape[0], _p(xadj), _p(adj), model, p, _p(pe), _p(S), S.shape[0], first, N,
                              seed, _p(reach))
    if t < 0:
        raise RuntimeError(f"or_influence_mc rc={-t}")
    return int(t), reach[:N].copy()
