"""Seeded synthetic directed graphs shaped like the social networks of the paper's Table 1.

This module produces INPUTS only.  It holds none of the influence-maximisation arithmetic (no edge hashing, no
sampling thresholds, no sketch registers): both the CPU oracle and the CUDA library consume the CSR arrays it returns
and derive everything else themselves.

Randomness comes from numpy's PCG64 bit generator through ``random_raw`` only, whose output stream is fixed by the
seed on every platform and numpy version; uniform doubles are formed as ``(x >> 11) * 2**-53``.

Every graph is returned in the layout of the paper's Section 3.3: an out-neighbour CSR ``xadj`` (int64, n+1) and
``adj`` (int32, m), rows sorted by target id, with self-loops removed and parallel edges merged (Section 2.1 says
parallel edges are merged in preprocessing).
"""
from __future__ import annotations

import dataclasses

import numpy as np

_INV53 = 1.0 / float(1 << 53)


def _raw(rng: np.random.PCG64, count: int) -> np.ndarray:
    return rng.random_raw(int(count)).astype(np.uint64, copy=False)


def _uniform(rng: np.random.PCG64, count: int) -> np.ndarray:
    return (_raw(rng, count) >> np.uint64(11)).astype(np.float64) * _INV53


def _below(rng: np.random.PCG64, count: int, bound: int) -> np.ndarray:
    """Integers in [0, bound) by multiply-shift of the high 32 bits (bias < 2**-32 for bound < 2**32)."""
    hi = _raw(rng, count) >> np.uint64(32)
    return ((hi * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)


@dataclasses.dataclass
class Graph:
    """Directed graph in out-neighbour CSR form."""

    n: int
    xadj: np.ndarray  # int64[n+1]
    adj: np.ndarray  # int32[m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.adj.shape[0])

    def edges(self) -> tuple[np.ndarray, np.ndarray]:
        src = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.xadj))
        return src, self.adj.astype(np.int64)


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, name: str = "") -> Graph:
    """Drop self-loops, merge parallel edges and build a row-sorted out-CSR."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    key = np.sort(src[keep] * np.int64(n) + dst[keep])  # sorted by (src, dst)
    if key.size:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    u = key // n
    v = key - u * n
    xadj = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(u, minlength=n), out=xadj[1:])
    return Graph(n=n, xadj=xadj, adj=v.astype(np.int32), name=name)


def erdos_renyi(n: int, m: int, seed: int) -> Graph:
    """Directed G(n, m): the first m distinct non-loop pairs of a uniform stream of (u, v) draws."""
    rng = np.random.PCG64(seed)
    if m > n * (n - 1):
        raise ValueError("more edges than ordered non-loop pairs")
    seen: dict[int, None] = {}
    while len(seen) < m:
        batch = 2 * (m - len(seen)) + 64
        u = _below(rng, batch, n)
        v = _below(rng, batch, n)
        for a, b in zip(u.tolist(), v.tolist()):
            if a != b:
                seen.setdefault(a * n + b, None)
                if len(seen) == m:
                    break
    key = np.fromiter(seen.keys(), dtype=np.int64, count=m)
    return csr_from_edges(n, key // n, key % n, name=f"er_n{n}_m{m}_s{seed}")


def rmat(scale: int, edge_factor: int, seed: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         relabel: bool = True) -> Graph:
    """R-MAT (Chakrabarti et al.) without noise, then a seeded relabelling of the vertex ids (Graph500 style)."""
    n = 1 << scale
    draws = edge_factor * n
    rng = np.random.PCG64(seed)
    src = np.zeros(draws, dtype=np.int64)
    dst = np.zeros(draws, dtype=np.int64)
    # quadrant thresholds on the 53-bit integer form of the uniform draw (exact: the thresholds are compared
    # against the same integers a uniform double would be built from)
    th_a = np.uint64(int(a * (1 << 53)))
    th_ab = np.uint64(int((a + b) * (1 << 53)))
    th_abc = np.uint64(int((a + b + c) * (1 << 53)))
    for _ in range(scale):
        y = _raw(rng, draws) >> np.uint64(11)
        row = y >= th_ab  # quadrant c or d: lower half of rows
        col = ((y >= th_a) & (y < th_ab)) | (y >= th_abc)  # quadrant b or d: right half of columns
        src <<= 1
        dst <<= 1
        src |= row
        dst |= col
    if relabel:
        perm = np.argsort(_raw(rng, n), kind="stable").astype(np.int64)
        src = perm[src]
        dst = perm[dst]
    return csr_from_edges(n, src, dst, name=f"rmat_s{scale}_ef{edge_factor}_seed{seed}")


def chung_lu(n: int, mean_degree: float, gamma: float, seed: int) -> Graph:
    """Directed Chung-Lu graph: source drawn with probability proportional to its out-weight, target to its
    in-weight, weights w_i = (i+1)^(-1/(gamma-1)); the in-weights are an independent permutation of the same list."""
    rng = np.random.PCG64(seed)
    w = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (gamma - 1.0))
    cdf_out = np.cumsum(w)
    cdf_out /= cdf_out[-1]
    perm_in = np.argsort(_raw(rng, n), kind="stable")
    cdf_in = np.cumsum(w[perm_in])
    cdf_in /= cdf_in[-1]
    draws = int(round(mean_degree * n))
    src = np.empty(draws, dtype=np.int64)
    dst = np.empty(draws, dtype=np.int64)
    chunk = 1 << 24
    for lo in range(0, draws, chunk):
        hi = min(draws, lo + chunk)
        src[lo:hi] = np.minimum(np.searchsorted(cdf_out, _uniform(rng, hi - lo), side="right"), n - 1)
        dst[lo:hi] = np.minimum(np.searchsorted(cdf_in, _uniform(rng, hi - lo), side="right"), n - 1)
    return csr_from_edges(n, src, dst, name=f"chunglu_n{n}_d{mean_degree}_g{gamma}_s{seed}")


def symmetrized(g: Graph) -> Graph:
    """The undirected graph of g stored with both directions of every edge (rows sorted, repeats merged)."""
    src, dst = g.edges()
    return csr_from_edges(g.n, np.concatenate([src, dst]), np.concatenate([dst, src]), name=g.name + "_sym")


def chain(n: int) -> Graph:
    """Directed path 0 -> 1 -> ... -> n-1."""
    return csr_from_edges(n, np.arange(n - 1), np.arange(1, n), name=f"chain{n}")


def random_small(n: int, m: int, seed: int) -> Graph:
    """Small uniform multigraph draw (loops and duplicates removed afterwards) for brute-force tests."""
    rng = np.random.PCG64(seed)
    return csr_from_edges(n, _below(rng, m, n), _below(rng, m, n), name=f"small_n{n}_m{m}_s{seed}")


def star_hub(n_leaves: int, seed: int) -> Graph:
    """One hub with out-edges to every leaf plus a sparse random layer among the leaves (a long ragged row)."""
    rng = np.random.PCG64(seed)
    n = n_leaves + 1
    src = np.concatenate([np.zeros(n_leaves, dtype=np.int64), 1 + _below(rng, 2 * n_leaves, n_leaves)])
    dst = np.concatenate([np.arange(1, n, dtype=np.int64), 1 + _below(rng, 2 * n_leaves, n_leaves)])
    return csr_from_edges(n, src, dst, name=f"hub{n_leaves}_s{seed}")


def cached(builder, key: str, cache_dir: str | None = None) -> Graph:
    """Build a graph once and keep it as .npz under ``cache_dir`` (default: ``_build/graphs`` beside this package);
    the file holds exactly what ``builder()`` returned, so a hit and a miss give identical arrays."""
    import os

    if cache_dir is None:
        cache_dir = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build", "graphs")
    path = os.path.join(cache_dir, key + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        return Graph(n=int(z["n"]), xadj=z["xadj"], adj=z["adj"], name=str(z["name"]))
    g = builder()
    os.makedirs(cache_dir, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, n=np.int64(g.n), xadj=g.xadj, adj=g.adj, name=np.str_(g.name))
    os.replace(tmp, path)
    return g
