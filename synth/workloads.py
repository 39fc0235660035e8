"""The five synthetic workloads: graph recipe plus the influence-maximisation parameters they are run with.

The paper measures on SNAP / MixGreedy graphs (Table 1 of Section 4) that are not available here; these seeded
graphs stand in for them with the same shapes (directed, power-law or uniform degree, mean degree 10-16).
Only inputs are described here: model name, probability, R, K and thresholds are passed to whichever
implementation runs them.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import graphs

IC = 0  # independent cascade, one constant probability p on every edge
WC = 1  # weighted cascade, p(u, v) = 1 / indeg(v)
PER_EDGE = 2  # one probability per edge


@dataclasses.dataclass
class Problem:
    graph: graphs.Graph
    model: int
    p: float
    R: int
    K: int
    eps_g: float
    eps_l: float = 0.3
    eps_c: float = 0.0
    seed: int = 1
    p_edge: np.ndarray | None = None
    name: str = ""


def er_2k() -> Problem:
    """Directed Erdos-Renyi n=2000, m=20000, IC p=0.05, R=64, K=10, eps_g=0.01."""
    g = graphs.erdos_renyi(2000, 20000, seed=1)
    return Problem(g, IC, 0.05, R=64, K=10, eps_g=0.01, seed=1, name="er_n2000_m20000_ic0.05_R64_K10")


def rmat20_wc(cache: bool = False) -> Problem:
    """R-MAT scale 20, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), weighted cascade, R=256, K=50, eps_g=0.01."""
    g = (graphs.cached(lambda: graphs.rmat(20, 16, seed=2), "rmat_s20_ef16_seed2") if cache
         else graphs.rmat(20, 16, seed=2))
    return Problem(g, WC, 0.0, R=256, K=50, eps_g=0.01, seed=2, name="rmat_s20_ef16_wc_R256_K50")


def chunglu22_ic(cache: bool = False) -> Problem:
    """Directed Chung-Lu n=2^22, mean degree 16, exponent 2.1, IC p=0.01, R=512, K=100, eps_g=0.02."""
    g = (graphs.cached(lambda: graphs.chung_lu(1 << 22, 16.0, 2.1, seed=3), "chunglu_n22_d16_g2.1_seed3") if cache
         else graphs.chung_lu(1 << 22, 16.0, 2.1, seed=3))
    return Problem(g, IC, 0.01, R=512, K=100, eps_g=0.02, seed=3, name="chunglu_n4M_d16_ic0.01_R512_K100")


def chunglu20_ic(cache: bool = False) -> Problem:
    """The Chung-Lu recipe at n=2^20 (mean degree 16, exponent 2.1, IC p=0.01, R=512): the profiling case of the
    n=2^22 workload, small enough for multi-pass profiler captures."""
    g = (graphs.cached(lambda: graphs.chung_lu(1 << 20, 16.0, 2.1, seed=3), "chunglu_n20_d16_g2.1_seed3") if cache
         else graphs.chung_lu(1 << 20, 16.0, 2.1, seed=3))
    return Problem(g, IC, 0.01, R=512, K=100, eps_g=0.02, seed=3, name="chunglu_n1M_d16_ic0.01_R512_K100")


_BATCH_MODELS = ((IC, 0.005), (IC, 0.01), (IC, 0.05), (WC, 0.0))
_BATCH_R = (64, 128, 256)


def batch_spec(i: int) -> tuple[int, int, int, float, int]:
    """(scale, edge_factor, model, p, R) of graph i of the 256-graph batch, drawn from its own stream."""
    x = np.random.PCG64([1000 + i, 1]).random_raw(4).astype(np.uint64)
    scale = 10 + int(x[0] % np.uint64(9))
    ef = 8 + int(x[1] % np.uint64(9))
    model, p = _BATCH_MODELS[int(x[2] % np.uint64(4))]
    R = _BATCH_R[int(x[3] % np.uint64(3))]
    return scale, ef, model, p, R


def batch_problem(i: int, max_scale: int | None = None) -> Problem:
    """Graph i of the batched workload: R-MAT with its own scale, edge factor, model and R; K=20, eps_g=0.01."""
    scale, ef, model, p, R = batch_spec(i)
    if max_scale is not None:
        scale = min(scale, max_scale)
    g = graphs.rmat(scale, ef, seed=1000 + i)
    return Problem(g, model, p, R=R, K=20, eps_g=0.01, seed=1000 + i, name=f"batch{i}_s{scale}_ef{ef}")


def batch(count: int = 256, max_scale: int | None = None) -> list[Problem]:
    return [batch_problem(i, max_scale) for i in range(count)]


def serve_pool_graph(i: int, max_scale: int | None = None) -> graphs.Graph:
    """Graph i of the 64-graph serving pool: R-MAT scale 12 + (i mod 9), edge factor 16."""
    scale = 12 + (i % 9)
    if max_scale is not None:
        scale = min(scale, max_scale)
    return graphs.rmat(scale, 16, seed=2000 + i)


def serve_queries(count: int = 10000, pool: int = 64, seed: int = 5) -> np.ndarray:
    """Query stream: columns (graph id, K, R, unit-rate exponential inter-arrival gap)."""
    rng = np.random.PCG64(seed)
    x = rng.random_raw(4 * count).astype(np.uint64).reshape(count, 4)
    gid = (x[:, 0] % np.uint64(pool)).astype(np.float64)
    K = (5 + x[:, 1] % np.uint64(96)).astype(np.float64)
    R = np.where((x[:, 2] & np.uint64(1)) == 0, 64.0, 256.0)
    u = ((x[:, 3] >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)
    gap = -np.log(u)
    return np.stack([gid, K, R, gap], axis=1)
