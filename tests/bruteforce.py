"""Brute-force references used to pin the oracle: explicit per-simulation breadth-first searches.

These use only the oracle's pinned primitives (edge hash, thresholds, live test, initial rank), never its diffusion,
reach or greedy code, so a mistake in Algorithm 1 or 2 as the oracle restates them shows up as a mismatch here.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def live_matrix(orc, n, xadj, adj, T, possible, X, undirected=False):
    """live[e, j] for every edge e and simulation j, from the oracle's pinned live test.  undirected: both directions
    of an edge take the hash of the key (min, max)."""
    m = adj.shape[0]
    R = X.shape[0]
    src = np.repeat(np.arange(n), np.diff(xadj))
    L = np.zeros((m, R), dtype=bool)
    for e in range(m):
        a, b = int(src[e]), int(adj[e])
        if undirected and b < a:
            a, b = b, a
        h = orc.edge_hash(a, b, n)
        for j in range(R):
            L[e, j] = orc.is_live(h, int(X[j]), int(T[e]), int(possible[e]))
    return L


def reach_set(n, xadj, adj, live, j, start, blocked=None, enter_blocked=False):
    """Vertices reachable from `start` over edges live in simulation j, never entering blocked (v, j); with
    enter_blocked a blocked vertex is entered but not left (a path ends there)."""
    seen = {start}
    q = deque([start])
    while q:
        u = q.popleft()
        if blocked is not None and blocked[u, j] and u != start:
            continue
        for e in range(xadj[u], xadj[u + 1]):
            v = int(adj[e])
            if v in seen or not live[e, j]:
                continue
            if blocked is not None and blocked[v, j] and not enter_blocked:
                continue
            seen.add(v)
            q.append(v)
    return seen


def registers(orc, n, xadj, adj, live, Y, blocked=None, literal=False):
    """M[v, j] = max initial rank over the reach set of v in sample j.  Residual blocking: blocked registers are 0
    and blocked vertices are not entered.  Literal blocking (Algorithms 1 and 2 as printed): a blocked register keeps
    its initial rank, and an unblocked v takes the max over the vertices it reaches by paths on which only the last
    vertex may be blocked."""
    R = Y.shape[0]
    M = np.zeros((n, R), np.uint8)
    rank = np.array([[orc.init_rank(v, int(Y[j])) for j in range(R)] for v in range(n)], dtype=np.int64)
    for v in range(n):
        for j in range(R):
            if blocked is not None and blocked[v, j]:
                M[v, j] = rank[v, j] if literal else 0
                continue
            M[v, j] = max(rank[x, j] for x in reach_set(n, xadj, adj, live, j, v, blocked, enter_blocked=literal))
    return M


def reached_by(n, xadj, adj, live, S, R):
    """reached[v, j] = 1 iff v is reachable from the set S in simulation j."""
    out = np.zeros((n, R), np.uint8)
    for j in range(R):
        for s in S:
            for v in reach_set(n, xadj, adj, live, j, int(s)):
                out[v, j] = 1
    return out


def greedy(orc, n, xadj, adj, live, Y, K, eps_g, eps_l, literal=False):
    """Algorithm 1 with every sketch formed by brute force (no diffusion), sigma by brute-force reach sets."""
    R = Y.shape[0]
    M = registers(orc, n, xadj, adj, live, Y)
    MS = np.zeros(R, np.int64)
    S: list[int] = []
    varsigma = 0.0
    out = dict(seeds=[], sigma=[], est=[], gsum=[], rebuilt=[])
    for k in range(K):
        best, best_g = -1, -1
        for v in range(n):
            if v in S:
                continue
            g = int(np.maximum(M[v].astype(np.int64), MS).sum())
            if g > best_g:
                best, best_g = v, g
        S.append(best)
        e = orc.estimate_from_sum(best_g, R)
        reached = reached_by(n, xadj, adj, live, S, R)
        sigma = float(reached.sum()) / R
        delta = sigma - varsigma
        err_l = float("inf") if delta == 0.0 else abs((e - delta) / delta)
        err_g = abs((e - delta) / sigma)
        out["seeds"].append(best)
        out["sigma"].append(sigma)
        out["est"].append(e)
        out["gsum"].append(best_g)
        if err_l < eps_l or err_g < eps_g:
            MS = np.maximum(MS, M[best].astype(np.int64))
            out["rebuilt"].append(0)
        else:
            out["rebuilt"].append(1)
            M = registers(orc, n, xadj, adj, live, Y, blocked=reached.astype(bool), literal=literal)
            MS = np.zeros(R, np.int64)
            varsigma = sigma
    return out
