"""The synthetic inputs are stable: the bench workload regenerates to the graph the golden file was computed on
(numpy PCG64 raw draws only, so the same arrays on every platform)."""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from synth import graphs, workloads

HERE = os.path.dirname(os.path.abspath(__file__))

# SHA-256 over the int64 xadj then the int32 adj of the R-MAT scale-20 workload as generated when the golden file
# was written
RMAT20_CSR_SHA256 = "983f23171976e4c8737563b7e2227fe03fd1a7bd2336e65b9f0237b52b1d5c03"


def test_rmat20_workload_is_the_golden_graph():
    with open(os.path.join(HERE, "golden", "rmat20_wc.json")) as f:
        gold = json.load(f)
    p = workloads.rmat20_wc(cache=False)
    g = p.graph
    assert (g.n, g.m, p.R, p.K, p.seed) == (gold["n"], gold["m"], gold["R"], gold["K"], gold["seed"])
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.xadj, np.int64).tobytes())
    h.update(np.ascontiguousarray(g.adj, np.int32).tobytes())
    assert h.hexdigest() == RMAT20_CSR_SHA256


def test_small_workloads_and_graph_invariants():
    w = workloads.er_2k()
    assert (w.graph.n, w.graph.m) == (2000, 20000)  # distinct non-loop pairs drawn to exactly m
    for g in (graphs.rmat(10, 8, seed=4), graphs.star_hub(300, seed=5), graphs.random_small(97, 700, seed=6)):
        assert g.xadj[0] == 0 and g.xadj[-1] == g.m and np.all(np.diff(g.xadj) >= 0)
        src = np.repeat(np.arange(g.n), np.diff(g.xadj))
        assert np.all(src != g.adj)  # no self-loops
        keys = src.astype(np.int64) * g.n + g.adj
        assert np.unique(keys).size == g.m  # no parallel edges
        for u in range(g.n):  # rows sorted by target
            row = g.adj[g.xadj[u]:g.xadj[u + 1]]
            assert np.all(np.diff(row) > 0)
