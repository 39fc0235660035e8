"""Shared helpers of the GPU tests: the library context and oracle comparisons."""
from __future__ import annotations

import numpy as np

import oracle

import paper_2105_04023_gb300 as im


def oracle_build(g, model, p, R, seed, p_edge=None, eps_c=0.0, undirected=False):
    return oracle.build_sketch(g.n, g.xadj, g.adj, model, p, R, seed, p_edge=p_edge, eps_c=eps_c,
                               undirected=undirected)


def gpu_build(ctx, g, model, p, R, seed, p_edge=None, eps_c=0.0, device=None, undirected=False):
    graph = im.Graph.from_synth(g, model, p, p_edge=p_edge, device=device, undirected=undirected)
    sk = ctx.im_build_sketches(graph, im.params(R=R, seed=seed, eps_c=eps_c))
    M = sk.im_sketch_registers()
    sweeps, visits, log = sk.im_sketch_info()
    return sk, M, sweeps, visits, log


def assert_build_parity(ctx, g, model, p, R, seed, p_edge=None, eps_c=0.0, device=None, undirected=False):
    Mo, so, vo, lo = oracle_build(g, model, p, R, seed, p_edge=p_edge, eps_c=eps_c, undirected=undirected)
    sk, Mg, sg, vg, lg = gpu_build(ctx, g, model, p, R, seed, p_edge=p_edge, eps_c=eps_c, device=device,
                                   undirected=undirected)
    if not np.array_equal(Mo, Mg):
        bad = np.argwhere(Mo != Mg)
        raise AssertionError(f"{len(bad)} registers differ, first (v, j) = {bad[:5].tolist()}: oracle "
                             f"{[int(Mo[tuple(b)]) for b in bad[:5]]} gpu {[int(Mg[tuple(b)]) for b in bad[:5]]}")
    assert sg == so, (sg, so)
    assert vg == vo, (vg, vo)
    assert np.array_equal(lg, lo), (lg, lo)
    return sk, Mo


def assert_select_parity(ctx, g, model, p, R, K, eps_g, eps_l=0.3, eps_c=0.0, seed=1, p_edge=None, device=None,
                         literal=False, undirected=False):
    ref = oracle.select_seeds(g.n, g.xadj, g.adj, model, p, R, K, eps_g, eps_l, eps_c, seed, p_edge=p_edge,
                              literal=literal, undirected=undirected)
    graph = im.Graph.from_synth(g, model, p, p_edge=p_edge, device=device, undirected=undirected)
    blocking = im.IM_BLOCK_LITERAL if literal else im.IM_BLOCK_RESIDUAL
    out = ctx.im_select_seeds(graph, im.params(R=R, K=K, eps_g=eps_g, eps_l=eps_l, eps_c=eps_c, seed=seed,
                                               blocking=blocking))
    assert out["seeds"].tolist() == ref["seeds"].tolist(), (out["seeds"], ref["seeds"])
    assert out["gsum"].tolist() == ref["gsum"].tolist()
    assert out["rebuilt"].tolist() == ref["rebuilt"].tolist()
    # sigma = reached / R and e = 2^(g/R) / phi are formed the same way on both sides from equal integers
    assert np.array_equal(out["sigma"], ref["sigma"])
    np.testing.assert_allclose(out["estimate"], ref["est"], rtol=1e-12)
    st = ctx.stats()
    assert st["visits"] == ref["visits"], (st["visits"], ref["visits"])
    assert st["sweeps"] == ref["sweeps"], (st["sweeps"], ref["sweeps"])
    assert st["builds"] == ref["builds"]
    return out, ref
