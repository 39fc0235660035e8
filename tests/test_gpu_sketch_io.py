"""Sketch export / import and selections that start from a built sketch (one build serving later runs with the same
graph, R, seed, eps_c and sweep limit): the exported registers are the oracle's, an imported sketch answers like the
original, and a selection from either equals a plain im_select_seeds and the oracle's Algorithm 1."""
from __future__ import annotations

import struct

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


@pytest.mark.parametrize("model,p,R,device", [(WC, 0.0, 256, None), (IC, 0.05, 128, "cuda"), (IC, 0.02, 512, None)])
def test_export_import_roundtrip(ctx, model, p, R, device):
    g = graphs.rmat(12, 12, seed=71)
    graph = im.Graph.from_synth(g, model, p, device=device)
    sk = ctx.im_build_sketches(graph, im.params(R=R, seed=17))
    data = sk.im_sketch_export()
    magic, n, m, R_h = struct.unpack_from("<Qqqi", data, 0)
    assert (magic, n, m, R_h) == (0x314354454B534D49, g.n, g.m, R)
    assert len(data) == struct.calcsize("<QqqiidQdqqQQii") + 8 * R + g.n * R
    M0, sweeps, visits, _ = oracle.build_sketch(g.n, g.xadj, g.adj, model, p, R, 17)
    regs = np.frombuffer(data[-g.n * R:], np.uint8).reshape(g.n, R)
    assert np.array_equal(regs, M0)
    X, Y = oracle.sim_words(17, R)
    off = len(data) - g.n * R - 8 * R
    assert np.array_equal(np.frombuffer(data[off:off + 4 * R], np.uint32), X)
    assert np.array_equal(np.frombuffer(data[off + 4 * R:off + 8 * R], np.uint32), Y)
    sk2 = ctx.im_sketch_import(graph, data)
    assert np.array_equal(sk2.im_sketch_registers(), M0)
    assert sk2.im_sketch_info()[:2] == (sweeps, visits)
    S = [3, 77, 1000]
    assert sk2.im_estimate(S, exact=True) == sk.im_estimate(S, exact=True)
    sk.close()
    sk2.close()


@pytest.mark.parametrize("literal", [False, True])
def test_select_from_sketch_equals_select(ctx, literal):
    g = graphs.rmat(12, 12, seed=72)
    graph = im.Graph.from_synth(g, WC)
    blocking = im.IM_BLOCK_LITERAL if literal else im.IM_BLOCK_RESIDUAL
    prm = im.params(R=128, K=10, eps_g=0.01, seed=5, blocking=blocking)
    sk = ctx.im_build_sketches(graph, im.params(R=128, seed=5))
    plain = ctx.im_select_seeds(graph, prm)
    from_sk = ctx.im_select_seeds_from(sk, prm)
    sk2 = ctx.im_sketch_import(graph, sk.im_sketch_export())
    from_imp = ctx.im_select_seeds_from(sk2, prm)
    ref = oracle.select_seeds(g.n, g.xadj, g.adj, WC, 0.0, 128, 10, 0.01, 0.3, 0.0, 5, literal=literal)
    for out in (from_sk, from_imp):
        for k in ("seeds", "gsum", "rebuilt", "sigma"):
            assert out[k].tolist() == plain[k].tolist(), k
    assert plain["seeds"].tolist() == ref["seeds"].tolist()
    assert plain["sigma"].tolist() == ref["sigma"].tolist()
    # the sketch is left as it was: a second selection from it gives the same
    again = ctx.im_select_seeds_from(sk, prm)
    assert again["seeds"].tolist() == plain["seeds"].tolist()
    sk.close()
    sk2.close()


def test_import_refuses_other_graphs_and_bad_bytes(ctx):
    g = graphs.rmat(11, 8, seed=73)
    h = graphs.rmat(11, 8, seed=74)  # same n, different edges
    sk = ctx.im_build_sketches(im.Graph.from_synth(g, WC), im.params(R=64, seed=1))
    data = sk.im_sketch_export()
    with pytest.raises(im.ImError):
        ctx.im_sketch_import(im.Graph.from_synth(h, WC), data)
    with pytest.raises(im.ImError):
        ctx.im_sketch_import(im.Graph.from_synth(g, IC, 0.1), data)  # another model
    with pytest.raises(im.ImError):
        ctx.im_sketch_import(im.Graph.from_synth(g, WC), data[:-1])  # truncated
    bad = bytearray(data)
    bad[0] ^= 1
    with pytest.raises(im.ImError):
        ctx.im_sketch_import(im.Graph.from_synth(g, WC), bytes(bad))
    with pytest.raises(im.ImError):  # the sketch's R and seed are fixed
        ctx.im_select_seeds_from(sk, im.params(R=64, K=3, seed=2))
    sk.close()
