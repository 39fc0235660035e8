"""Influence scorer (Section 4's sample-then-diffuse oracle with mt19937, reading R15): the CUDA path against the
CPU oracle, per sample and bit-exact (reach counts are integers)."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

import oracle
from synth import graphs, workloads

import paper_2105_04023_gb300 as im

pytestmark = pytest.mark.gpu

IC, WC, PER_EDGE = 0, 1, 2
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctx():
    from paper_2105_04023_gb300 import build

    build.build()
    c = im.Context(0)
    yield c
    c.close()


def _check(ctx, g, model, p, seeds, N, seed, p_edge=None, device="cuda"):
    total, ref = oracle.influence_mc(g.n, g.xadj, g.adj, model, p, seeds, N, seed, p_edge=p_edge)
    sigma, reach = ctx.im_influence_mc(im.Graph.from_synth(g, model, p, p_edge=p_edge, device=device), seeds, N, seed)
    assert reach.tolist() == ref.tolist(), (model, N, np.flatnonzero(reach != ref)[:8])
    assert sigma == total / N  # both sides divide the same integers


@pytest.mark.parametrize("N", [64, 192, 512, 1024, 1088])
@pytest.mark.parametrize("model,p", [(IC, 0.12), (WC, 0.0)])
def test_mc_matches_oracle_per_sample(ctx, N, model, p):
    # three generator streams per sample; 192 runs as one 256-sample batch with 64 unused columns, 512 with 16-edge
    # search tasks, 1088 as a full 1024-sample batch plus a 64-sample one
    g = graphs.erdos_renyi(3000, 21000, seed=41)
    _check(ctx, g, model, p, [7, 100, 7, 2999], N, seed=99)


def test_mc_per_edge_model_and_rmat(ctx):
    g = graphs.rmat(12, 8, seed=17)
    pe = np.random.default_rng(3).uniform(0.0, 0.4, g.adj.shape[0]).astype(np.float32)
    pe[::7] = 0.0
    _check(ctx, g, PER_EDGE, 0.0, [0, 1, 2, 3, 4], 256, seed=5, p_edge=pe)


def test_mc_host_memory_graph(ctx):
    g = graphs.star_hub(5000, seed=8)
    _check(ctx, g, IC, 0.3, [0], 128, seed=12, device=None)


def test_mc_degenerate_graphs(ctx):
    empty = graphs.csr_from_edges(10, np.zeros(0, np.int64), np.zeros(0, np.int64))
    sigma, reach = ctx.im_influence_mc(im.Graph.from_synth(empty, IC, 0.5, device="cuda"), [1, 1, 4], 64, 1)
    assert (reach == 2).all() and sigma == 2.0
    g = graphs.chain(300)
    _check(ctx, g, IC, 1.0, [0], 64, seed=2)  # every edge live: the whole chain, 299 levels
    _check(ctx, g, IC, 0.0, list(range(300)), 64, seed=2)  # every vertex a seed


@pytest.mark.parametrize("case", ["nsamples", "seed_range", "k"])
def test_mc_invalid_arguments(ctx, case):
    g = im.Graph.from_synth(graphs.chain(20), IC, 0.5, device="cuda")
    with pytest.raises(im.ImError) as ei:
        if case == "nsamples":
            ctx.im_influence_mc(g, [0], 100, 1)
        elif case == "seed_range":
            ctx.im_influence_mc(g, [20], 64, 1)
        else:
            ctx.im_influence_mc(g, [], 64, 1)
    assert ei.value.status == im._lib.IM_EINVAL


def test_mc_rmat20_sampled(ctx):
    # the bench workload: 1024 samples of the R-MAT scale-20 WC graph from the first 10 seeds the select picks; the
    # oracle evaluates three of the samples one at a time
    with open(os.path.join(HERE, "golden", "rmat20_wc.json")) as f:
        seeds = json.load(f)["select"]["seeds"][:10]
    prob = workloads.rmat20_wc(cache=True)
    g = prob.graph
    sigma, reach = ctx.im_influence_mc(im.Graph.from_synth(g, prob.model, prob.p, device="cuda"), seeds, 1024, 77)
    assert sigma == reach.sum() / 1024
    for s in (0, 511, 1023):
        _, ref = oracle.influence_mc(g.n, g.xadj, g.adj, prob.model, prob.p, seeds, 1, 77, first=s)
        assert int(reach[s]) == int(ref[0]), s
