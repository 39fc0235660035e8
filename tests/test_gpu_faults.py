"""Failure detection on the device: a bounded wait that runs out ends the call with IM_ECUDA, names the wait, and
leaves the device usable.

Every spin-wait in the kernels has an iteration limit after which the kernel raises a fault bit in the problem's
counters and returns; the host reads the bits after each engine tick.  These tests lower two limits for one
context (environment variables read when a context is created, for tests only) so that a wait runs out with no
fault, trap or hang of the GPU:
  IM_TEST_CAS_LIMIT=0      the compare-and-swap byte max of a push sweep gives up at once (fault bit 2);
  IM_TEST_BARRIER_LIMIT=0  the grid barrier of the persistent search gives up at its first poll (fault bit 4).
A second context on the same device then runs a selection that matches the oracle.
"""
from __future__ import annotations

import pytest

import oracle
from synth import graphs

import paper_2105_04023_gb300 as im

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2105_04023_gb300 import build

    build.build()


def _context_with(monkeypatch, **env):
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    try:
        return im.Context(0)
    finally:
        for k in env:
            monkeypatch.delenv(k)


def _clean_select_matches_oracle(g):
    ctx = im.Context(0)
    try:
        out = ctx.im_select_seeds(im.Graph.from_synth(g, im.IM_WC), im.params(R=128, K=4, eps_g=0.01, seed=3))
        ref = oracle.select_seeds(g.n, g.xadj, g.adj, oracle.WC, 0.0, 128, 4, 0.01, 0.3, 0.0, 3)
        assert out["seeds"].tolist() == ref["seeds"].tolist()
        assert out["sigma"].tolist() == ref["sigma"].tolist()
    finally:
        ctx.close()


def test_register_update_limit_reports_fault(monkeypatch):
    g = graphs.rmat(10, 8, seed=4)
    ctx = _context_with(monkeypatch, IM_TEST_CAS_LIMIT="0")
    try:
        with pytest.raises(im.ImError) as err:
            ctx.im_build_sketches(im.Graph.from_synth(g, im.IM_WC), im.params(R=128, seed=3))
        assert err.value.status == 3  # IM_ECUDA
        assert "register update" in str(err.value)
        # the same context still runs calls that do not push (a search-only influence score)
        sig, reach = ctx.im_influence_mc(im.Graph.from_synth(g, im.IM_WC), [0, 1], 64, 5)
        tot, ref = oracle.influence_mc(g.n, g.xadj, g.adj, oracle.WC, 0.0, [0, 1], 64, 5)
        assert reach.tolist() == ref.tolist()
    finally:
        ctx.close()
    _clean_select_matches_oracle(g)


def test_grid_barrier_limit_reports_fault(monkeypatch):
    g = graphs.rmat(10, 8, seed=4)
    ctx = _context_with(monkeypatch, IM_PERSISTENT="1", IM_TEST_BARRIER_LIMIT="0")
    try:
        with pytest.raises(im.ImError) as err:
            ctx.im_select_seeds(im.Graph.from_synth(g, im.IM_WC), im.params(R=128, K=3, eps_g=0.01, seed=3))
        assert err.value.status == 3
        assert "grid barrier" in str(err.value)
    finally:
        ctx.close()
    _clean_select_matches_oracle(g)
