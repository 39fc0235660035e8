"""The allocation-free estimate (im_estimate_static) gives what im_estimate gives, call after call.

Some callers cannot allocate device memory while they serve a request: a serving thread on a latency budget
(cudaMalloc can synchronise the device and serialises on a process-wide lock), or a host process that accounts
for every device byte through its own allocator.  im_estimate_static serves them from a static scratch array in
the library.  This file is collected last, so a run that stops at the first failure has run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_estimate_static_matches_estimate_on_consecutive_calls():
    import torch

    import paper_2105_04023_gb300 as im
    from paper_2105_04023_gb300 import build
    from synth import graphs

    build.build()
    ctx = im.Context(0)
    try:
        g = graphs.rmat(12, 12, seed=61)
        for R in (256, 64):
            sk = ctx.im_build_sketches(im.Graph.from_synth(g, im.IM_WC), im.params(R=R, seed=8))
            M = torch.from_numpy(sk.im_sketch_registers()).cuda()
            # two calls in a row on the shared scratch: a small set, then a set spread over several blocks
            for S in ([5, 77, 1000], list(range(0, 4000, 23))):
                seeds = torch.tensor(S, dtype=torch.int32, device="cuda")
                e_static, g_static = ctx.im_estimate_static(M, seeds)
                e_ref, _ = sk.im_estimate(S)
                assert e_static == pytest.approx(e_ref, rel=1e-12)
                ref_sum = int(M.cpu().numpy()[np.array(S)].max(axis=0).astype(np.int64).sum())
                assert g_static == ref_sum
            sk.close()
        # arguments outside the stated limits are refused, and the next call is unaffected
        bad = torch.tensor([1, g.n], dtype=torch.int32, device="cuda")
        with pytest.raises(im.ImError):
            ctx.im_estimate_static(M, bad)
        too_many = torch.zeros(4097, dtype=torch.int32, device="cuda")
        with pytest.raises(im.ImError):
            ctx.im_estimate_static(M, too_many)
        e_after, _ = ctx.im_estimate_static(M, torch.tensor([5, 77, 1000], dtype=torch.int32, device="cuda"))
        assert e_after > 0
    finally:
        ctx.close()
