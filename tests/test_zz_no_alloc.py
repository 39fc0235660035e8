"""The allocation-free estimate (im_estimate_static) gives what im_estimate gives, call after call.

Some callers cannot allocate device memory while they serve a request: a serving thread on a latency budget
(cudaMalloc can synchronise the device and serialises on a process-wide lock), or a host process that accounts
for every device byte through its own allocator.  im_estimate_static serves them from a static scratch array in
the library.  Its results are checked against im_estimate and against the CPU oracle's estimate of the same
register rows; the device's free memory must not move across calls.  This file is collected last, so a run that
stops at the first failure has run every other test.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_estimate_static_matches_estimate_on_consecutive_calls():
    import torch

    import oracle
    import paper_2105_04023_gb300 as im
    from paper_2105_04023_gb300 import build
    from synth import graphs

    build.build()
    ctx = im.Context(0)
    try:
        g = graphs.rmat(12, 12, seed=61)
        for R in (256, 64):
            sk = ctx.im_build_sketches(im.Graph.from_synth(g, im.IM_WC), im.params(R=R, seed=8))
            Mh = sk.im_sketch_registers()
            M = torch.from_numpy(Mh).cuda()
            # two calls in a row on the shared scratch: a small set, then a set spread over several blocks
            for S in ([5, 77, 1000], list(range(0, 4000, 23))):
                seeds = torch.tensor(S, dtype=torch.int32, device="cuda")
                e_static, g_static = ctx.im_estimate_static(M, seeds)
                e_ref, _ = sk.im_estimate(S)
                assert e_static == pytest.approx(e_ref, rel=1e-12)
                e_orc, g_orc = oracle.estimate_set(Mh, S)
                assert g_static == g_orc
                assert e_static == pytest.approx(e_orc, rel=1e-12)
            sk.close()
        # any byte values: the merge is an unsigned byte max, not one that relies on registers below 128
        rng = np.random.default_rng(3)
        B = rng.integers(0, 256, size=(300, 128), dtype=np.uint8)
        S = [0, 17, 299, 150]
        e_b, g_b = ctx.im_estimate_static(torch.from_numpy(B).cuda(), torch.tensor(S, dtype=torch.int32,
                                                                                   device="cuda"))
        assert g_b == oracle.estimate_set(B, S)[1]
        # no device memory is taken by repeated calls (after a warm-up call), and the caller's device is kept
        seeds = torch.tensor([5, 77, 1000], dtype=torch.int32, device="cuda")
        ctx.im_estimate_static(M, seeds)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(5):
            ctx.im_estimate_static(M, seeds)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert torch.cuda.current_device() == 0
        # arguments outside the stated limits are refused, and the next call is unaffected
        bad = torch.tensor([1, g.n], dtype=torch.int32, device="cuda")
        with pytest.raises(im.ImError):
            ctx.im_estimate_static(M, bad)
        too_many = torch.zeros(4097, dtype=torch.int32, device="cuda")
        with pytest.raises(im.ImError):
            ctx.im_estimate_static(M, too_many)
        # a register matrix that does not start on a 4-byte boundary is refused on the host, before any launch
        est = ctypes.c_double()
        st = ctx._L.im_estimate_static(ctx.h, M.data_ptr() + 1, g.n - 1, 64, seeds.data_ptr(), 3,
                                       ctypes.addressof(est), None)
        assert st == 1  # IM_EINVAL
        e_after, g_after = ctx.im_estimate_static(M, seeds)
        assert g_after == oracle.estimate_set(Mh, [5, 77, 1000])[1]
    finally:
        ctx.close()
