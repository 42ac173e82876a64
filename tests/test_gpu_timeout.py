"""Failure detection on the tensor cores: a bounded wait that runs out.

The tensor-core surrogate waits on an mbarrier for each MMA's completion with a time limit, after
which it records DMB_BAD_TIMEOUT, waits (bounded) for the MMAs it has in flight, releases its
tensor memory and ends.  The fault is injected on the host (dmb_debug_tc_timeout): one commit is
left out, so one warpgroup's wait runs out after 1 ms.  No GPU fault is involved.
"""
import ctypes
import time

import numpy as np
import pytest

from gpu_common import require_gpu, torch

pytestmark = pytest.mark.gpu


def _ctx(engine_nwg):
    from paper_2603_24688_gb300 import dmb
    ctx = dmb.Context(1e-24, 0, 2.0, 100.0, True, (1.0, 1.0, 1.0), 9, rate_mode=dmb.DMB_RATE_MLP)
    n = ctypes.c_int64()
    ctx.lib.dmb_surrogate_params(ctx.h, None, ctypes.byref(n))
    rng = np.random.default_rng(5)
    ctx.dmb_load_surrogate((rng.uniform(-1, 1, n.value) * 0.2).astype(np.float32))
    shapes = ctx.dmb_get_shapes()
    shapes["tc_warpgroups"] = engine_nwg
    ctx.dmb_set_shapes(shapes)
    assert ctx.dmb_get_shapes()["tc_warpgroups"] == engine_nwg
    return ctx


def _infer(ctx, X, Y):
    return ctx.lib.dmb_surrogate_infer_tc(ctx.h, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                          ctypes.c_void_p(Y.data_ptr()))


@pytest.mark.parametrize("nwg", [2, 3, 4])
def test_timed_out_wait_returns_timeout_and_the_context_recovers(nwg):
    require_gpu()
    from paper_2603_24688_gb300 import dmb
    ctx = _ctx(nwg)
    rng = np.random.default_rng(nwg)
    X = torch.from_numpy(rng.uniform(-1, 1, (200_000, 4)).astype(np.float32)).cuda()
    Y0 = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
    assert _infer(ctx, X, Y0) == dmb.DMB_OK
    # the injected fault: the call reports the timed-out wait, quickly
    assert ctx.lib.dmb_debug_tc_timeout(ctx.h, 1) == dmb.DMB_OK
    Y1 = torch.empty_like(Y0)
    t0 = time.time()
    st = _infer(ctx, X, Y1)
    assert st == dmb.DMB_ERR_TIMEOUT, (st, ctx.lib.dmb_last_error(ctx.h))
    assert b"timed out" in ctx.lib.dmb_last_error(ctx.h)
    assert time.time() - t0 < 10.0
    # tensor memory was released and the status cleared: the next calls succeed, bit for bit
    for _ in range(2):
        Y2 = torch.empty_like(Y0)
        assert _infer(ctx, X, Y2) == dmb.DMB_OK, ctx.lib.dmb_last_error(ctx.h)
        torch.cuda.synchronize()
        assert torch.equal(Y2, Y0)
    # a second context on the same device allocates tensor memory normally too
    ctx2 = _ctx(nwg)
    Y3 = torch.empty_like(Y0)
    assert _infer(ctx2, X, Y3) == dmb.DMB_OK
    torch.cuda.synchronize()
    assert torch.equal(Y3, Y0)


def test_fault_injection_flag_is_one_shot_and_checked():
    require_gpu()
    from paper_2603_24688_gb300 import dmb
    ctx = _ctx(4)
    assert ctx.lib.dmb_debug_tc_timeout(ctx.h, 2) == dmb.DMB_ERR_ARG
    assert ctx.lib.dmb_debug_tc_timeout(ctx.h, 1) == dmb.DMB_OK
    assert ctx.lib.dmb_debug_tc_timeout(ctx.h, 0) == dmb.DMB_OK     # cancelled
    X = torch.zeros((1000, 4), dtype=torch.float32, device="cuda")
    Y = torch.empty((1000, 2), dtype=torch.float32, device="cuda")
    assert _infer(ctx, X, Y) == dmb.DMB_OK
