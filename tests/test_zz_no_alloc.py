"""The allocation-free surrogate gradient against the allocating entry point.

dmb_surrogate_grad_noalloc exists for callers that cannot allocate device memory when they need
the gradient (graph capture, an external allocator, allocation-free loops); it must give the
same loss and gradient as dmb_surrogate_grad, on consecutive calls that reuse its fixed work
array.  This file is collected last so a failure here does not hide the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import require_gpu, torch

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the float32 tolerance of the other GPU tests


def _ctx():
    from paper_2603_24688_gb300 import dmb
    ctx = dmb.Context(1e-24, 0, 2.0, 100.0, True, (1.0, 1.0, 1.0), 9, rate_mode=dmb.DMB_RATE_MLP)
    rng = np.random.default_rng(21)
    n = ctypes.c_int64()
    ctx.lib.dmb_surrogate_params(ctx.h, None, ctypes.byref(n))
    ctx.dmb_load_surrogate((rng.uniform(-1, 1, n.value) * 0.2).astype(np.float32))
    return ctx


@pytest.mark.parametrize("B", [1000, 4096])
def test_noalloc_gradient_matches_allocating_gradient(B):
    require_gpu()
    ctx = _ctx()
    rng = np.random.default_rng(B)
    n = ctypes.c_int64()
    ctx.lib.dmb_surrogate_params(ctx.h, None, ctypes.byref(n))
    for call in range(2):   # two calls in a row: the shared work array is reused
        X = torch.from_numpy(rng.uniform(-1, 1, (B, 4)).astype(np.float32)).cuda()
        Y = torch.from_numpy(rng.normal(size=(B, 2)).astype(np.float32)).cuda()
        g_ref = torch.empty(n.value, dtype=torch.float32, device="cuda")
        g_new = torch.full((n.value,), float("nan"), dtype=torch.float32, device="cuda")
        loss_ref = ctx.dmb_surrogate_grad(X, Y, g_ref)
        # through the C ABI directly
        loss = ctypes.c_double()
        st = ctx.lib.dmb_surrogate_grad_noalloc(ctx.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                                B, ctypes.c_void_p(g_new.data_ptr()), ctypes.byref(loss))
        assert st == 0, ctx.lib.dmb_last_error(ctx.h)
        torch.cuda.synchronize()
        a, b = g_new.cpu().numpy(), g_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        np.testing.assert_allclose(a, b, rtol=TOL, atol=TOL * np.abs(b).max())
        assert abs(loss.value - loss_ref) <= TOL * abs(loss_ref)


def test_noalloc_rejects_batches_beyond_its_array():
    require_gpu()
    ctx = _ctx()
    X = torch.zeros((4097, 4), dtype=torch.float32, device="cuda")
    Y = torch.zeros((4097, 2), dtype=torch.float32, device="cuda")
    g = torch.zeros(40000, dtype=torch.float32, device="cuda")
    loss = ctypes.c_double()
    st = ctx.lib.dmb_surrogate_grad_noalloc(ctx.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), 4097,
                                            ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss))
    assert st == 1
    assert b"4096" in ctx.lib.dmb_last_error(ctx.h)
