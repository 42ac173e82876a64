"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_24688_gb300 import build, dmb
    build.build()
    dmb.load()


def make_ctx(w, fp64=False):
    from paper_2603_24688_gb300 import dmb
    return dmb.Context.from_params(w["params"], fp64=fp64)


def device_inputs(w):
    from paper_2603_24688_gb300 import dmb
    return dmb.to_device(w["dm"]), dmb.to_device(w["gas"])


def gpu_pairs(ctx, dm, gas, cap=None):
    ctx.dmb_build_grid(dm, gas)
    n = ctx.dmb_neighbors()
    out = torch.empty((max(n, 1), 2), dtype=torch.int32, device="cuda")
    ctx.dmb_neighbors(out)
    torch.cuda.synchronize()
    p = out[:n].cpu().numpy().view(np.uint32).astype(np.int64)
    return p[:, 0], p[:, 1]


def pair_band_mask(w, pi, pj):
    """Pairs within 1e-6 relative of the kernel radius h_i + h_j (exempt from bit-exactness)."""
    from oracle.pairs import pair_distance
    d = pair_distance(w["dm"]["pos"][pi], w["gas"]["pos"][pj], w["params"]["periodic"], w["params"]["box"])
    r = w["dm"]["h"][pi] + w["gas"]["h"][pj]
    return np.abs(d - r) <= 1e-6 * r
