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


def transfer_scales(w, pi, pj, params, g=None):
    """Per gas particle, the sums of the absolute pair terms of its mean field: (acc [N_B, 3],
    du/dt [N_B]).  A float32 evaluation of the pair terms with relative error eps is off by at
    most eps times these, however much the signed terms cancel (the heating is a difference of
    two positive sums, w^2 A and e B; Eq. gas-dTdt)."""
    from oracle import units
    from oracle.meanfield import pair_rates
    gg, wv, A, B = pair_rates(w["dm"], w["gas"], pi, pj, params, g)
    mu = w["gas"]["mu"][pj]
    coef = w["dm"]["mass"][pi] * units.MSUN_PER_MP / (params["m_chi_mp"] + mu) * gg
    nb = len(w["gas"]["h"])
    sa = np.zeros((nb, 3))
    for c in range(3):
        np.add.at(sa[:, c], pj, np.abs(coef * A * wv[:, c]))
    su = np.zeros(nb)
    np.add.at(su, pj, np.abs(coef * A * np.sum(wv * wv, axis=1)) + np.abs(coef * mu / (params["m_chi_mp"] + mu) * B))
    return sa, su
