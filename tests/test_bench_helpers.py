"""Host-side helpers of bench.py: its copy of the surrogate's envelopes agrees with the oracle's
restatement (both restate the library's), the CPU-baseline sub-cubes stay bounded in dense
regions, the gas temperature ratio of the galaxy workload, and the NUMA binding's fallback."""
import numpy as np

import bench
from oracle import mlp as O
from oracle import units
from paper_2603_24688_gb300 import workloads as W


def test_envelopes_match_the_oracle():
    for n in (-4, -3, -2, -1, 0, 1, 2, 5):
        a, b = bench.envelope(n), O.envelope(n)
        for ea, eb in zip(a, b):
            assert np.allclose(ea, eb, rtol=1e-14, atol=0), (n, ea, eb)


def test_subcubes_are_bounded_in_dense_regions():
    w = W.subsample(W.named("galaxy1M"), 40_000, 40_000, seed=4)
    cubes, (smin, smax) = bench._subcubes(w, 12, 20_000, seed=3)
    assert len(cubes) == 12 and 0 < smin <= smax
    first = len(cubes[0][0]["h"]) * len(cubes[0][1]["h"])
    for d, g in cubes[1:]:
        assert 0 < len(d["h"]) * len(g["h"]) <= 2 * first
        assert len(d["h"]) and len(g["h"])


def test_workload_tau_of_the_galaxy():
    w = W.named("galaxy1M")
    lo, hi = bench.workload_tau(w)
    T, mu = w["gas"]["T"], w["gas"]["mu"]
    ref = units.varsigma2_kms2(T[T > 0], mu[T > 0]) / w["params"]["v0_kms"] ** 2
    assert np.isclose(lo, ref.min(), rtol=1e-6) and np.isclose(hi, ref.max(), rtol=1e-6)


def test_numa_binding_falls_back_without_a_device():
    import torch
    if torch.cuda.is_available():
        return
    assert bench.bind_to_gpu_numa_node(0) is None
