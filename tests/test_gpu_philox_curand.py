"""Known-answer pin of the oracle's Philox4x32-10 against an independent implementation.

No published test vectors are available here, so the oracle's generator (oracle/philox.py,
written from Salmon et al., SC'11) is compared word for word with cuRAND's device function
curand_Philox4x32_10(counter, key), an implementation that shares nothing with this repository.
A wrong multiplier, Weyl constant, word order or key schedule in the oracle fails here.  The
small reference kernel (tests/native/curand_philox_ref.cu) is compiled by this test with nvcc;
it is not part of the library.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from gpu_common import require_gpu
from oracle import philox as P

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    require_gpu()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("curand") / "libcurand_philox_ref.so")
    src = os.path.join(HERE, "native", "curand_philox_ref.cu")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    "-o", out, src], check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.curand_philox_words.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    lib.curand_philox_words.restype = ctypes.c_int
    return lib


def _curand(lib, ctr, key):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(ctr)
    rc = lib.curand_philox_words(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, len(ctr))
    assert rc == 0, f"CUDA error {rc}"
    return out


def _oracle(ctr, key):
    out = np.zeros((len(ctr), 4), dtype=np.uint32)
    # the oracle takes one key per call: group the rows by key
    keys, inv = np.unique(key, axis=0, return_inverse=True)
    for k, (k0, k1) in enumerate(keys):
        m = inv.reshape(-1) == k
        c = ctr[m].astype(np.uint64)
        w = P.philox4x32_10(c[:, 0], c[:, 1], c[:, 2], c[:, 3], int(k0), int(k1))
        out[m] = np.stack([x.astype(np.uint32) for x in w], axis=1)
    return out


def test_oracle_matches_curand_on_random_counters_and_keys(curand_lib):
    rng = np.random.default_rng(2603)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    got = _oracle(ctr, key)
    ref = _curand(curand_lib, ctr, key)
    bad = np.nonzero(np.any(got != ref, axis=1))[0]
    assert bad.size == 0, (bad[:5], got[bad[:2]], ref[bad[:2]])


def test_oracle_matches_curand_on_edge_counters(curand_lib):
    edge = [0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF]
    ctr = np.array([[a, b, c, d] for a in edge for b in (0, 0xFFFFFFFF) for c in edge for d in (0, 0x80000000)],
                   dtype=np.uint32)
    for k0, k1 in ((0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0x260324688 & 0xFFFFFFFF, 0x2)):
        key = np.tile(np.array([[k0, k1]], dtype=np.uint32), (len(ctr), 1))
        np.testing.assert_array_equal(_oracle(ctr, key), _curand(curand_lib, ctr, key))


def test_method_streams_match_curand(curand_lib):
    # the three counter layouts of the method (pair, DM and Bernoulli streams), seed as key
    seed, step = 0x260324688 + 3, (5 << 32) | 17
    ids_i = np.arange(0, 2000, 7, dtype=np.uint64)
    ids_j = (ids_i * 2654435761) & 0xFFFFFFFF
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    for words, ctr in (
            (P.pair_words(seed, step, ids_i, ids_j),
             np.stack([ids_i, ids_j, np.full_like(ids_i, step & 0xFFFFFFFF),
                       np.full_like(ids_i, (step >> 32) & 0x7FFFFFFF)], axis=1)),
            (P.dm_words(seed, step, ids_i),
             np.stack([ids_i, np.zeros_like(ids_i), np.full_like(ids_i, step & 0xFFFFFFFF),
                       np.full_like(ids_i, ((step >> 32) & 0x7FFFFFFF) | 0x80000000)], axis=1)),
            (P.bern_words(seed, step, ids_i, ids_j),
             np.stack([ids_i, ids_j, np.full_like(ids_i, step & 0xFFFFFFFF),
                       np.full_like(ids_i, ((step >> 32) & 0x3FFFFFFF) | 0x40000000)], axis=1))):
        key = np.tile(np.array([[k0, k1]], dtype=np.uint32), (len(ids_i), 1))
        ref = _curand(curand_lib, ctr.astype(np.uint32), key)
        got = np.stack([w.astype(np.uint32) for w in words], axis=1)
        np.testing.assert_array_equal(got, ref)
