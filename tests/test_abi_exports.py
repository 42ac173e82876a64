"""The C ABI library loads on a machine without a GPU and exports every symbol of dmb.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dmb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dmb_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ("dmb_build_grid", "dmb_neighbors", "dmb_meanfield_gas", "dmb_mc_scatter_dm", "dmb_step"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2603_24688_gb300 import build, dmb
    try:
        build.build()
    except RuntimeError as e:  # no CUDA toolkit: nothing to check here
        pytest.skip(str(e))
    lib = dmb.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(dmb.EXPORTS) == set(_declared())        # the binding covers every entry point


def test_no_fallback_without_library(tmp_path):
    from paper_2603_24688_gb300 import dmb
    with pytest.raises(RuntimeError):
        dmb.load(str(tmp_path / "missing.so"))


def test_timestep_bins_keep_every_substep_between_1_and_10_percent():
    import numpy as np
    from paper_2603_24688_gb300 import workloads as W
    b = W.timestep_bins(400_000, 7)
    assert b.dtype == np.uint8 and b.min() == 0 and b.max() == 11
    for s in (1, 2, 3, 4, 6, 8, 64, 512, 1024, 1536):
        frac = np.mean(s % (2.0 ** b) == 0)
        assert 0.009 < frac < 0.102, (s, frac)
    assert np.all(0 % (2.0 ** b) == 0)          # substep 0: everything active


def test_setters_refuse_a_null_context_without_touching_a_gpu():
    import ctypes
    from paper_2603_24688_gb300 import build, dmb
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    lib = dmb.load()
    lib.dmb_set_anisotropy.argtypes = [ctypes.c_void_p, ctypes.c_double]
    lib.dmb_set_anisotropy.restype = ctypes.c_int
    lib.dmb_set_mc_variant.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    lib.dmb_set_mc_variant.restype = ctypes.c_int
    assert lib.dmb_set_anisotropy(None, 0.5) == dmb.DMB_ERR_ARG
    assert lib.dmb_set_mc_variant(None, 0) == dmb.DMB_ERR_ARG
