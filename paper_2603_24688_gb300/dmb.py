"""Thin ctypes binding of libdmb.so (the C ABI declared in include/dmb.h).

Argument marshalling only: every step of the interaction runs in the library's CUDA
kernels.  Device arrays are passed as torch CUDA tensors (float64 / uint32 / uint8 /
float32, contiguous); host outputs come back as Python values or numpy arrays.
There is no CPU fallback: if the library cannot be loaded every call raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdmb.so")

DMB_OK, DMB_ERR_ARG, DMB_ERR_CUDA, DMB_ERR_OOM, DMB_ERR_TIMEOUT, DMB_ERR_DOMAIN, DMB_ERR_STATE = range(7)
DMB_RATE_CLOSED, DMB_RATE_QUAD, DMB_RATE_MLP = range(3)
NO_PARTNER = 0xFFFFFFFF
STATUS_NAMES = {0: "DMB_OK", 1: "DMB_ERR_ARG", 2: "DMB_ERR_CUDA", 3: "DMB_ERR_OOM", 4: "DMB_ERR_TIMEOUT",
                5: "DMB_ERR_DOMAIN", 6: "DMB_ERR_STATE"}

EXPORTS = ["dmb_create", "dmb_destroy", "dmb_last_error", "dmb_build_grid", "dmb_neighbors", "dmb_meanfield_gas",
           "dmb_mc_scatter_dm", "dmb_step", "dmb_debug_overlap", "dmb_debug_rates", "dmb_debug_philox",
           "dmb_launch_count", "dmb_set_timing", "dmb_stage_times",
           "dmb_search_stats", "dmb_train_surrogate", "dmb_surrogate_params", "dmb_load_surrogate",
           "dmb_surrogate_infer", "dmb_surrogate_grad", "dmb_surrogate_fallbacks", "dmb_step_batched",
           "dmb_surrogate_grad_noalloc", "dmb_set_bins", "dmb_substep_info", "dmb_substep", "dmb_set_graph",
           "dmb_set_surrogate_engine", "dmb_surrogate_infer_tc", "dmb_autotune", "dmb_set_shapes",
           "dmb_get_shapes", "dmb_rebin_dm", "dmb_set_mc_variant", "dmb_set_anisotropy", "dmb_debug_tc_timeout",
           "dmb_set_cross_section", "dmb_debug_rates_screened", "dmb_save_shapes", "dmb_load_shapes",
           "dmb_set_surrogate_scope", "dmb_set_fusion", "dmb_set_surrogate_epilogue", "dmb_set_pair_weights"]


class DmbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("sigma0_cm2", ctypes.c_double), ("v0_kms", ctypes.c_double), ("n", ctypes.c_int32),
                ("periodic", ctypes.c_int32), ("m_chi_mp", ctypes.c_double), ("box", ctypes.c_double * 3),
                ("rate_mode", ctypes.c_int32), ("fp64", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class Box(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("sigma0_cm2", ctypes.c_double), ("m_chi_mp", ctypes.c_double)]


class DM(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("mass", ctypes.c_void_p),
                ("h", ctypes.c_void_p), ("id", ctypes.c_void_p)]


class Gas(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("mass", ctypes.c_void_p),
                ("h", ctypes.c_void_p), ("T", ctypes.c_void_p), ("mu", ctypes.c_void_p), ("id", ctypes.c_void_p)]


_lib = None


def load(path=LIB_PATH):
    """Load libdmb.so once; raises if it is missing (no fallback path exists)."""
    global _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2603_24688_gb300.build`")
    if _lib is not None and path == LIB_PATH:
        return _lib
    lib = ctypes.CDLL(path)
    c = ctypes
    vp, i64, u64, dbl = c.c_void_p, c.c_int64, c.c_uint64, c.c_double
    sig = {
        "dmb_create": ([c.POINTER(vp), c.POINTER(Params), vp], c.c_int),
        "dmb_destroy": ([vp], c.c_int),
        "dmb_last_error": ([vp], c.c_char_p),
        "dmb_build_grid": ([vp, c.POINTER(DM), c.POINTER(Gas)], c.c_int),
        "dmb_neighbors": ([vp, c.POINTER(i64), vp, i64], c.c_int),
        "dmb_meanfield_gas": ([vp, vp, vp], c.c_int),
        "dmb_mc_scatter_dm": ([vp, u64, dbl, vp, vp, vp, vp, vp], c.c_int),
        "dmb_step": ([vp, c.POINTER(DM), c.POINTER(Gas), u64, dbl, vp], c.c_int),
        "dmb_debug_overlap": ([vp, i64, vp, vp], c.c_int),
        "dmb_debug_rates": ([vp, i64, vp, vp], c.c_int),
        "dmb_debug_philox": ([vp, i64, vp, vp], c.c_int),
        "dmb_launch_count": ([vp], i64),
        "dmb_set_timing": ([vp, c.c_int], c.c_int),
        "dmb_stage_times": ([vp, c.POINTER(c.c_double), c.POINTER(i64)], c.c_int),
        "dmb_search_stats": ([vp, c.POINTER(c.c_uint64)], c.c_int),
        "dmb_train_surrogate": ([vp, i64, c.c_int32, u64, c.POINTER(c.c_double)], c.c_int),
        "dmb_surrogate_params": ([vp, c.POINTER(c.c_float), c.POINTER(i64)], c.c_int),
        "dmb_load_surrogate": ([vp, c.POINTER(c.c_float), i64], c.c_int),
        "dmb_surrogate_infer": ([vp, vp, i64, vp], c.c_int),
        "dmb_surrogate_grad": ([vp, vp, vp, c.c_int32, vp, c.POINTER(c.c_double)], c.c_int),
        "dmb_surrogate_fallbacks": ([vp, c.POINTER(i64)], c.c_int),
        "dmb_step_batched": ([vp, c.POINTER(DM), vp, c.POINTER(Gas), vp, c.POINTER(Box), c.c_int32, u64, dbl,
                              vp], c.c_int),
        "dmb_surrogate_grad_noalloc": ([vp, vp, vp, c.c_int32, vp, c.POINTER(c.c_double)], c.c_int),
        "dmb_set_bins": ([vp, vp, vp], c.c_int),
        "dmb_substep_info": ([vp, u64, c.POINTER(i64)], c.c_int),
        "dmb_substep": ([vp, c.POINTER(DM), c.POINTER(Gas), u64, dbl, vp], c.c_int),
        "dmb_set_graph": ([vp, c.c_int], c.c_int),
        "dmb_set_surrogate_engine": ([vp, c.c_int32], c.c_int),
        "dmb_surrogate_infer_tc": ([vp, vp, i64, vp], c.c_int),
        "dmb_autotune": ([vp, c.POINTER(DM), c.POINTER(Gas), c.POINTER(c.c_int32), c.POINTER(c.c_double)], c.c_int),
        "dmb_set_shapes": ([vp, c.POINTER(c.c_int32)], c.c_int),
        "dmb_get_shapes": ([vp, c.POINTER(c.c_int32)], c.c_int),
        "dmb_rebin_dm": ([vp, vp, vp, i64, c.c_int32, u64, vp, c.POINTER(i64)], c.c_int),
        "dmb_set_mc_variant": ([vp, c.c_int32], c.c_int),
        "dmb_set_anisotropy": ([vp, c.c_double], c.c_int),
        "dmb_debug_tc_timeout": ([vp, c.c_int32], c.c_int),
        "dmb_set_cross_section": ([vp, c.c_int32, dbl], c.c_int),
        "dmb_debug_rates_screened": ([vp, i64, vp, vp], c.c_int),
        "dmb_save_shapes": ([vp, c.c_char_p, c.c_char_p], c.c_int),
        "dmb_load_shapes": ([vp, c.c_char_p, c.c_char_p], c.c_int),
        "dmb_set_surrogate_scope": ([vp, c.c_int32], c.c_int),
        "dmb_set_fusion": ([vp, c.c_int32], c.c_int),
        "dmb_set_surrogate_epilogue": ([vp, c.c_int32], c.c_int),
        "dmb_set_pair_weights": ([vp, c.c_int32], c.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(t, dtype=None):
    if t is None:
        return None
    import torch
    if not t.is_cuda:
        raise ValueError("device arrays must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("device arrays must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """Owns a dmb_ctx.  Methods mirror the C entry points with the same names."""

    def __init__(self, sigma0_cm2, n, m_chi_mp, v0_kms=100.0, periodic=False, box=(0.0, 0.0, 0.0), seed=0,
                 fp64=False, rate_mode=DMB_RATE_CLOSED, stream=None):
        import torch
        self.lib = load()
        p = Params()
        p.sigma0_cm2 = float(sigma0_cm2)
        p.v0_kms = float(v0_kms)
        p.n = int(n)
        p.periodic = 1 if periodic else 0
        p.m_chi_mp = float(m_chi_mp)
        for k in range(3):
            p.box[k] = float(box[k])
        p.rate_mode = int(rate_mode)
        p.fp64 = 1 if fp64 else 0
        p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        self.params = p
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self.lib.dmb_create(ctypes.byref(h), ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream))
        if st != DMB_OK:
            raise DmbError(st, self.lib.dmb_last_error(None).decode())
        self.h = h
        self._keep = []

    @classmethod
    def from_params(cls, params, fp64=False, stream=None):
        return cls(params["sigma0_cm2"], params["n"], params["m_chi_mp"], params["v0_kms"], params["periodic"],
                   tuple(params["box"]), params["seed"], fp64=fp64, stream=stream)

    def _check(self, st):
        if st != DMB_OK:
            raise DmbError(st, self.lib.dmb_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.dmb_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def dm_struct(dm):
        import torch
        s = DM()
        s.n = int(dm["h"].numel())
        s.pos = _ptr(dm["pos"], torch.float64)
        s.vel = _ptr(dm["vel"], torch.float64)
        s.mass = _ptr(dm["mass"], torch.float64)
        s.h = _ptr(dm["h"], torch.float64)
        s.id = _ptr(dm["id"], torch.int32)
        return s

    @staticmethod
    def gas_struct(gas):
        import torch
        s = Gas()
        s.n = int(gas["h"].numel())
        s.pos = _ptr(gas["pos"], torch.float64)
        s.vel = _ptr(gas["vel"], torch.float64)
        s.mass = _ptr(gas["mass"], torch.float64)
        s.h = _ptr(gas["h"], torch.float64)
        s.T = _ptr(gas["T"], torch.float64)
        s.mu = _ptr(gas["mu"], torch.float64)
        s.id = _ptr(gas["id"], torch.int32)
        return s

    def dmb_build_grid(self, dm, gas):
        self._dm_s, self._gas_s = self.dm_struct(dm), self.gas_struct(gas)
        self._keep = [dm, gas]
        self._check(self.lib.dmb_build_grid(self.h, ctypes.byref(self._dm_s), ctypes.byref(self._gas_s)))

    def dmb_neighbors(self, pairs_out=None):
        n = ctypes.c_int64()
        cap = 0 if pairs_out is None else pairs_out.numel() // 2
        import torch
        self._check(self.lib.dmb_neighbors(self.h, ctypes.byref(n), _ptr(pairs_out, torch.int32), cap))
        return n.value

    def dmb_meanfield_gas(self, acc, dudt):
        import torch
        self._check(self.lib.dmb_meanfield_gas(self.h, _ptr(acc, torch.float64), _ptr(dudt, torch.float64)))

    def dmb_mc_scatter_dm(self, step, dt, vel_out, scattered=None, partner=None, p_ratio_max=None, p_total=None):
        import torch
        self._check(self.lib.dmb_mc_scatter_dm(self.h, int(step), float(dt), _ptr(vel_out, torch.float64),
                                               _ptr(scattered, torch.uint8), _ptr(partner, torch.int32),
                                               _ptr(p_ratio_max, torch.float32), _ptr(p_total, torch.float64)))

    def dmb_step(self, dm, gas, step, dt, want_sums=True):
        d, g = self.dm_struct(dm), self.gas_struct(gas)
        sums = (ctypes.c_double * 16)()
        self._check(self.lib.dmb_step(self.h, ctypes.byref(d), ctypes.byref(g), int(step), float(dt),
                                      sums if want_sums else None))
        return np.array(sums[:]) if want_sums else None

    def dmb_step_batched(self, dm, dm_box, gas, gas_box, boxes, step, dt, want_sums=True):
        """boxes: sequence of (box[3], sigma0_cm2, m_chi_mp); dm_box / gas_box: CUDA int32 tensors."""
        import torch
        d, g = self.dm_struct(dm), self.gas_struct(gas)
        tbl = (Box * len(boxes))()
        for k, (bx, sg, mc) in enumerate(boxes):
            for c in range(3):
                tbl[k].box[c] = float(bx[c])
            tbl[k].sigma0_cm2 = float(sg)
            tbl[k].m_chi_mp = float(mc)
        sums = (ctypes.c_double * 16)()
        self._check(self.lib.dmb_step_batched(self.h, ctypes.byref(d), _ptr(dm_box, torch.int32), ctypes.byref(g),
                                              _ptr(gas_box, torch.int32), tbl, len(boxes), int(step), float(dt),
                                              sums if want_sums else None))
        return np.array(sums[:]) if want_sums else None

    def dmb_set_bins(self, dm_bin, gas_bin):
        """dm_bin, gas_bin: CUDA uint8 tensors (caller order), kept alive by the context."""
        import torch
        self._bins = (dm_bin, gas_bin)
        self._check(self.lib.dmb_set_bins(self.h, _ptr(dm_bin, torch.uint8), _ptr(gas_bin, torch.uint8)))

    def dmb_substep_info(self, substep):
        out = (ctypes.c_int64 * 5)()
        self._check(self.lib.dmb_substep_info(self.h, int(substep), out))
        return tuple(int(v) for v in out)

    def dmb_substep(self, dm, gas, substep, dt_min, want_sums=True):
        d, g = self.dm_struct(dm), self.gas_struct(gas)
        sums = (ctypes.c_double * 16)()
        self._check(self.lib.dmb_substep(self.h, ctypes.byref(d), ctypes.byref(g), int(substep), float(dt_min),
                                         sums if want_sums else None))
        return np.array(sums[:]) if want_sums else None

    def dmb_set_surrogate_engine(self, engine):
        self._check(self.lib.dmb_set_surrogate_engine(self.h, int(engine)))

    def dmb_surrogate_infer_tc(self, X, Y):
        import torch
        self._check(self.lib.dmb_surrogate_infer_tc(self.h, _ptr(X, torch.float32), X.shape[0],
                                                    _ptr(Y, torch.float32)))

    SHAPE_NAMES = ("unit", "seg", "mf_blocks_per_sm", "mc_blocks_per_sm", "tc_warpgroups")

    def dmb_autotune(self, dm, gas):
        """Returns (shapes dict, candidate times in ms)."""
        d, g = self.dm_struct(dm), self.gas_struct(gas)
        sh = (ctypes.c_int32 * 5)()
        rep = (ctypes.c_double * 23)(*([float("nan")] * 23))
        self._check(self.lib.dmb_autotune(self.h, ctypes.byref(d), ctypes.byref(g), sh, rep))
        return dict(zip(self.SHAPE_NAMES, [int(v) for v in sh])), [v for v in rep if v == v]

    def dmb_set_shapes(self, shapes):
        v = (ctypes.c_int32 * 5)(*[int(shapes[k]) for k in self.SHAPE_NAMES])
        self._check(self.lib.dmb_set_shapes(self.h, v))

    def dmb_save_shapes(self, path, key):
        self._check(self.lib.dmb_save_shapes(self.h, str(path).encode(), str(key).encode()))

    def dmb_load_shapes(self, path, key):
        """True if shapes were stored under key (and are now set), False if absent."""
        st = self.lib.dmb_load_shapes(self.h, str(path).encode(), str(key).encode())
        if st == DMB_ERR_STATE:
            return False
        self._check(st)
        return True

    def dmb_get_shapes(self):
        v = (ctypes.c_int32 * 5)()
        self._check(self.lib.dmb_get_shapes(self.h, v))
        return dict(zip(self.SHAPE_NAMES, [int(x) for x in v]))

    def dmb_rebin_dm(self, p_ratio_max, dm_bin, max_bin, substep=0, active=None):
        """p_ratio_max: CUDA float32 [n]; dm_bin: CUDA uint8 [n] (updated in place); returns the
        number of bins that moved."""
        import torch
        out = ctypes.c_int64()
        self._check(self.lib.dmb_rebin_dm(self.h, _ptr(p_ratio_max, torch.float32), _ptr(dm_bin, torch.uint8),
                                          int(dm_bin.numel()), int(max_bin), int(substep),
                                          _ptr(active, torch.uint8), ctypes.byref(out)))
        return out.value

    def dmb_set_mc_variant(self, variant):
        """0: one categorical draw per DM particle (default); 1: per-pair Bernoulli draws."""
        self._check(self.lib.dmb_set_mc_variant(self.h, int(variant)))

    def dmb_set_anisotropy(self, beta):
        """dsigma/dOmega proportional to 1 + beta cos theta, beta in [-1, 1] (0: isotropic)."""
        self._check(self.lib.dmb_set_anisotropy(self.h, float(beta)))

    def dmb_set_cross_section(self, family, v_c_kms=0.0):
        """0: sigma0 (v/v0)^n; 1: the screened law sigma0 / (1 + (v/v_c)^2)^2."""
        self._check(self.lib.dmb_set_cross_section(self.h, int(family), float(v_c_kms)))

    def dmb_debug_rates_screened(self, inp, out):
        import torch
        self._check(self.lib.dmb_debug_rates_screened(self.h, inp.shape[0], _ptr(inp, torch.float64),
                                                      _ptr(out, torch.float64)))

    def dmb_set_fusion(self, on=True):
        """1: one pass evaluates each pair for the mean field and the Monte Carlo; 0: separate passes."""
        self._check(self.lib.dmb_set_fusion(self.h, 1 if on else 0))

    def dmb_set_pair_weights(self, mode):
        """-1: stored for pair sets kept for later calls (dmb_neighbors); 0: never; 1: always."""
        self._check(self.lib.dmb_set_pair_weights(self.h, int(mode)))

    def dmb_set_surrogate_epilogue(self, mode):
        """1: the surrogate's tensor-core kernel sums the mean field itself; 0: it stores the rates."""
        self._check(self.lib.dmb_set_surrogate_epilogue(self.h, int(mode)))

    def dmb_set_surrogate_scope(self, scope):
        """0: train for the scan's indices {-4, -2, 0, 2} and n; 1: for the context's n only."""
        self._check(self.lib.dmb_set_surrogate_scope(self.h, int(scope)))

    def dmb_set_graph(self, on=True):
        self._check(self.lib.dmb_set_graph(self.h, 1 if on else 0))

    def dmb_debug_overlap(self, inp, out):
        import torch
        self._check(self.lib.dmb_debug_overlap(self.h, inp.shape[0], _ptr(inp, torch.float64), _ptr(out, torch.float64)))

    def dmb_debug_rates(self, inp, out):
        import torch
        self._check(self.lib.dmb_debug_rates(self.h, inp.shape[0], _ptr(inp, torch.float64), _ptr(out, torch.float64)))

    def dmb_debug_philox(self, ctr, out):
        import torch
        self._check(self.lib.dmb_debug_philox(self.h, ctr.shape[0], _ptr(ctr, torch.int32), _ptr(out, torch.int32)))

    def dmb_launch_count(self):
        return int(self.lib.dmb_launch_count(self.h))

    def dmb_train_surrogate(self, nsamples=1 << 20, epochs=30, seed=1):
        """Train the rate surrogate on the device; returns the 8-entry report."""
        rep = (ctypes.c_double * 8)()
        self._check(self.lib.dmb_train_surrogate(self.h, int(nsamples), int(epochs), int(seed), rep))
        return np.array(rep[:])

    def dmb_surrogate_params(self):
        n = ctypes.c_int64()
        self._check(self.lib.dmb_surrogate_params(self.h, None, ctypes.byref(n)))
        out = np.zeros(n.value, dtype=np.float32)
        self._check(self.lib.dmb_surrogate_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                  ctypes.byref(n)))
        return out

    def dmb_load_surrogate(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self.lib.dmb_load_surrogate(self.h, params.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                params.size))

    def dmb_surrogate_infer(self, X, Y):
        import torch
        self._check(self.lib.dmb_surrogate_infer(self.h, _ptr(X, torch.float32), X.shape[0], _ptr(Y, torch.float32)))

    def dmb_surrogate_grad(self, X, Y, grad):
        import torch
        loss = ctypes.c_double()
        self._check(self.lib.dmb_surrogate_grad(self.h, _ptr(X, torch.float32), _ptr(Y, torch.float32), X.shape[0],
                                                _ptr(grad, torch.float32), ctypes.byref(loss)))
        return loss.value

    def dmb_surrogate_grad_noalloc(self, X, Y, grad, want_loss=True):
        """dmb_surrogate_grad with its work buffers in the library's fixed device array (B <= 4096).

        want_loss=False passes no loss pointer, so the call does not synchronise the stream."""
        import torch
        loss = ctypes.c_double()
        self._check(self.lib.dmb_surrogate_grad_noalloc(self.h, _ptr(X, torch.float32), _ptr(Y, torch.float32),
                                                        X.shape[0], _ptr(grad, torch.float32),
                                                        ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def dmb_debug_tc_timeout(self, on=True):
        """Fault injection: the next tensor-core surrogate launch times out one wait (DMB_ERR_TIMEOUT)."""
        self._check(self.lib.dmb_debug_tc_timeout(self.h, 1 if on else 0))

    def dmb_surrogate_fallbacks(self):
        n = ctypes.c_int64()
        self._check(self.lib.dmb_surrogate_fallbacks(self.h, ctypes.byref(n)))
        return n.value

    def dmb_search_stats(self):
        """Counters of the last pair search: (4 passes) x (nodes, leaves, tests, 0)."""
        out = (ctypes.c_uint64 * 16)()
        self._check(self.lib.dmb_search_stats(self.h, out))
        return np.array(out[:], dtype=np.uint64).reshape(4, 4)

    def dmb_set_timing(self, on=True):
        self._check(self.lib.dmb_set_timing(self.h, 1 if on else 0))

    def dmb_stage_times(self):
        """Return (ms per stage [8], steps) accumulated since the last call."""
        ms = (ctypes.c_double * 8)()
        n = ctypes.c_int64()
        self._check(self.lib.dmb_stage_times(self.h, ms, ctypes.byref(n)))
        return np.array(ms[:]), n.value


def to_device(particles, device="cuda"):
    """numpy particle dict (workloads format) -> dict of CUDA tensors (ids as int32 bit patterns)."""
    import torch
    out = {}
    for k, v in particles.items():
        if k == "id":
            out[k] = torch.from_numpy(np.asarray(v, dtype=np.uint32).view(np.int32).copy()).to(device)
        else:
            out[k] = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(device)
    return out
