"""GB300 (sm_103a) implementation of the multi-step reconstruction of
radio-interferometric images (Wang, Prunet, Mignot, Ferrari).

A thin ctypes binding over ``libmstep.so`` (``include/mstep.h``): argument
marshalling only, every step of the path runs in the library's CUDA kernels.
Buffers are torch tensors on the plan's device; the calls are ordered on the
current torch stream.  There is no CPU fallback: if the library cannot be
loaded the import fails.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmstep.so")

MS_OK, MS_ERR_ARG, MS_ERR_CUDA, MS_ERR_OOM, MS_ERR_NUMERIC = 0, 1, 2, 3, 4
MS_ERR_TIMEOUT, MS_ERR_NOT_CONVERGED, MS_ERR_STATE, MS_ERR_UNSUPPORTED = 5, 6, 7, 8
MS_FP64, MS_FP32, MS_FP32_KAHAN = 0, 1, 2
MS_PART_L, MS_PART_H, MS_PART_ALL = 0, 1, 2
MS_STEP_LOW, MS_STEP_FULL, MS_STEP_SINGLE, MS_STEP_LOW_H, MS_STEP_FULL_L = 0, 1, 2, 3, 4
MS_LAMBDA_NORM2_2N, MS_LAMBDA_MAX_FIXED = 0, 1

PRECISIONS = {"fp64": MS_FP64, "fp32": MS_FP32, "fp32_kahan": MS_FP32_KAHAN}
MS_DICT_DAUBECHIES, MS_DICT_IUWT = 0, 1
DICTIONARIES = {"daubechies": MS_DICT_DAUBECHIES, "iuwt": MS_DICT_IUWT}
MS_CONV_CIRCULAR, MS_CONV_LINEAR = 0, 1
CONVOLUTIONS = {"circular": MS_CONV_CIRCULAR, "linear": MS_CONV_LINEAR}
PARTS = {"L": MS_PART_L, "H": MS_PART_H, "ALL": MS_PART_ALL}
STEPS = {"low": MS_STEP_LOW, "full": MS_STEP_FULL, "single": MS_STEP_SINGLE,
         "low_h": MS_STEP_LOW_H, "full_l": MS_STEP_FULL_L}


class MsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"mstep status {status}: {message}")
        self.status = status


class ms_plan_desc(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("flags", ctypes.c_void_p),
                ("nvis", ctypes.c_int64), ("nchan", ctypes.c_int32), ("npix", ctypes.c_int32),
                ("pixel_size", ctypes.c_double), ("ell_px", ctypes.c_double),
                ("delta_px", ctypes.c_double), ("kernel_width", ctypes.c_int32),
                ("oversample", ctypes.c_int32), ("es_beta", ctypes.c_double),
                ("levels", ctypes.c_int32), ("n_bases", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("device", ctypes.c_int32),
                ("dictionary", ctypes.c_int32), ("convolution", ctypes.c_int32)]


class ms_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("major_cycles", ctypes.c_int32), ("total_iterations", ctypes.c_int32),
                ("objective", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("theta", ctypes.c_double), ("sigma2", ctypes.c_double),
                ("eta2", ctypes.c_double), ("elapsed_ms", ctypes.c_double),
                ("grid_ms", ctypes.c_double), ("fft_ms", ctypes.c_double),
                ("minor_ms", ctypes.c_double), ("gridded_vis", ctypes.c_int64),
                ("objective_trace", ctypes.POINTER(ctypes.c_double))]


class ms_kernel_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 16), ("total_ms", ctypes.c_double * 16)]


KERNEL_FAMILIES = ["degrid", "grid", "fold", "fft_grid", "pad_crop", "synth", "synth_l1",
                   "fft_r2c", "spec_mul", "fft_c2r", "analysis", "analysis_l1", "linear_psf"]


class ms_recon_opts(ctypes.Structure):
    _fields_ = [("n_major", ctypes.c_int32), ("fista_iters", ctypes.c_int32),
                ("rel_tol", ctypes.c_double), ("lambda_rule", ctypes.c_int32),
                ("lambda_low", ctypes.c_double), ("lambda_full", ctypes.c_double),
                ("lambda_single", ctypes.c_double), ("sigma2", ctypes.c_double),
                ("eta2", ctypes.c_double), ("warm_start", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGNATURES = {
    "ms_plan_create": [ctypes.POINTER(ms_plan_desc), ctypes.POINTER(_P)],
    "ms_plan_destroy": [_P],
    "ms_last_error": [_P],
    "ms_partition_counts": [_P, _I32, ctypes.POINTER(_I64)],
    "ms_partition_rows": [_P, _I32, _I32, _P],
    "ms_partition_layout": [_P, _I32, _I32, ctypes.POINTER(_I64)],
    "ms_degrid": [_P, _I32, _I32, _P, _P, _P, _P],
    "ms_grid": [_P, _I32, _I32, _P, _P, _P],
    "ms_grid_static_scratch": [_P, _I32, _I32, _P, _P, _P],
    "ms_grid_batch": [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                      ctypes.POINTER(_P), ctypes.POINTER(_P), _P],
    "ms_degrid_batch": [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                        ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _P],
    "ms_minor_cycle_batch": [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                             ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_D),
                             ctypes.POINTER(_D), ctypes.POINTER(_D), _I32, _D, ctypes.POINTER(_P),
                             ctypes.POINTER(ms_stats), ctypes.POINTER(_D), _P],
    "ms_reconstruct_two_step_batch": [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_P),
                                      ctypes.POINTER(ms_recon_opts), ctypes.POINTER(_P),
                                      ctypes.POINTER(_P), ctypes.POINTER(ms_stats), _P],
    "ms_reconstruct_single_step_batch": [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_P),
                                         ctypes.POINTER(ms_recon_opts), ctypes.POINTER(_P),
                                         ctypes.POINTER(ms_stats), _P],
    "ms_reconstruct_step": [_P, _I32, _I32, _P, ctypes.POINTER(ms_recon_opts), _P, _P, _P,
                            ctypes.POINTER(ms_stats), _P],
    "ms_reconstruct_interleaved": [_P, _I32, _P, ctypes.POINTER(ms_recon_opts), _P, _P, _P,
                                   ctypes.POINTER(ms_stats), _P],
    "ms_plan_autotune": [ctypes.POINTER(ms_plan_desc), _I32, _I32, ctypes.POINTER(_I32),
                         ctypes.POINTER(_I32), ctypes.POINTER(_D)],
    "ms_residual_image": [_P, _I32, _I32, _P, _P, _P, _P],
    "ms_psf": [_P, _I32, _I32, _P, _P],
    "ms_dictionary_synthesis": [_P, _P, _P, _P],
    "ms_dictionary_analysis": [_P, _P, _P, _P],
    "ms_sigma2_hat": [_P, _P, ctypes.POINTER(_D), _P],
    "ms_lipschitz": [_P, _I32, _I32, _D, _D, _I32, ctypes.POINTER(_D), ctypes.POINTER(_D), _P],
    "ms_minor_cycle": [_P, _I32, _I32, _P, _P, _D, _D, _D, _I32, _D, _P, _P,
                       ctypes.POINTER(ms_stats), _P],
    "ms_reconstruct_two_step": [_P, _I32, _P, ctypes.POINTER(ms_recon_opts), _P, _P, _P,
                                ctypes.POINTER(ms_stats), _P],
    "ms_reconstruct_single_step": [_P, _I32, _P, ctypes.POINTER(ms_recon_opts), _P, _P,
                                   ctypes.POINTER(ms_stats), _P],
    "ms_unet_create": [_I32, _I32, _I32, ctypes.c_uint64, _I32, ctypes.POINTER(_P)],
    "ms_unet_destroy": [_P],
    "ms_unet_last_error": [_P],
    "ms_unet_param_count": [_P, ctypes.POINTER(_I64)],
    "ms_unet_get_params": [_P, _P, _I64],
    "ms_unet_set_params": [_P, _P, _I64],
    "ms_unet_forward": [_P, _P, _I32, _I32, _P, _P],
    "ms_unet_gradients": [_P, _P, _P, _I32, _I32, _P, _P, ctypes.POINTER(_D), _P],
    "ms_unet_train_step": [_P, _P, _P, _I32, _I32, ctypes.c_float, ctypes.POINTER(_D), _P],
    "ms_unet_keep_intermediates": [_P, _I32],
    "ms_unet_layer_tensor": [_P, _I32, _I32, _P, _I64],
    "ms_set_profiling": [_P, _I32],
    "ms_set_objective_target": [_P, _D],
    "ms_lambda": [_P, _I32, _D, _I32, _P, ctypes.POINTER(_D), _P],
    "ms_warm_start_coefficients": [_P, _P, _P, _P, _P, _P, _P],
    "ms_get_kernel_profile": [_P, ctypes.POINTER(ms_kernel_profile), _I32],
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmstep.so (built by ``_build.build``).  Raises if it is missing:
    the package has no other implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2406_18356_gb300._build.build()")
    lib = ctypes.CDLL(path)
    for name, args in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = (ctypes.c_char_p if name in ("ms_last_error", "ms_unet_last_error")
                      else ctypes.c_int)
    _lib = lib
    return lib


def exported_symbols() -> List[str]:
    return list(_SIGNATURES)


# ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _stream_handle(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


@dataclass
class Stats:
    iterations: int
    converged: bool
    major_cycles: int
    total_iterations: int
    objective: float
    lam: float
    theta: float
    sigma2: float
    eta2: float
    elapsed_ms: float
    grid_ms: float
    fft_ms: float
    minor_ms: float
    gridded_vis: int
    trace: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @classmethod
    def from_c(cls, s: ms_stats) -> "Stats":
        n = s.iterations + 1 if s.objective_trace else 0
        tr = np.array(s.objective_trace[:n]) if n else np.zeros(0)
        return cls(s.iterations, bool(s.converged), s.major_cycles, s.total_iterations,
                   s.objective, s.lambda_, s.theta, s.sigma2, s.eta2, s.elapsed_ms,
                   s.grid_ms, s.fft_ms, s.minor_ms, s.gridded_vis, tr)


@dataclass
class ReconOptions:
    n_major: int = 5
    fista_iters: int = 100
    rel_tol: float = 0.0
    lambda_rule: str = "norm2_2n"      # or "max_fixed"
    lambda_low: float = 0.05
    lambda_full: float = 0.05
    lambda_single: float = 0.01
    sigma2: float = 0.0                # <= 0: estimate (Sect. 4.3)
    eta2: float = 0.0                  # <= 0: 1e-3 sigma^2
    warm_start: Optional["WarmStartNet"] = None   # network for step two's first start

    def to_c(self) -> ms_recon_opts:
        rule = {"norm2_2n": MS_LAMBDA_NORM2_2N, "max_fixed": MS_LAMBDA_MAX_FIXED}[self.lambda_rule]
        net = self.warm_start._h if self.warm_start is not None else None
        return ms_recon_opts(self.n_major, self.fista_iters, self.rel_tol, rule, self.lambda_low,
                             self.lambda_full, self.lambda_single, self.sigma2, self.eta2, net)


class Plan:
    """Owns an ``ms_plan``.  See ``include/mstep.h`` for the semantics."""

    def __init__(self, u, v, npix: int, pixel_size: float, ell_px: float, delta_px: float,
                 flags=None, precision: str = "fp64", levels: int = 4, n_bases: int = 8,
                 kernel_width: int = 7, oversample: int = 2, es_beta: float = 0.0,
                 tile: int = 0, chunk: int = 0, device: int = 0,
                 dictionary: str = "daubechies", convolution: str = "circular"):
        lib = load_library()
        u = np.ascontiguousarray(np.atleast_2d(np.asarray(u, dtype=np.float64)))
        v = np.ascontiguousarray(np.atleast_2d(np.asarray(v, dtype=np.float64)))
        if u.shape != v.shape:
            raise ValueError("u and v must have the same shape")
        fl = None
        if flags is not None:
            fl = np.ascontiguousarray(np.atleast_2d(np.asarray(flags, dtype=np.uint8)))
            if fl.shape != u.shape:
                raise ValueError("flags must match u")
        self.nchan, self.nvis = u.shape
        self.npix = int(npix)
        self.precision = precision
        self.prec = PRECISIONS[precision]
        self.dictionary = dictionary
        # coefficient planes: M Daubechies bases, or J + 1 IUWT planes
        self.levels = levels
        self.n_bases = levels + 1 if dictionary == "iuwt" else n_bases
        self.device = device
        self.convolution = convolution
        d = ms_plan_desc(u.ctypes.data, v.ctypes.data, fl.ctypes.data if fl is not None else None,
                         self.nvis, self.nchan, self.npix, pixel_size, ell_px, delta_px,
                         kernel_width, oversample, es_beta, levels, n_bases, self.prec, tile,
                         chunk, device, DICTIONARIES[dictionary], CONVOLUTIONS[convolution])
        h = _P()
        st = lib.ms_plan_create(ctypes.byref(d), ctypes.byref(h))
        if st != MS_OK:
            raise MsError(st, "ms_plan_create failed (see stderr)")
        self._h = h
        self._lib = lib

    # -- helpers -------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.ms_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != MS_OK:
            msg = self._lib.ms_last_error(self._h)
            raise MsError(st, msg.decode() if msg else "")

    @property
    def real_dtype(self):
        torch = _torch()
        return torch.float64 if self.prec == MS_FP64 else torch.float32

    @property
    def complex_dtype(self):
        torch = _torch()
        return torch.complex128 if self.prec == MS_FP64 else torch.complex64

    def _dev(self):
        return _torch().device("cuda", self.device)

    def _need(self, t, dtype, numel, name):
        if t is None:
            raise ValueError(f"{name} is required")
        if not t.is_cuda or t.device.index != self.device:
            raise ValueError(f"{name} must be on cuda:{self.device}")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous() or t.numel() != numel:
            raise ValueError(f"{name} must be contiguous with {numel} elements")
        return t.data_ptr()

    def _image(self, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty((self.npix, self.npix), dtype=self.real_dtype, device=self._dev())
        return out

    # -- ABI -----------------------------------------------------------------
    def partition_counts(self, chan: int = 0):
        out = (_I64 * 4)()
        self._check(self._lib.ms_partition_counts(self._h, chan, out))
        return {"L": out[0], "H": out[1], "LH": out[2], "ALL": out[3]}

    def partition_layout(self, part: str, chan: int = 0):
        """(work items, cells per work-item tile, bytes per scratch cell)"""
        out = (_I64 * 3)()
        self._check(self._lib.ms_partition_layout(self._h, PARTS[part], chan, out))
        return int(out[0]), int(out[1]), int(out[2])

    def partition_rows(self, part: str, chan: int = 0) -> np.ndarray:
        n = self.partition_counts(chan)[part]
        rows = np.zeros(max(n, 1), dtype=np.int32)
        self._check(self._lib.ms_partition_rows(self._h, PARTS[part], chan, rows.ctypes.data))
        return rows[:n]

    def degrid(self, part: str, image, vis_obs=None, out=None, chan: int = 0, stream=None):
        torch = _torch()
        n2 = self.npix * self.npix
        if out is None:
            out = torch.zeros(self.nvis, dtype=self.complex_dtype, device=self._dev())
        self._check(self._lib.ms_degrid(
            self._h, PARTS[part], chan, self._need(image, self.real_dtype, n2, "image"),
            self._need(vis_obs, self.complex_dtype, self.nvis, "vis_obs") if vis_obs is not None else None,
            self._need(out, self.complex_dtype, self.nvis, "vis_out"), _stream_handle(stream)))
        return out

    def grid(self, part: str, vis, out=None, chan: int = 0, stream=None):
        out = self._image(out)
        self._check(self._lib.ms_grid(
            self._h, PARTS[part], chan, self._need(vis, self.complex_dtype, self.nvis, "vis"),
            self._need(out, self.real_dtype, self.npix ** 2, "dirty"), _stream_handle(stream)))
        return out

    def grid_static_scratch(self, part: str, vis, out, chan: int = 0, stream=None):
        """ms_grid with the gridding tiles in the library's fixed static
        scratch; `out` (N*N real, on the device) is required, so the call
        allocates nothing."""
        self._check(self._lib.ms_grid_static_scratch(
            self._h, PARTS[part], chan, self._need(vis, self.complex_dtype, self.nvis, "vis"),
            self._need(out, self.real_dtype, self.npix ** 2, "dirty"), _stream_handle(stream)))
        return out

    def _jobs(self, jobs):
        n = len(jobs)
        chans = (_I32 * n)(*[int(c) for c, _ in jobs])
        parts = (_I32 * n)(*[PARTS[p] for _, p in jobs])
        return n, chans, parts

    def grid_batch(self, jobs, vis, outs=None, stream=None):
        """jobs: [(chan, part)], vis: one dev complex [nvis] tensor per job
        (that channel's visibilities), outs: dirty images (allocated if None)."""
        n, chans, parts = self._jobs(jobs)
        if outs is None:
            outs = [self._image() for _ in range(n)]
        vp = (_P * n)(*[self._need(v, self.complex_dtype, self.nvis, "vis") for v in vis])
        op = (_P * n)(*[self._need(o, self.real_dtype, self.npix ** 2, "dirty") for o in outs])
        self._check(self._lib.ms_grid_batch(self._h, n, chans, parts, vp, op,
                                            _stream_handle(stream)))
        return outs

    def degrid_batch(self, jobs, images, vis_obs=None, outs=None, stream=None):
        """jobs: [(chan, part)], images: one dev N*N real tensor per job;
        vis_obs: None or one dev complex [nvis] tensor per job."""
        torch = _torch()
        n, chans, parts = self._jobs(jobs)
        if outs is None:
            outs = [torch.zeros(self.nvis, dtype=self.complex_dtype, device=self._dev())
                    for _ in range(n)]
        ip = (_P * n)(*[self._need(x, self.real_dtype, self.npix ** 2, "image") for x in images])
        op = (_P * n)(*[self._need(o, self.complex_dtype, self.nvis, "vis_out") for o in outs])
        ob = None
        if vis_obs is not None:
            ob = (_P * n)(*[self._need(v, self.complex_dtype, self.nvis, "vis_obs")
                            for v in vis_obs])
        self._check(self._lib.ms_degrid_batch(self._h, n, chans, parts, ip, ob, op,
                                              _stream_handle(stream)))
        return outs

    def residual_image(self, part: str, vis_obs, model, out=None, chan: int = 0, stream=None):
        out = self._image(out)
        n2 = self.npix ** 2
        self._check(self._lib.ms_residual_image(
            self._h, PARTS[part], chan, self._need(vis_obs, self.complex_dtype, self.nvis, "vis_obs"),
            self._need(model, self.real_dtype, n2, "model"),
            self._need(out, self.real_dtype, n2, "out"), _stream_handle(stream)))
        return out

    def psf(self, part: str, chan: int = 0, out=None, stream=None):
        out = self._image(out)
        self._check(self._lib.ms_psf(self._h, PARTS[part], chan,
                                     self._need(out, self.real_dtype, self.npix ** 2, "psf"),
                                     _stream_handle(stream)))
        return out

    def dictionary_synthesis(self, alpha, out=None, stream=None):
        out = self._image(out)
        n2 = self.npix ** 2
        self._check(self._lib.ms_dictionary_synthesis(
            self._h, self._need(alpha, self.real_dtype, self.n_bases * n2, "alpha"),
            self._need(out, self.real_dtype, n2, "x"), _stream_handle(stream)))
        return out

    def dictionary_analysis(self, x, out=None, stream=None):
        torch = _torch()
        n2 = self.npix ** 2
        if out is None:
            out = torch.empty((self.n_bases, self.npix, self.npix), dtype=self.real_dtype,
                              device=self._dev())
        self._check(self._lib.ms_dictionary_analysis(
            self._h, self._need(x, self.real_dtype, n2, "x"),
            self._need(out, self.real_dtype, self.n_bases * n2, "alpha"), _stream_handle(stream)))
        return out

    def sigma2_hat(self, image, stream=None) -> float:
        out = _D()
        self._check(self._lib.ms_sigma2_hat(self._h, self._need(image, self.real_dtype,
                                                                self.npix ** 2, "image"),
                                            ctypes.byref(out), _stream_handle(stream)))
        return out.value

    def lipschitz(self, step: str, chan: int = 0, sigma2: float = 0.0, eta2: float = 0.0,
                  power_iters: int = 0, stream=None):
        c, p = _D(), _D()
        self._check(self._lib.ms_lipschitz(self._h, STEPS[step], chan, sigma2, eta2, power_iters,
                                           ctypes.byref(c), ctypes.byref(p),
                                           _stream_handle(stream)))
        return c.value, p.value

    def minor_cycle(self, step: str, residual, lam: float, max_iters: int, l_low=None,
                    sigma2: float = 0.0, eta2: float = 0.0, rel_tol: float = 0.0,
                    beta=None, model_out=None, chan: int = 0, stream=None):
        n2 = self.npix ** 2
        model_out = self._image(model_out)
        st = ms_stats()
        self._check(self._lib.ms_minor_cycle(
            self._h, STEPS[step], chan, self._need(residual, self.real_dtype, n2, "residual"),
            self._need(l_low, self.real_dtype, n2, "l_low") if l_low is not None else None,
            sigma2, eta2, lam, max_iters, rel_tol,
            self._need(beta, self.real_dtype, self.n_bases * n2, "beta") if beta is not None else None,
            self._need(model_out, self.real_dtype, n2, "model_out"), ctypes.byref(st),
            _stream_handle(stream)))
        return model_out, Stats.from_c(st)

    def minor_cycle_batch(self, jobs, max_iters: int, rel_tol: float = 0.0, outs=None,
                          stream=None):
        """Batched minor cycles.  jobs: list of dicts with keys step ("low" /
        "full" / "single"), residual (dev N*N), lam, and for "full" l_low,
        sigma2, eta2; optional chan (0).  Returns (models, [Stats]) with each
        Stats' trace the job's F(beta_0..beta_K)."""
        n = len(jobs)
        n2 = self.npix ** 2
        if outs is None:
            outs = [self._image() for _ in range(n)]
        steps = (_I32 * n)(*[STEPS[j["step"]] for j in jobs])
        chans = (_I32 * n)(*[int(j.get("chan", 0)) for j in jobs])
        res = (_P * n)(*[self._need(j["residual"], self.real_dtype, n2, "residual") for j in jobs])
        lows = (_P * n)(*[self._need(j["l_low"], self.real_dtype, n2, "l_low")
                          if j["step"] == "full" else None for j in jobs])
        lams = (_D * n)(*[float(j["lam"]) for j in jobs])
        s2 = (_D * n)(*[float(j.get("sigma2", 0.0)) for j in jobs])
        e2 = (_D * n)(*[float(j.get("eta2", 0.0)) for j in jobs])
        op = (_P * n)(*[self._need(o, self.real_dtype, n2, "model_out") for o in outs])
        st = (ms_stats * n)()
        traces = np.full((n, max_iters + 1), np.nan)
        self._check(self._lib.ms_minor_cycle_batch(
            self._h, n, steps, chans, res, lows, lams, s2, e2, max_iters, rel_tol, op, st,
            traces.ctypes.data_as(ctypes.POINTER(_D)), _stream_handle(stream)))
        stats = []
        for j in range(n):
            s = Stats.from_c(st[j])
            s.trace = traces[j, :st[j].iterations + 1].copy()
            stats.append(s)
        return outs, stats

    def _recon_batch(self, two: bool, vis, opts, chans, low_outs, outs, stream):
        opts = opts or ReconOptions()
        n = len(vis)
        chans = list(range(n)) if chans is None else list(chans)
        n2 = self.npix ** 2
        outs = outs if outs is not None else [self._image() for _ in range(n)]
        ch = (_I32 * n)(*chans)
        vp = (_P * n)(*[self._need(v, self.complex_dtype, self.nvis, "vis") for v in vis])
        op = (_P * n)(*[self._need(o, self.real_dtype, n2, "img_out") for o in outs])
        st = (ms_stats * n)()
        co = opts.to_c()
        if two:
            low_outs = low_outs if low_outs is not None else [self._image() for _ in range(n)]
            lp = (_P * n)(*[self._need(o, self.real_dtype, n2, "low_out") for o in low_outs])
            self._check(self._lib.ms_reconstruct_two_step_batch(
                self._h, n, ch, vp, ctypes.byref(co), lp, op, st, _stream_handle(stream)))
        else:
            self._check(self._lib.ms_reconstruct_single_step_batch(
                self._h, n, ch, vp, ctypes.byref(co), op, st, _stream_handle(stream)))
        return low_outs if two else None, outs, [Stats.from_c(st[j]) for j in range(n)]

    def reconstruct_two_step_batch(self, vis, opts: Optional[ReconOptions] = None, chans=None,
                                   low_outs=None, outs=None, stream=None):
        """The two-step method on several channels at once: vis[j] is channel
        chans[j]'s visibilities (default chans = 0..len(vis)-1).  Returns
        (low images, final images, [Stats])."""
        return self._recon_batch(True, vis, opts, chans, low_outs, outs, stream)

    def reconstruct_single_step_batch(self, vis, opts: Optional[ReconOptions] = None,
                                      chans=None, outs=None, stream=None):
        _, outs, st = self._recon_batch(False, vis, opts, chans, None, outs, stream)
        return outs, st

    def reconstruct_step(self, step: str, vis, opts: Optional[ReconOptions] = None,
                         low_image=None, chan: int = 0, out=None, model_out=None, stream=None):
        """One step of the method (ms_reconstruct_step): returns (image, Stats)."""
        opts = opts or ReconOptions()
        out = self._image(out)
        co = opts.to_c()
        st = ms_stats()
        n2 = self.npix ** 2
        self._check(self._lib.ms_reconstruct_step(
            self._h, STEPS[step], chan, self._need(vis, self.complex_dtype, self.nvis, "vis"),
            ctypes.byref(co),
            self._need(low_image, self.real_dtype, n2, "low_image") if low_image is not None else None,
            self._need(out, self.real_dtype, n2, "img_out"),
            self._need(model_out, self.real_dtype, n2, "model_out") if model_out is not None else None,
            ctypes.byref(st), _stream_handle(stream)))
        return out, Stats.from_c(st)

    def reconstruct_interleaved(self, vis, opts: Optional[ReconOptions] = None, chan: int = 0,
                                out=None, node_l=None, node_h=None, stream=None):
        """The interleaved two-image pipeline (ms_reconstruct_interleaved):
        returns (combined image, node L's image, node H's image,
        [Stats of node L, Stats of node H])."""
        opts = opts or ReconOptions()
        out, node_l, node_h = self._image(out), self._image(node_l), self._image(node_h)
        co = opts.to_c()
        st = (ms_stats * 2)()
        n2 = self.npix ** 2
        self._check(self._lib.ms_reconstruct_interleaved(
            self._h, chan, self._need(vis, self.complex_dtype, self.nvis, "vis"), ctypes.byref(co),
            self._need(out, self.real_dtype, n2, "img_out"),
            self._need(node_l, self.real_dtype, n2, "node_l_out"),
            self._need(node_h, self.real_dtype, n2, "node_h_out"), st, _stream_handle(stream)))
        return out, node_l, node_h, [Stats.from_c(st[0]), Stats.from_c(st[1])]

    def reconstruct_two_step(self, vis, opts: Optional[ReconOptions] = None, chan: int = 0,
                             low_out=None, out=None, model_out=None, stream=None):
        opts = opts or ReconOptions()
        low_out, out = self._image(low_out), self._image(out)
        co = opts.to_c()
        st = ms_stats()
        n2 = self.npix ** 2
        self._check(self._lib.ms_reconstruct_two_step(
            self._h, chan, self._need(vis, self.complex_dtype, self.nvis, "vis"), ctypes.byref(co),
            self._need(low_out, self.real_dtype, n2, "img_low_out"),
            self._need(out, self.real_dtype, n2, "img_out"),
            self._need(model_out, self.real_dtype, n2, "model_out") if model_out is not None else None,
            ctypes.byref(st), _stream_handle(stream)))
        return low_out, out, Stats.from_c(st)

    def reconstruct_single_step(self, vis, opts: Optional[ReconOptions] = None, chan: int = 0,
                                out=None, model_out=None, stream=None):
        opts = opts or ReconOptions()
        out = self._image(out)
        co = opts.to_c()
        st = ms_stats()
        n2 = self.npix ** 2
        self._check(self._lib.ms_reconstruct_single_step(
            self._h, chan, self._need(vis, self.complex_dtype, self.nvis, "vis"), ctypes.byref(co),
            self._need(out, self.real_dtype, n2, "img_out"),
            self._need(model_out, self.real_dtype, n2, "model_out") if model_out is not None else None,
            ctypes.byref(st), _stream_handle(stream)))
        return out, Stats.from_c(st)


    def set_profiling(self, on: bool):
        self._check(self._lib.ms_set_profiling(self._h, 1 if on else 0))

    def lam(self, residual, coef: float = 0.05, n: int = 1, rule: str = "norm2_2n",
            stream=None) -> float:
        """lambda of major cycle n from its residual image (ms_lambda)."""
        r = {"norm2_2n": MS_LAMBDA_NORM2_2N, "max_fixed": MS_LAMBDA_MAX_FIXED}[rule]
        out = _D()
        self._check(self._lib.ms_lambda(
            self._h, r, float(coef), int(n),
            self._need(residual, self.real_dtype, self.npix ** 2, "residual"),
            ctypes.byref(out), _stream_handle(stream)))
        return float(out.value)

    def warm_start_coefficients(self, net: "WarmStartNet", low_image, residual_h1,
                                beta_out=None, x0_out=None, stream=None):
        """(beta, x0): W^H x0 / M with x0 the network's start of step two."""
        torch = _torch()
        n2 = self.npix ** 2
        if beta_out is None:
            beta_out = torch.empty((self.n_bases, self.npix, self.npix), dtype=self.real_dtype,
                                   device=low_image.device)
        if x0_out is None:
            x0_out = self._image(None)
        self._check(self._lib.ms_warm_start_coefficients(
            self._h, net._h, self._need(low_image, self.real_dtype, n2, "low_image"),
            self._need(residual_h1, self.real_dtype, n2, "residual_h1"),
            self._need(beta_out, self.real_dtype, self.n_bases * n2, "beta_out"),
            self._need(x0_out, self.real_dtype, n2, "x0_out"), _stream_handle(stream)))
        return beta_out, x0_out

    def set_objective_target(self, target: float = float("-inf")):
        """Later minor cycles also stop once F(beta_k) <= target (-inf: off)."""
        self._check(self._lib.ms_set_objective_target(self._h, float(target)))

    def kernel_profile(self, reset: bool = False) -> dict:
        """{family: (timed launch groups, total ms)} from CUDA events."""
        out = ms_kernel_profile()
        self._check(self._lib.ms_get_kernel_profile(self._h, ctypes.byref(out), 1 if reset else 0))
        return {name: (out.launches[i], out.total_ms[i]) for i, name in enumerate(KERNEL_FAMILIES)}


# module-level names matching the C ABI -------------------------------------
def ms_plan_create(*args, **kw) -> Plan:
    return Plan(*args, **kw)


def ms_plan_destroy(plan: Plan):
    plan.close()


def ms_partition_counts(plan: Plan, chan: int = 0):
    return plan.partition_counts(chan)


def ms_partition_layout(plan: Plan, part: str, chan: int = 0):
    return plan.partition_layout(part, chan)


def ms_partition_rows(plan: Plan, part: str, chan: int = 0):
    return plan.partition_rows(part, chan)


def ms_degrid(plan: Plan, part, image, vis_obs=None, out=None, chan=0, stream=None):
    return plan.degrid(part, image, vis_obs, out, chan, stream)


def ms_grid(plan: Plan, part, vis, out=None, chan=0, stream=None):
    return plan.grid(part, vis, out, chan, stream)


def ms_grid_static_scratch(plan: Plan, part, vis, out, chan=0, stream=None):
    return plan.grid_static_scratch(part, vis, out, chan, stream)


def ms_grid_batch(plan: Plan, jobs, vis, outs=None, stream=None):
    return plan.grid_batch(jobs, vis, outs, stream)


def ms_degrid_batch(plan: Plan, jobs, images, vis_obs=None, outs=None, stream=None):
    return plan.degrid_batch(jobs, images, vis_obs, outs, stream)


def ms_reconstruct_interleaved(plan: Plan, vis, opts=None, chan: int = 0, stream=None):
    return plan.reconstruct_interleaved(vis, opts, chan, stream=stream)


def ms_minor_cycle_batch(plan: Plan, jobs, max_iters: int, rel_tol: float = 0.0, outs=None,
                         stream=None):
    return plan.minor_cycle_batch(jobs, max_iters, rel_tol, outs, stream)


def ms_reconstruct_two_step_batch(plan: Plan, vis, opts=None, chans=None, low_outs=None,
                                  outs=None, stream=None):
    return plan.reconstruct_two_step_batch(vis, opts, chans, low_outs, outs, stream)


def ms_reconstruct_single_step_batch(plan: Plan, vis, opts=None, chans=None, outs=None,
                                     stream=None):
    return plan.reconstruct_single_step_batch(vis, opts, chans, outs, stream)


def ms_plan_autotune(u, v, npix: int, pixel_size: float, ell_px: float, delta_px: float,
                     flags=None, precision: str = "fp32", levels: int = 4, n_bases: int = 8,
                     chan: int = 0, reps: int = 3, device: int = 0):
    """Fastest (tile, chunk) of the gridding layout for these rows on this GPU,
    and its degrid + grid time in ms (see ms_plan_autotune in mstep.h)."""
    lib = load_library()
    u = np.ascontiguousarray(np.atleast_2d(np.asarray(u, dtype=np.float64)))
    v = np.ascontiguousarray(np.atleast_2d(np.asarray(v, dtype=np.float64)))
    fl = None
    if flags is not None:
        fl = np.ascontiguousarray(np.atleast_2d(np.asarray(flags, dtype=np.uint8)))
    d = ms_plan_desc(u.ctypes.data, v.ctypes.data, fl.ctypes.data if fl is not None else None,
                     u.shape[1], u.shape[0], int(npix), pixel_size, ell_px, delta_px, 7, 2, 0.0,
                     levels, n_bases, PRECISIONS[precision], 0, 0, device)
    t, c, ms_ = _I32(), _I32(), _D()
    st = lib.ms_plan_autotune(ctypes.byref(d), chan, reps, ctypes.byref(t), ctypes.byref(c),
                              ctypes.byref(ms_))
    if st != MS_OK:
        raise MsError(st, "ms_plan_autotune failed")
    return int(t.value), int(c.value), float(ms_.value)


def ms_residual_image(plan: Plan, part, vis_obs, model, out=None, chan=0, stream=None):
    return plan.residual_image(part, vis_obs, model, out, chan, stream)


def ms_psf(plan: Plan, part, chan=0, out=None, stream=None):
    return plan.psf(part, chan, out, stream)


def ms_dictionary_synthesis(plan: Plan, alpha, out=None, stream=None):
    return plan.dictionary_synthesis(alpha, out, stream)


def ms_dictionary_analysis(plan: Plan, x, out=None, stream=None):
    return plan.dictionary_analysis(x, out, stream)


def ms_sigma2_hat(plan: Plan, image, stream=None):
    return plan.sigma2_hat(image, stream)


def ms_lipschitz(plan: Plan, step, chan=0, sigma2=0.0, eta2=0.0, power_iters=0, stream=None):
    return plan.lipschitz(step, chan, sigma2, eta2, power_iters, stream)


def ms_minor_cycle(plan: Plan, step, residual, lam, max_iters, **kw):
    return plan.minor_cycle(step, residual, lam, max_iters, **kw)


def ms_reconstruct_two_step(plan: Plan, vis, opts=None, **kw):
    return plan.reconstruct_two_step(vis, opts, **kw)


def ms_reconstruct_single_step(plan: Plan, vis, opts=None, **kw):
    return plan.reconstruct_single_step(vis, opts, **kw)


def ms_set_profiling(plan: Plan, on: bool):
    plan.set_profiling(on)


def ms_lambda(plan: Plan, residual, coef=0.05, n=1, rule="norm2_2n", stream=None):
    return plan.lam(residual, coef, n, rule, stream)


def ms_warm_start_coefficients(plan: Plan, net, low_image, residual_h1, beta_out=None,
                               x0_out=None, stream=None):
    return plan.warm_start_coefficients(net, low_image, residual_h1, beta_out, x0_out, stream)


def ms_set_objective_target(plan: Plan, target: float):
    plan.set_objective_target(target)


def ms_get_kernel_profile(plan: Plan, reset: bool = False):
    return plan.kernel_profile(reset)


class WarmStartNet:
    """Owns an ``ms_unet`` (the learned warm start; see mstep.h).  Images are
    FP32 CUDA tensors, channels last: input [H, W, 2], output [H, W]."""

    def __init__(self, levels: int = 3, width: int = 16, max_side: int = 1024,
                 seed: int = 0, device: int = 0):
        self._lib = load_library()
        h = _P()
        st = self._lib.ms_unet_create(levels, width, max_side, seed, device, ctypes.byref(h))
        if st != MS_OK:
            raise MsError(st, "ms_unet_create failed")
        self._h = h
        self.levels, self.width, self.max_side, self.device = levels, width, max_side, device

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ms_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != MS_OK:
            msg = self._lib.ms_unet_last_error(self._h)
            raise MsError(st, msg.decode() if msg else "")

    def _t(self, t, shape, name):
        torch = _torch()
        if t is None or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() \
                or tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of shape {shape}")
        return t.data_ptr()

    def param_count(self) -> int:
        n = _I64()
        self._check(self._lib.ms_unet_param_count(self._h, ctypes.byref(n)))
        return int(n.value)

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count(), np.float32)
        self._check(self._lib.ms_unet_get_params(self._h, out.ctypes.data, out.size))
        return out

    def set_params(self, params) -> None:
        p = np.ascontiguousarray(np.asarray(params, np.float32))
        self._check(self._lib.ms_unet_set_params(self._h, p.ctypes.data, p.size))

    def forward(self, x, out=None, stream=None):
        torch = _torch()
        H, W = x.shape[0], x.shape[1]
        if out is None:
            out = torch.empty((H, W), dtype=torch.float32, device=x.device)
        self._check(self._lib.ms_unet_forward(self._h, self._t(x, (H, W, 2), "in"), H, W,
                                              self._t(out, (H, W), "out"),
                                              _stream_handle(stream)))
        return out

    def gradients(self, x, target, stream=None):
        """(output, loss, flat gradient array) for checking."""
        torch = _torch()
        H, W = x.shape[0], x.shape[1]
        out = torch.empty((H, W), dtype=torch.float32, device=x.device)
        g = np.zeros(self.param_count(), np.float32)
        loss = _D()
        self._check(self._lib.ms_unet_gradients(
            self._h, self._t(x, (H, W, 2), "in"), self._t(target, (H, W), "target"), H, W,
            out.data_ptr(), g.ctypes.data, ctypes.byref(loss), _stream_handle(stream)))
        return out, float(loss.value), g

    def keep_intermediates(self, keep: bool = True) -> None:
        """Keep every layer's pre-activation gradient in later gradients()
        calls (a checking aid)."""
        self._check(self._lib.ms_unet_keep_intermediates(self._h, 1 if keep else 0))

    def layer_tensor(self, layer: int, which: str, shape) -> np.ndarray:
        """A layer's stored bfloat16 input ('in'), output ('out') or kept
        pre-activation gradient ('grad') of the last pass, as FP32 [H_l, W_l, c]."""
        code = {"in": 0, "out": 1, "grad": 2}[which]
        out = np.zeros(shape, np.float32)
        self._check(self._lib.ms_unet_layer_tensor(self._h, layer, code, out.ctypes.data,
                                                   out.size))
        return out

    def train_step(self, x, target, lr: float, stream=None) -> float:
        H, W = x.shape[0], x.shape[1]
        loss = _D()
        self._check(self._lib.ms_unet_train_step(
            self._h, self._t(x, (H, W, 2), "in"), self._t(target, (H, W), "target"), H, W,
            ctypes.c_float(lr), ctypes.byref(loss), _stream_handle(stream)))
        return float(loss.value)


def ms_unet_create(levels=3, width=16, max_side=1024, seed=0, device=0):
    return WarmStartNet(levels, width, max_side, seed, device)


def ms_unet_destroy(net: WarmStartNet):
    net.close()


def ms_unet_last_error(net: WarmStartNet):
    msg = net._lib.ms_unet_last_error(net._h)
    return msg.decode() if msg else ""


def ms_unet_param_count(net: WarmStartNet):
    return net.param_count()


def ms_unet_get_params(net: WarmStartNet):
    return net.get_params()


def ms_unet_set_params(net: WarmStartNet, params):
    net.set_params(params)


def ms_unet_forward(net: WarmStartNet, x, out=None, stream=None):
    return net.forward(x, out, stream)


def ms_unet_gradients(net: WarmStartNet, x, target, stream=None):
    return net.gradients(x, target, stream)


def ms_unet_train_step(net: WarmStartNet, x, target, lr, stream=None):
    return net.train_step(x, target, lr, stream)


def ms_unet_keep_intermediates(net: WarmStartNet, keep=True):
    net.keep_intermediates(keep)


def ms_unet_layer_tensor(net: WarmStartNet, layer, which, shape):
    return net.layer_tensor(layer, which, shape)
