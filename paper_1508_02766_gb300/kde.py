"""Thin Python binding of the C ABI in include/kde_gb300.h.

Argument marshalling only: every step of the estimator runs in the CUDA
library.  Tensors are PyTorch device tensors (their data pointers are passed
through); streams are the current PyTorch CUDA stream unless one is given.
The library must be built (``build.build()``); loading fails loudly if it is
missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

F32, F64 = 0, 1
RANGE_CORRECTED, RANGE_PER_AXIS = 0, 1
LAYOUT_CORRECTED, LAYOUT_WAND = 0, 1
MAX_D, MAX_STAGES = 3, 16

_STATUS = {0: "KDE_OK", 1: "KDE_ERR_INVALID_ARG", 2: "KDE_ERR_NOT_SPD", 4: "KDE_ERR_WORKSPACE",
           5: "KDE_ERR_CUDA", 7: "KDE_ERR_UNSUPPORTED"}


class KDEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("precision", ctypes.c_int),
                ("range_mode", ctypes.c_int), ("layout_mode", ctypes.c_int),
                ("P_min", ctypes.c_int64 * MAX_D), ("cols_variant", ctypes.c_int),
                ("dft_tc", ctypes.c_int), ("engine", ctypes.c_int), ("slab_passes", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("precision", ctypes.c_int),
                ("M", ctypes.c_int64 * MAX_D), ("L", ctypes.c_int64 * MAX_D),
                ("P", ctypes.c_int64 * MAX_D), ("Q", ctypes.c_int64),
                ("delta", ctypes.c_double * MAX_D), ("lambda_max", ctypes.c_double),
                ("det_H", ctypes.c_double), ("kspec_elems", ctypes.c_int64),
                ("kspec_bytes", ctypes.c_size_t), ("workspace_bytes", ctypes.c_size_t),
                ("nstages", ctypes.c_int * MAX_D),
                ("radix", (ctypes.c_int * MAX_STAGES) * MAX_D), ("engine", ctypes.c_int),
                ("split", (ctypes.c_int * 3) * MAX_D), ("slab_passes", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64 * 2), ("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
                ("H", ctypes.c_double * 4), ("n", ctypes.c_int64)]


EXPORTS = [
    "kde_plan_info_compute", "kde_plan_create", "kde_plan_get_info", "kde_plan_destroy",
    "kde_bin", "kde_kernel_grid", "kde_fft_eval", "kde_status_string", "kde_last_error",
    "kde_launch_count", "kde_profile_enable", "kde_profile_count", "kde_profile_entry",
    "kde_fft_eval_noalloc", "kde_bin_workspace_bytes", "kde_power_spectrum", "kde_lscv",
    "kde_lscv_workspace_bytes", "kde_batch_plan_create", "kde_batch_plan_query",
    "kde_batch_set_shape", "kde_batch_get_shape", "kde_batch_tune", "kde_batch_eval",
    "kde_batch_plan_destroy", "kde_standardize2", "kde_features2", "kde_mlp_create",
    "kde_mlp_destroy", "kde_mlp_param_count", "kde_mlp_get_params", "kde_mlp_set_params",
    "kde_mlp_get_state", "kde_mlp_set_state", "kde_mlp_forward", "kde_mlp_loss_grad",
    "kde_mlp_train_step", "kde_mlp_status", "kde_gemm_bf16", "kde_autocorrelation",
    "kde_lscv_autocorr", "kde_lscv_autocorr_workspace_bytes", "kde_lscv_autocorr_batch",
    "kde_lscv_cands_create", "kde_lscv_cands_destroy", "kde_lscv_autocorr_cands",
    "kde_wait_probe", "kde_plan_check", "kde_outside_check", "kde_noalloc_scratch_bytes",
    "kde_fft_eval_multi", "kde_fft_eval_multi_workspace_bytes", "kde_batch_set_mode",
    "kde_batch_get_mode", "kde_batch_check", "kde_batch_set_wait", "kde_batch_get_config",
    "kde_batch_set_queue_order", "kde_debug_status", "kde_prepare2_batch",
    "kde_prepare2_batch_workspace_bytes", "kde_lscv_autocorr_cands_batch",
    "kde_lscv_autocorr_cands_batch_workspace_bytes", "kde_lscv_theta_select",
    "kde_lscv_theta_select_workspace_bytes", "kde_mlp_status_copy", "kde_bin_accumulate",
    "kde_fft_eval_consume",
]
FEAT_DIM = 1088

_lib = None


def lib():
    """Load libkde_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"{_build.LIB} is missing: run paper_1508_02766_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB)
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.kde_plan_info_compute.argtypes = [ctypes.c_int, i64p, dp, dp, dp, ctypes.POINTER(Opts),
                                        ctypes.POINTER(PlanInfo)]
    L.kde_plan_create.argtypes = [ctypes.c_int, i64p, dp, dp, dp, ctypes.POINTER(Opts),
                                  ctypes.POINTER(vp)]
    L.kde_plan_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    L.kde_plan_destroy.argtypes = [vp]
    L.kde_bin.argtypes = [vp, ctypes.c_int, i64, ctypes.c_int, dp, dp, i64p, vp, vp, vp,
                          ctypes.c_size_t, vp]
    L.kde_bin_accumulate.argtypes = L.kde_bin.argtypes
    L.kde_bin_workspace_bytes.argtypes = [i64, ctypes.c_int, i64p, ctypes.POINTER(ctypes.c_size_t)]
    L.kde_kernel_grid.argtypes = [vp, i64, vp, vp, ctypes.c_size_t, vp]
    L.kde_fft_eval.argtypes = [vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    L.kde_fft_eval_consume.argtypes = L.kde_fft_eval.argtypes
    L.kde_fft_eval_noalloc.argtypes = [vp, vp, vp, vp, vp]
    L.kde_power_spectrum.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, vp]
    L.kde_lscv.argtypes = [vp, i64, ctypes.c_int, dp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    L.kde_lscv_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.kde_batch_plan_create.argtypes = [ctypes.c_int, ctypes.POINTER(BatchItem), ctypes.POINTER(Opts),
                                        ctypes.POINTER(vp)]
    L.kde_batch_plan_query.argtypes = [vp, i64p, i64p, ctypes.POINTER(ctypes.c_size_t)]
    L.kde_batch_set_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.kde_batch_get_shape.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.kde_batch_tune.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, vp, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_float)]
    L.kde_batch_eval.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, vp]
    L.kde_batch_plan_destroy.argtypes = [vp]
    L.kde_lscv_autocorr_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.kde_autocorrelation.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, vp]
    L.kde_lscv_autocorr.argtypes = [vp, i64, ctypes.c_int, dp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    fp = ctypes.POINTER(ctypes.c_float)
    L.kde_standardize2.argtypes = [vp, i64, vp, vp, vp]
    L.kde_features2.argtypes = [vp, ctypes.c_int, i64, vp, vp, vp]
    L.kde_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_uint64, ctypes.POINTER(vp)]
    L.kde_mlp_destroy.argtypes = [vp]
    L.kde_mlp_param_count.argtypes = [vp, i64p]
    L.kde_mlp_get_params.argtypes = [vp, fp, i64]
    L.kde_mlp_set_params.argtypes = [vp, fp, i64]
    L.kde_mlp_get_state.argtypes = [vp, fp, fp, i64p]
    L.kde_mlp_set_state.argtypes = [vp, fp, fp, i64]
    L.kde_mlp_forward.argtypes = [vp, vp, ctypes.c_int, vp, vp]
    L.kde_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp, vp]
    L.kde_mlp_train_step.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_float, vp, vp]
    L.kde_mlp_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.kde_mlp_status_copy.argtypes = [vp, vp, vp]
    L.kde_gemm_bf16.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp,
                                ctypes.c_int, vp, ctypes.c_int, vp, vp]
    L.kde_fft_eval_multi.argtypes = [vp, i64, ctypes.c_int, dp, vp, vp, vp, ctypes.c_size_t, vp]
    L.kde_fft_eval_multi_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.kde_debug_status.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.kde_batch_set_mode.argtypes = [vp, ctypes.c_int]
    L.kde_batch_set_queue_order.argtypes = [vp, ctypes.c_int]
    L.kde_batch_get_mode.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.kde_batch_check.argtypes = [vp, vp]
    L.kde_batch_set_wait.argtypes = [vp, ctypes.c_uint32, ctypes.c_int]
    L.kde_batch_get_config.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       i64p]
    L.kde_prepare2_batch.argtypes = [vp, ctypes.c_int, vp, i64p, vp, vp, vp, vp, vp,
                                     ctypes.c_size_t, vp]
    L.kde_prepare2_batch_workspace_bytes.argtypes = [vp, ctypes.c_int, i64,
                                                     ctypes.POINTER(ctypes.c_size_t)]
    L.kde_lscv_autocorr_cands_batch.argtypes = [vp, ctypes.c_int, i64p, vp, vp, vp, vp,
                                                ctypes.c_size_t, vp]
    L.kde_lscv_autocorr_cands_batch_workspace_bytes.argtypes = [vp, ctypes.c_int,
                                                                ctypes.POINTER(ctypes.c_size_t)]
    L.kde_lscv_theta_select.argtypes = [vp, ctypes.c_int, i64p, vp, dp, ctypes.c_int, dp, dp, vp,
                                        vp, vp, vp, ctypes.c_size_t, vp]
    L.kde_lscv_theta_select_workspace_bytes.argtypes = [vp, ctypes.c_int, ctypes.c_int,
                                                        ctypes.POINTER(ctypes.c_size_t)]
    L.kde_plan_check.argtypes = [vp, vp]
    L.kde_outside_check.argtypes = [vp, vp, i64p]
    L.kde_noalloc_scratch_bytes.argtypes = []
    L.kde_noalloc_scratch_bytes.restype = ctypes.c_size_t
    L.kde_status_string.restype = ctypes.c_char_p
    L.kde_status_string.argtypes = [ctypes.c_int]
    L.kde_last_error.restype = ctypes.c_char_p
    L.kde_launch_count.restype = i64
    L.kde_profile_enable.argtypes = [ctypes.c_int]
    L.kde_profile_entry.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                    dp, i64p]
    for name in ("kde_plan_info_compute", "kde_plan_create", "kde_plan_get_info",
                 "kde_plan_destroy", "kde_bin", "kde_kernel_grid", "kde_fft_eval",
                 "kde_fft_eval_noalloc", "kde_profile_enable", "kde_profile_entry",
                 "kde_bin_workspace_bytes", "kde_power_spectrum", "kde_lscv",
                 "kde_lscv_workspace_bytes", "kde_batch_plan_create", "kde_batch_plan_query",
                 "kde_batch_set_shape", "kde_batch_get_shape", "kde_batch_tune", "kde_batch_eval",
                 "kde_batch_plan_destroy", "kde_standardize2", "kde_features2",
                 "kde_mlp_create", "kde_mlp_destroy", "kde_mlp_param_count",
                 "kde_mlp_get_params", "kde_mlp_set_params", "kde_mlp_get_state",
                 "kde_mlp_set_state", "kde_mlp_forward", "kde_mlp_loss_grad",
                 "kde_mlp_train_step", "kde_mlp_status", "kde_gemm_bf16",
                 "kde_autocorrelation", "kde_lscv_autocorr", "kde_lscv_autocorr_workspace_bytes",
                 "kde_lscv_autocorr_batch", "kde_lscv_cands_create", "kde_lscv_cands_destroy",
                 "kde_lscv_autocorr_cands", "kde_wait_probe", "kde_plan_check",
                 "kde_outside_check", "kde_fft_eval_multi", "kde_fft_eval_multi_workspace_bytes",
                 "kde_batch_set_mode", "kde_batch_get_mode", "kde_batch_check", "kde_batch_set_wait",
                 "kde_batch_get_config", "kde_batch_set_queue_order", "kde_debug_status",
                 "kde_prepare2_batch", "kde_prepare2_batch_workspace_bytes",
                 "kde_lscv_autocorr_cands_batch",
                 "kde_lscv_autocorr_cands_batch_workspace_bytes", "kde_lscv_theta_select",
                 "kde_lscv_theta_select_workspace_bytes", "kde_mlp_status_copy",
                 "kde_bin_accumulate", "kde_fft_eval_consume"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise KDEError(status, lib().kde_last_error().decode())


def _darr(vals, n=None):
    vals = [float(v) for v in np.asarray(vals, dtype=np.float64).ravel()]
    return (ctypes.c_double * len(vals))(*vals)


def _iarr(vals):
    vals = [int(v) for v in vals]
    return (ctypes.c_int64 * len(vals))(*vals)


COLS_VARIANTS = {"auto": 0, "lines": 1, "simd": 2}
ENGINES = {"auto": 0, "stockham": 1, "two_phase": 2}
SLAB_PASSES = {"off": 0, "on": 1}


def _opts(tau=3.7, precision="f32", range_mode="corrected", layout="corrected", P_min=None,
          cols="auto", dft="fft", engine="auto", slab="off"):
    o = Opts()
    o.cols_variant = COLS_VARIANTS[cols]
    o.engine = ENGINES[engine]
    o.slab_passes = SLAB_PASSES[slab]
    o.dft_tc = {"fft": 0, "tc": 1}[dft]
    o.tau = tau
    o.precision = F32 if precision == "f32" else F64
    o.range_mode = RANGE_CORRECTED if range_mode == "corrected" else RANGE_PER_AXIS
    o.layout_mode = LAYOUT_CORRECTED if layout == "corrected" else LAYOUT_WAND
    for k, p in enumerate(P_min or []):
        o.P_min[k] = int(p)
    return o


@dataclass
class Info:
    d: int
    precision: str
    M: tuple
    L: tuple
    P: tuple
    Q: int
    delta: tuple
    lambda_max: float
    det_H: float
    kspec_elems: int
    kspec_bytes: int
    workspace_bytes: int
    radices: tuple
    engine: str
    split: tuple
    slab_passes: bool


def _info(pi: PlanInfo) -> Info:
    d = pi.d
    return Info(d, "f32" if pi.precision == F32 else "f64", tuple(pi.M[:d]), tuple(pi.L[:d]),
                tuple(pi.P[:d]), pi.Q, tuple(pi.delta[:d]), pi.lambda_max, pi.det_H,
                pi.kspec_elems, pi.kspec_bytes, pi.workspace_bytes,
                tuple(tuple(pi.radix[k][:pi.nstages[k]]) for k in range(d)),
                {1: "stockham", 2: "two_phase"}.get(pi.engine, "stockham"),
                tuple(tuple(v for v in pi.split[k][:3] if v) or (0, 0) for k in range(d)),
                bool(pi.slab_passes))


def kde_plan_info_compute(M, lo, hi, H, **opts) -> Info:
    """Host-only planning (Eq. 4, Eq. 15, padded sizes); needs no GPU."""
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    pi = PlanInfo()
    o = _opts(**opts)
    _check(lib().kde_plan_info_compute(d, _iarr(M), _darr(lo), _darr(hi), _darr(H),
                                       ctypes.byref(o), ctypes.byref(pi)))
    return _info(pi)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Plan:
    """kde_plan_create / kde_plan_destroy; the plan owns its twiddle tables."""

    def __init__(self, M, lo, hi, H, **opts):
        H = np.asarray(H, dtype=np.float64)
        self.d = H.shape[0]
        self.M = tuple(int(m) for m in M)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        h = ctypes.c_void_p()
        o = _opts(**opts)
        _check(lib().kde_plan_create(self.d, _iarr(M), _darr(lo), _darr(hi), _darr(H),
                                     ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        pi = PlanInfo()
        _check(lib().kde_plan_get_info(h, ctypes.byref(pi)))
        self.info = _info(pi)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().kde_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def real_dtype(self):
        import torch
        return torch.float32 if self.info.precision == "f32" else torch.float64

    def workspace(self, device="cuda"):
        import torch
        nbytes = max(16, self.info.workspace_bytes)
        return torch.empty(nbytes, dtype=torch.uint8, device=device)


def kde_bin_workspace_bytes(n, d, M) -> int:
    """Scratch bytes of the tiled binning method (host only)."""
    b = ctypes.c_size_t()
    _check(lib().kde_bin_workspace_bytes(int(n), int(d), _iarr(M), ctypes.byref(b)))
    return int(b.value)


def bin_workspace(n, d, M, device="cuda"):
    import torch
    return torch.empty(max(256, kde_bin_workspace_bytes(n, d, M)), dtype=torch.uint8, device=device)


def kde_bin(X, lo, hi, M, counts=None, n_outside=None, workspace=None, method="auto",
            stream=None, accumulate=False):
    """Linear binning into int64 counts (units 2^-32).  X: (n, d) float32/float64
    CUDA tensor, or a pinned host tensor that the kernels read in place.
    method "direct" (global atomics), "tiled" (sort by tile, shared-memory
    accumulation; uses a workspace, allocated here if not given) or "auto"
    (direct: the faster on every workload measured).  Both methods give
    bit-identical counts.  accumulate=True adds to the given counts and
    n_outside (kde_bin_accumulate) instead of overwriting them."""
    import torch
    if not (X.is_cuda or X.is_pinned()) or X.dim() != 2 or not X.is_contiguous():
        raise ValueError("X must be a contiguous (n, d) CUDA or pinned host tensor")
    if X.dtype not in (torch.float32, torch.float64):
        raise ValueError("X must be float32 or float64")
    n, d = X.shape
    M = tuple(int(m) for m in M)
    dev = X.device if X.is_cuda else torch.device("cuda")
    if method == "auto":
        method = "direct"
    if method not in ("direct", "tiled"):
        raise ValueError("method must be 'auto', 'direct' or 'tiled'")
    if counts is None:
        counts = torch.empty(M, dtype=torch.int64, device=dev)
    if method == "tiled" and workspace is None:
        workspace = bin_workspace(n, d, M, dev)
    if method == "direct":
        workspace = None
    if accumulate and counts is None:
        raise ValueError("accumulate=True needs the counts to add to")
    wsb = 0 if workspace is None else workspace.numel() * workspace.element_size()
    fn = lib().kde_bin_accumulate if accumulate else lib().kde_bin
    _check(fn(_ptr(X) if n else ctypes.c_void_p(0),
                         F32 if X.dtype == torch.float32 else F64, n, d,
                         _darr(lo), _darr(hi), _iarr(M), _ptr(counts), _ptr(n_outside),
                         _ptr(workspace), wsb, _stream_ptr(stream)))
    return counts


def kde_kernel_grid(plan: Plan, n, Kspec=None, workspace=None, stream=None):
    """Real kernel spectrum K (Eq. 6 and Eq. 10) with 1/n, 2^-32 and 1/prod(P) folded in."""
    import torch
    if Kspec is None:
        Kspec = torch.empty(plan.info.kspec_elems, dtype=plan.real_dtype(), device="cuda")
    if workspace is None:
        workspace = plan.workspace()
    _check(lib().kde_kernel_grid(plan.handle, int(n), _ptr(Kspec), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), _stream_ptr(stream)))
    return Kspec


def kde_fft_eval(plan: Plan, counts, Kspec, density=None, workspace=None, stream=None,
                 consume=False):
    """Density on the grid: F^{-1}(F(c) K) cropped to M (Eq. 10, Eq. 14).
    density may be a pinned host tensor, which the last pass writes in place.
    consume=True (kde_fft_eval_consume) leaves the counts zeroed, ready for
    the next kde_bin(..., accumulate=True)."""
    import torch
    if density is not None and not (density.is_cuda or density.is_pinned()):
        raise ValueError("density must be a CUDA or pinned host tensor")
    if density is None:
        density = torch.empty(plan.M, dtype=plan.real_dtype(), device="cuda")
    if workspace is None:
        workspace = plan.workspace()
    fn = lib().kde_fft_eval_consume if consume else lib().kde_fft_eval
    _check(fn(plan.handle, _ptr(counts), _ptr(Kspec), _ptr(density),
              _ptr(workspace), workspace.numel() * workspace.element_size(),
              _stream_ptr(stream)))
    return density


def kde_power_spectrum(plan: Plan, counts, W=None, workspace=None, stream=None):
    """w |F(c)|^2 on the half spectrum, in the plan's kernel-spectrum order."""
    import torch
    if W is None:
        W = torch.empty(plan.info.kspec_elems, dtype=plan.real_dtype(), device="cuda")
    if workspace is None:
        workspace = plan.workspace()
    _check(lib().kde_power_spectrum(plan.handle, _ptr(counts), _ptr(W), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(),
                                    _stream_ptr(stream)))
    return W


def kde_lscv_workspace_bytes(plan: Plan) -> int:
    b = ctypes.c_size_t()
    _check(lib().kde_lscv_workspace_bytes(plan.handle, ctypes.byref(b)))
    return int(b.value)


def kde_lscv(plan: Plan, n, H, W, lscv=None, pair_sums=None, workspace=None, stream=None):
    """LSCV(H_i) for a batch of candidate bandwidths (host array nH x d x d)."""
    import torch
    H = np.ascontiguousarray(np.asarray(H, dtype=np.float64))
    nH = H.shape[0]
    if lscv is None:
        lscv = torch.empty(nH, dtype=torch.float64, device="cuda")
    if workspace is None:
        workspace = torch.empty(max(256, kde_lscv_workspace_bytes(plan)), dtype=torch.uint8,
                                device="cuda")
    Hc = H.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(lib().kde_lscv(plan.handle, int(n), nH, Hc, _ptr(W), _ptr(pair_sums), _ptr(lscv),
                          _ptr(workspace), workspace.numel() * workspace.element_size(),
                          _stream_ptr(stream)))
    return lscv


def kde_lscv_autocorr_workspace_bytes(plan: Plan) -> int:
    b = ctypes.c_size_t()
    _check(lib().kde_lscv_autocorr_workspace_bytes(plan.handle, ctypes.byref(b)))
    return int(b.value)


def kde_autocorrelation(plan: Plan, counts, R=None, workspace=None, stream=None):
    """R = F^{-1}|F(c)|^2 on the plan's padding (P_0 x P_1, sample units)."""
    import torch
    if R is None:
        R = torch.empty(plan.info.P[0], plan.info.P[1], dtype=plan.real_dtype(), device="cuda")
    if workspace is None:
        workspace = torch.empty(kde_lscv_autocorr_workspace_bytes(plan), dtype=torch.uint8,
                                device="cuda")
    _check(lib().kde_autocorrelation(plan.handle, _ptr(counts), _ptr(R), _ptr(workspace),
                                     workspace.numel() * workspace.element_size(),
                                     _stream_ptr(stream)))
    return R


def kde_lscv_autocorr(plan: Plan, n, H, R, lscv=None, pair_sums=None, workspace=None, stream=None):
    """LSCV(H_i) from the counts' autocorrelation (host array nH x 2 x 2)."""
    import torch
    H = np.ascontiguousarray(np.asarray(H, dtype=np.float64))
    nH = H.shape[0]
    if lscv is None:
        lscv = torch.empty(nH, dtype=torch.float64, device="cuda")
    if workspace is None:
        workspace = torch.empty(kde_lscv_autocorr_workspace_bytes(plan), dtype=torch.uint8,
                                device="cuda")
    Hc = H.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(lib().kde_lscv_autocorr(plan.handle, int(n), nH, Hc, _ptr(R), _ptr(pair_sums),
                                   _ptr(lscv), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(),
                                   _stream_ptr(stream)))
    return lscv


def kde_lscv_autocorr_batch(plan: Plan, ns, H, R, lscv=None, pair_sums=None, workspace=None,
                            stream=None):
    """LSCV of nH candidates for each of nsets datasets: ns (nsets sample
    counts), H (host, nsets x nH x 2 x 2), R (device, nsets x P_0 x P_1);
    returns lscv (nsets x nH, FP64)."""
    import torch
    H = np.ascontiguousarray(np.asarray(H, dtype=np.float64))
    nsets, nH = H.shape[0], H.shape[1]
    n = np.ascontiguousarray(np.asarray(ns, dtype=np.int64))
    if n.shape != (nsets,):
        raise ValueError("ns must hold one sample count per set")
    if lscv is None:
        lscv = torch.empty(nsets, nH, dtype=torch.float64, device="cuda")
    if workspace is None:
        workspace = torch.empty(kde_lscv_autocorr_workspace_bytes(plan), dtype=torch.uint8,
                                device="cuda")
    _check(lib().kde_lscv_autocorr_batch(
        plan.handle, nsets, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), nH,
        H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(R), _ptr(pair_sums), _ptr(lscv),
        _ptr(workspace), workspace.numel() * workspace.element_size(), _stream_ptr(stream)))
    return lscv


def kde_wait_probe(arrive, limit, out=None, stream=None):
    """The tensor-core kernels' bounded mbarrier wait on a barrier that is
    (arrive=True) or is never (arrive=False) completed; returns a device
    int64 pair (0 completed / 1 gave up, cycles waited)."""
    import torch
    if out is None:
        out = torch.empty(2, dtype=torch.int64, device="cuda")
    _check(lib().kde_wait_probe(int(bool(arrive)), ctypes.c_uint32(int(limit)), _ptr(out),
                                _stream_ptr(stream)))
    return out


class LscvCands:
    """A candidate list prepared once on a plan (kde_lscv_cands_*): its
    parameters stay on the device, so scoring it against a dataset's
    autocorrelation launches kernels only.  Keeps its plan alive."""

    def __init__(self, plan: Plan, H):
        H = np.ascontiguousarray(np.asarray(H, dtype=np.float64))
        self.plan = plan
        self.nH = H.shape[0]
        h = ctypes.c_void_p()
        _check(lib().kde_lscv_cands_create(plan.handle, self.nH,
                                           H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           ctypes.byref(h)))
        self.handle = h

    def score(self, n, R, lscv=None, pair_sums=None, workspace=None, stream=None):
        """LSCV of every candidate for n samples with autocorrelation R."""
        import torch
        if lscv is None:
            lscv = torch.empty(self.nH, dtype=torch.float64, device="cuda")
        if workspace is None:
            workspace = torch.empty(kde_lscv_autocorr_workspace_bytes(self.plan), dtype=torch.uint8,
                                    device="cuda")
        _check(lib().kde_lscv_autocorr_cands(self.handle, int(n), _ptr(R), _ptr(pair_sums),
                                             _ptr(lscv), _ptr(workspace),
                                             workspace.numel() * workspace.element_size(),
                                             _stream_ptr(stream)))
        return lscv

    def batch_workspace_bytes(self, nsets):
        b = ctypes.c_size_t()
        _check(lib().kde_lscv_autocorr_cands_batch_workspace_bytes(self.handle, int(nsets),
                                                                   ctypes.byref(b)))
        return b.value

    def score_batch(self, ns, Rs, lscv=None, pair_sums=None, workspace=None, stream=None):
        """LSCV of every candidate for every dataset: ns (nsets sample
        counts), Rs (nsets x P_0 x P_1 autocorrelations); returns an
        nsets x nH tensor (kde_lscv_autocorr_cands_batch)."""
        import torch
        ns = np.ascontiguousarray(np.asarray(ns, dtype=np.int64))
        B = int(ns.shape[0])
        if Rs.shape[0] != B or not Rs.is_contiguous():
            raise ValueError("Rs must be a contiguous (nsets, P_0, P_1) tensor")
        if lscv is None:
            lscv = torch.empty(B, self.nH, dtype=torch.float64, device=Rs.device)
        if workspace is None:
            workspace = torch.empty(max(256, self.batch_workspace_bytes(B)), dtype=torch.uint8,
                                    device=Rs.device)
        _check(lib().kde_lscv_autocorr_cands_batch(
            self.handle, B, ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(Rs),
            _ptr(pair_sums), _ptr(lscv), _ptr(workspace),
            workspace.numel() * workspace.element_size(), _stream_ptr(stream)))
        return lscv

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.kde_lscv_cands_destroy(h)
            self.handle = None


class BatchPlan:
    """A ragged batch of 2-D problems (kde_batch_plan_*): problems is a list of
    (M, lo, hi, H, n); samples are passed concatenated in problem order."""

    def __init__(self, problems, **opts):
        arr = (BatchItem * len(problems))()
        for i, (M, lo, hi, H, n) in enumerate(problems):
            arr[i].M[:] = [int(m) for m in M]
            arr[i].lo[:] = [float(v) for v in lo]
            arr[i].hi[:] = [float(v) for v in hi]
            arr[i].H[:] = [float(v) for v in np.asarray(H, dtype=np.float64).ravel()]
            arr[i].n = int(n)
        o = _opts(**opts)
        h = ctypes.c_void_p()
        _check(lib().kde_batch_plan_create(len(problems), arr, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.precision = opts.get("precision", "f32")
        xr, de, wb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        _check(lib().kde_batch_plan_query(h, ctypes.byref(xr), ctypes.byref(de), ctypes.byref(wb)))
        self.x_rows, self.density_elems, self.workspace_bytes = xr.value, de.value, wb.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().kde_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def real_dtype(self):
        import torch
        return torch.float32 if self.precision == "f32" else torch.float64

    def workspace(self, device="cuda"):
        import torch
        return torch.empty(max(256, self.workspace_bytes), dtype=torch.uint8, device=device)

    def set_shape(self, tpl_rows, tpl_cols):
        _check(lib().kde_batch_set_shape(self._h, int(tpl_rows), int(tpl_cols)))

    def shape(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().kde_batch_get_shape(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def _query(self):
        xr, de, wb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        _check(lib().kde_batch_plan_query(self._h, ctypes.byref(xr), ctypes.byref(de),
                                          ctypes.byref(wb)))
        self.x_rows, self.density_elems, self.workspace_bytes = xr.value, de.value, wb.value

    def tune(self, X, density, workspace, reps=3, stream=None):
        """Chooses padding, radix order, mode and threads per line by timing
        (kde_batch_tune); returns the best time in ms."""
        ms = ctypes.c_float()
        _check(lib().kde_batch_tune(self._h, _ptr(X), _ptr(density), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(),
                                    _stream_ptr(stream), int(reps), ctypes.byref(ms)))
        self._query()
        return ms.value

    MODES = {"persistent": 0, "staged": 1}

    def set_mode(self, mode):
        _check(lib().kde_batch_set_mode(self._h, self.MODES[mode]))

    def mode(self):
        m = ctypes.c_int()
        _check(lib().kde_batch_get_mode(self._h, ctypes.byref(m)))
        return {v: k for k, v in self.MODES.items()}[m.value]

    def config(self, count):
        """(padding policy, radix order, padded lengths per problem)."""
        pad, order = ctypes.c_int(), ctypes.c_int()
        P = (ctypes.c_int64 * (2 * count))()
        _check(lib().kde_batch_get_config(self._h, ctypes.byref(pad), ctypes.byref(order), P))
        return ({0: "smallest", 1: "fewest_stages"}[pad.value],
                {0: "largest_first", 1: "smallest_first"}[order.value & 255],
                [(P[2 * i], P[2 * i + 1]) for i in range(count)],
                {0: "stages", 1: "problems"}[order.value >> 8])

    def set_queue_order(self, order):
        _check(lib().kde_batch_set_queue_order(self._h, {"stages": 0, "problems": 1}[order]))

    def set_wait(self, polls, withhold_stage=-1):
        _check(lib().kde_batch_set_wait(self._h, int(polls), int(withhold_stage)))

    def check(self, stream=None):
        """Raises KDEError(KDE_ERR_TIMEOUT) if a wait of the persistent kernel
        gave up since the last check (synchronises)."""
        _check(lib().kde_batch_check(self._h, _stream_ptr(stream)))

    def eval(self, X, density=None, workspace=None, stream=None):
        import torch
        if density is None:
            density = torch.empty(self.density_elems, dtype=self.real_dtype(), device="cuda")
        if workspace is None:
            workspace = self.workspace()
        _check(lib().kde_batch_eval(self._h, _ptr(X), _ptr(density), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(),
                                    _stream_ptr(stream)))
        return density


def kde_fft_eval_multi_workspace_bytes(plan: Plan) -> int:
    b = ctypes.c_size_t()
    _check(lib().kde_fft_eval_multi_workspace_bytes(plan.handle, ctypes.byref(b)))
    return int(b.value)


def kde_fft_eval_multi(plan: Plan, n, H, counts, density=None, workspace=None, stream=None):
    """Densities for every bandwidth in H (k x 2 x 2) on the plan's grid from
    one count spectrum: returns a (k, M_0, M_1) float32 tensor."""
    import torch
    H = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(-1, 2, 2))
    k = H.shape[0]
    if density is None:
        density = torch.empty((k,) + tuple(plan.M), dtype=torch.float32, device=counts.device)
    if workspace is None:
        workspace = torch.empty(max(256, kde_fft_eval_multi_workspace_bytes(plan)),
                                dtype=torch.uint8, device=counts.device)
    _check(lib().kde_fft_eval_multi(plan.handle, int(n), k, _darr(H.ravel()), _ptr(counts),
                                    _ptr(density), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), _stream_ptr(stream)))
    return density


def noalloc_scratch_bytes() -> int:
    """Size of the library's fixed scratch array (kde_noalloc_scratch_bytes)."""
    return int(lib().kde_noalloc_scratch_bytes())


def kde_fft_eval_noalloc(plan: Plan, counts, Kspec, density, stream=None):
    """kde_fft_eval with the library's fixed scratch array instead of a
    workspace (for callers that cannot allocate device memory at the call).
    The output tensor must be provided.  Plans needing more than
    noalloc_scratch_bytes() of scratch raise KDE_ERR_WORKSPACE."""
    _check(lib().kde_fft_eval_noalloc(plan.handle, _ptr(counts), _ptr(Kspec), _ptr(density),
                                      _stream_ptr(stream)))
    return density


def kde_eval(X, H, lo, hi, M, n=None, stream=None, **opts):
    """bin -> kernel grid -> FFT evaluation on one stream; returns (density, counts, plan)."""
    plan = Plan(M, lo, hi, H, **opts)
    counts = kde_bin(X, lo, hi, M, stream=stream)
    ws = plan.workspace()
    K = kde_kernel_grid(plan, X.shape[0] if n is None else n, workspace=ws, stream=stream)
    dens = kde_fft_eval(plan, counts, K, workspace=ws, stream=stream)
    return dens, counts, plan


def plan_check(plan: Plan, stream=None):
    """Raises KDEError(KDE_ERR_TIMEOUT) if a bounded device-side wait in one
    of the plan's kernels gave up since the last check (synchronises)."""
    _check(lib().kde_plan_check(plan.handle, _stream_ptr(stream)))


def outside_check(n_outside, stream=None) -> int:
    """Number of samples kde_bin dropped (device counter n_outside); raises
    KDEError(KDE_ERR_OUT_OF_RANGE) if it is nonzero (synchronises)."""
    v = ctypes.c_int64(0)
    st = lib().kde_outside_check(_ptr(n_outside), _stream_ptr(stream), ctypes.byref(v))
    if st not in (0, 3):
        _check(st)
    if st == 3:
        raise KDEError(st, f"{v.value} samples fell outside the grid")
    return v.value


def launch_count() -> int:
    return int(lib().kde_launch_count())


def profile_enable(on: bool):
    _check(lib().kde_profile_enable(1 if on else 0))


def profile_read():
    """{kernel name: (total ms, launches)} for launches since profile_enable(True)."""
    L = lib()
    out = {}
    for i in range(L.kde_profile_count()):
        name = ctypes.c_char_p()
        ms = ctypes.c_double()
        cnt = ctypes.c_int64()
        _check(L.kde_profile_entry(i, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(cnt)))
        out[name.value.decode()] = (ms.value, cnt.value)
    return out


class PreparedPath:
    """bin, kernel grid and FFT evaluation on fixed buffers, with every C
    argument marshalled once.  ``bin()``, ``kernel_grid()`` and ``fft_eval()``
    enqueue one call each on their stream (kernel_grid may use its own
    stream); ``__call__`` enqueues all three in order on one stream.
    counts_kept_zero=True: the counts start at zero (the caller zeroes them
    once) and every step keeps them so: bin() adds (kde_bin_accumulate) and
    fft_eval() leaves them zeroed (kde_fft_eval_consume), so no step zeroes
    them before binning."""

    def __init__(self, plan: Plan, X, counts, Kspec, density, workspace, n=None,
                 n_outside=None, bin_workspace=None, stream=None, kgen_stream=None,
                 counts_kept_zero=False):
        import torch
        L = lib()
        self._L = L
        self.plan = plan
        s = _stream_ptr(stream)
        sk = _stream_ptr(kgen_stream) if kgen_stream is not None else s
        nX, d = X.shape
        bwb = 0 if bin_workspace is None else bin_workspace.numel() * bin_workspace.element_size()
        self._bin = (_ptr(X), F32 if X.dtype == torch.float32 else F64, nX, d, _darr(plan.lo),
                     _darr(plan.hi), _iarr(plan.M), _ptr(counts), _ptr(n_outside),
                     _ptr(bin_workspace), bwb, s)
        wsb = workspace.numel() * workspace.element_size()
        # kernel_grid and fft_eval share the workspace only when ordered; with a
        # separate kernel-grid stream the caller passes kgen_workspace ordering
        self._kg = (plan.handle, int(nX if n is None else n), _ptr(Kspec), _ptr(workspace), wsb, sk)
        self._ev = (plan.handle, _ptr(counts), _ptr(Kspec), _ptr(density), _ptr(workspace), wsb, s)
        self._keep = (X, counts, Kspec, density, workspace, n_outside, bin_workspace)
        self._bin_fn = L.kde_bin_accumulate if counts_kept_zero else L.kde_bin
        self._ev_fn = L.kde_fft_eval_consume if counts_kept_zero else L.kde_fft_eval

    def bin(self):
        _check(self._bin_fn(*self._bin))

    def kernel_grid(self):
        _check(self._L.kde_kernel_grid(*self._kg))

    def fft_eval(self):
        _check(self._ev_fn(*self._ev))

    def __call__(self):
        self.bin()
        self.kernel_grid()
        self.fft_eval()


# ---------------------------------------------------------------------------
# Learned bandwidth proposal (features, MLP, tensor-core GEMM).
# ---------------------------------------------------------------------------
def kde_standardize2(X, Z=None, moments=None, stream=None):
    """Standardised samples Z (n x 2 float32) and moments[8] (float64)."""
    import torch
    if Z is None:
        Z = torch.empty_like(X)
    if moments is None:
        moments = torch.empty(8, dtype=torch.float64, device=X.device)
    _check(lib().kde_standardize2(_ptr(X), X.shape[0], _ptr(Z), _ptr(moments), _stream_ptr(stream)))
    return Z, moments


def kde_features2(counts, n, moments, feat=None, stream=None):
    """feat[FEAT_DIM] from M x M counts of n standardised samples."""
    import torch
    if feat is None:
        feat = torch.empty(FEAT_DIM, dtype=torch.float32, device=counts.device)
    _check(lib().kde_features2(_ptr(counts), counts.shape[0], int(n), _ptr(moments), _ptr(feat),
                               _stream_ptr(stream)))
    return feat


class FeaturePrep:
    """The per-dataset preparation of the learned selection with every fixed
    argument marshalled once: kde_standardize2 into Z, kde_bin (direct) of Z
    on the plan's grid, kde_features2, kde_autocorrelation.  run(X, feat, R)
    then makes the four C calls with only X's pointer and length and the two
    outputs changing, on the stream passed to run() (default: torch's current
    stream at that call, like every other binding); Z, counts, moments and
    the workspace are owned here."""

    def __init__(self, plan: Plan, n_max, workspace):
        import torch
        dev = workspace.device
        self.plan = plan
        self.Z = torch.empty(n_max, 2, dtype=torch.float32, device=dev)
        self.counts = torch.empty(plan.M, dtype=torch.int64, device=dev)
        self.moments = torch.empty(8, dtype=torch.float64, device=dev)
        self.ws = workspace
        self._L = lib()
        self._lo, self._hi, self._M = _darr(plan.lo), _darr(plan.hi), _iarr(plan.M)
        self._pZ, self._pc, self._pm = _ptr(self.Z), _ptr(self.counts), _ptr(self.moments)
        self._pws = _ptr(workspace)
        self._wsb = workspace.numel() * workspace.element_size()
        self._null = ctypes.c_void_p(0)

    def run(self, X, feat, R, stream=None):
        """X: n x 2 float32 CUDA tensor (n <= n_max); feat (FEAT_DIM) and R
        (P_0 x P_1) receive the features and the autocorrelation."""
        L, s = self._L, _stream_ptr(stream)
        n = int(X.shape[0])
        if n > self.Z.shape[0] or X.dim() != 2 or X.shape[1] != 2 or not X.is_contiguous() \
                or X.dtype != self.Z.dtype or not X.is_cuda:
            raise ValueError("X must be a contiguous (n, 2) float32 CUDA tensor with n <= n_max")
        px = ctypes.c_void_p(X.data_ptr())
        _check(L.kde_standardize2(px, n, self._pZ, self._pm, s))
        _check(L.kde_bin(self._pZ, F32, n, 2, self._lo, self._hi, self._M, self._pc, self._null,
                         self._null, 0, s))
        _check(L.kde_features2(self._pc, self.plan.M[0], n, self._pm,
                               ctypes.c_void_p(feat.data_ptr()), s))
        _check(L.kde_autocorrelation(self.plan.handle, self._pc, ctypes.c_void_p(R.data_ptr()),
                                     self._pws, self._wsb, s))
        return feat


def lscv_theta_select_workspace_bytes(plan: Plan, nsets, J):
    b = ctypes.c_size_t()
    _check(lib().kde_lscv_theta_select_workspace_bytes(plan.handle, int(nsets), int(J),
                                                       ctypes.byref(b)))
    return b.value


def kde_lscv_theta_select(plan: Plan, ns, theta, box_lo, box_hi, offsets, ref, R, lscv=None,
                          out=None, workspace=None, stream=None):
    """Candidates built on the device (kde_lscv_theta_select): theta (nsets x
    3 FP32 CUDA tensor), box and offsets (J x 3) and ref (nsets x 3) on the
    host, R the nsets autocorrelations.  Returns out (nsets x 6 FP64 CUDA:
    best index among the J offsets, its LSCV, the reference's LSCV, its
    theta)."""
    import torch
    ns = np.ascontiguousarray(np.asarray(ns, dtype=np.int64))
    B = int(ns.shape[0])
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.float64).reshape(-1, 3))
    J = int(off.shape[0])
    refa = np.ascontiguousarray(np.asarray(ref, dtype=np.float64).reshape(B, 3))
    box = np.ascontiguousarray(np.concatenate([np.asarray(box_lo, dtype=np.float64).reshape(3),
                                               np.asarray(box_hi, dtype=np.float64).reshape(3)]))
    if theta.dtype != torch.float32 or not theta.is_contiguous() or tuple(theta.shape) != (B, 3):
        raise ValueError("theta must be a contiguous (nsets, 3) float32 tensor")
    if out is None:
        out = torch.empty(B, 6, dtype=torch.float64, device=theta.device)
    if workspace is None:
        workspace = torch.empty(max(256, lscv_theta_select_workspace_bytes(plan, B, J)),
                                dtype=torch.uint8, device=theta.device)
    dptr = ctypes.POINTER(ctypes.c_double)
    _check(lib().kde_lscv_theta_select(
        plan.handle, B, ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(theta),
        box.ctypes.data_as(dptr), J, off.ctypes.data_as(dptr), refa.ctypes.data_as(dptr), _ptr(R),
        _ptr(lscv), _ptr(out), _ptr(workspace), workspace.numel() * workspace.element_size(),
        _stream_ptr(stream)))
    return out


class BatchPrep:
    """kde_prepare2_batch: the per-dataset preparation (standardise, bin on
    the plan's grid, features, autocorrelation) of up to nsets_max datasets
    holding up to n_total_max samples in all, in one call.  Owns the counts,
    moments and workspace; run() writes the features and autocorrelations
    into the caller's tensors."""

    def __init__(self, plan: Plan, nsets_max, n_total_max, device="cuda"):
        import torch
        self.plan = plan
        self.nsets_max, self.n_total_max = int(nsets_max), int(n_total_max)
        b = ctypes.c_size_t()
        _check(lib().kde_prepare2_batch_workspace_bytes(plan.handle, self.nsets_max,
                                                        self.n_total_max, ctypes.byref(b)))
        self.ws = torch.empty(max(256, b.value), dtype=torch.uint8, device=device)
        self.counts = torch.empty((self.nsets_max,) + tuple(plan.M), dtype=torch.int64,
                                  device=device)
        self.moments = torch.empty(self.nsets_max, 8, dtype=torch.float64, device=device)

    def run(self, X, offsets, feat, R, stream=None):
        """X: concatenated (n_total, 2) float32 CUDA tensor; offsets: nsets + 1
        row offsets (host); feat (nsets, FEAT_DIM) and R (nsets, P_0, P_1)
        receive the features and the autocorrelations."""
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        B = int(off.shape[0]) - 1
        if B < 0 or B > self.nsets_max or int(off[-1]) > self.n_total_max:
            raise ValueError("batch larger than this BatchPrep was made for")
        if X.dim() != 2 or X.shape[1] != 2 or not X.is_contiguous() or X.dtype.itemsize != 4 \
                or not X.is_cuda or X.shape[0] < int(off[-1]):
            raise ValueError("X must be a contiguous (n_total, 2) float32 CUDA tensor")
        if feat.shape[0] < B or R.shape[0] < B or not feat.is_contiguous() or not R.is_contiguous():
            raise ValueError("feat and R need one contiguous row per dataset")
        _check(lib().kde_prepare2_batch(
            self.plan.handle, B, _ptr(X), off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            _ptr(self.counts), _ptr(self.moments), _ptr(feat), _ptr(R), _ptr(self.ws),
            self.ws.numel() * self.ws.element_size(), _stream_ptr(stream)))
        return feat, R


def kde_gemm_bf16(A, B, C=None, status=None, stream=None):
    """C = A B^T on the tensor cores (A: M x K, B: N x K, bfloat16)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    if C is None:
        C = torch.empty(M, N, dtype=torch.float32, device=A.device)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib().kde_gemm_bf16(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C),
                               C.stride(0), _ptr(status), _stream_ptr(stream)))
    return C, status


class MLP:
    """kde_mlp_create / kde_mlp_destroy and the calls on one network."""

    def __init__(self, in_dim=FEAT_DIM, hidden=256, out_dim=3, max_batch=256, seed=0):
        L = lib()
        h = ctypes.c_void_p()
        _check(L.kde_mlp_create(in_dim, hidden, out_dim, max_batch, seed, ctypes.byref(h)))
        self.handle = h
        self.in_dim, self.hidden, self.out_dim, self.max_batch = in_dim, hidden, out_dim, max_batch
        n = ctypes.c_int64()
        _check(L.kde_mlp_param_count(h, ctypes.byref(n)))
        self.nparam = n.value

    def __del__(self):
        if getattr(self, "handle", None):
            lib().kde_mlp_destroy(self.handle)
            self.handle = None

    def get_params(self):
        out = np.empty(self.nparam, dtype=np.float32)
        _check(lib().kde_mlp_get_params(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        self.nparam))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().kde_mlp_set_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        self.nparam))

    def get_state(self):
        m = np.empty(self.nparam, dtype=np.float32)
        v = np.empty(self.nparam, dtype=np.float32)
        step = ctypes.c_int64()
        fp = ctypes.POINTER(ctypes.c_float)
        _check(lib().kde_mlp_get_state(self.handle, m.ctypes.data_as(fp), v.ctypes.data_as(fp),
                                       ctypes.byref(step)))
        return m, v, step.value

    def set_state(self, m, v, step):
        m = np.ascontiguousarray(m, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        _check(lib().kde_mlp_set_state(self.handle, m.ctypes.data_as(fp), v.ctypes.data_as(fp),
                                       int(step)))

    def forward(self, X, Y=None, stream=None):
        import torch
        if Y is None:
            Y = torch.empty(X.shape[0], self.out_dim, dtype=torch.float32, device=X.device)
        _check(lib().kde_mlp_forward(self.handle, _ptr(X), X.shape[0], _ptr(Y), _stream_ptr(stream)))
        return Y

    def loss_grad(self, X, T, loss=None, grads=None, stream=None):
        import torch
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=X.device)
        if grads is None:
            grads = torch.empty(self.nparam, dtype=torch.float32, device=X.device)
        _check(lib().kde_mlp_loss_grad(self.handle, _ptr(X), _ptr(T), X.shape[0], _ptr(loss),
                                       _ptr(grads), _stream_ptr(stream)))
        return loss, grads

    def train_step(self, X, T, lr, loss=None, stream=None):
        _check(lib().kde_mlp_train_step(self.handle, _ptr(X), _ptr(T), X.shape[0], float(lr),
                                        _ptr(loss), _stream_ptr(stream)))
        return loss

    def status(self):
        f = ctypes.c_int()
        _check(lib().kde_mlp_status(self.handle, ctypes.byref(f)))
        return f.value

    def check(self):
        """Raises KDEError(KDE_ERR_TIMEOUT) if a tensor-core wait of this
        network gave up (its last results are then invalid); synchronises."""
        if self.status():
            raise KDEError(6, "a tensor-core wait of the network gave up; results are invalid")

    def status_copy(self, dst, stream=None):
        """Enqueues a copy of the status flag into dst (one int32, device or
        pinned host tensor) on the stream, without synchronising; a caller
        that reads its results anyway then checks dst (kde_mlp_status_copy)."""
        _check(lib().kde_mlp_status_copy(self.handle, _ptr(dst), _stream_ptr(stream)))
        return dst
