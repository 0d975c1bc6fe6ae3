"""ctypes binding of include/pat.h (argument marshalling only).

Every function here has the name of the C entry point it calls and forwards
device pointers taken from torch tensors plus the current CUDA stream.  No
step of the operator runs in Python: if the CUDA library cannot be loaded the
import fails loudly; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

PAT_OK = 0
PAT_ERR_WORKSPACE = 4
PAT_OP_FORWARD, PAT_OP_ADJOINT, PAT_OP_RECON, PAT_OP_FORWARD_DC, PAT_OP_AUTOTUNE, PAT_OP_CONV_SPLIT = 1, 2, 3, 4, 5, 6
PAT_FLAG_ALLOW_CLIP = 1
PAT_FLAG_CONV_TC = 2
PAT_FLAG_PIECEWISE_PLANES = 4
_STATUS = {0: "PAT_OK", 1: "PAT_ERR_INVALID_ARG", 2: "PAT_ERR_GEOMETRY", 3: "PAT_ERR_WINDOW",
           4: "PAT_ERR_WORKSPACE", 5: "PAT_ERR_CUDA", 6: "PAT_ERR_UNSUPPORTED"}


class PatError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class pat_grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("reserved", C.c_int32), ("origin", C.c_double * 3), ("pitch", C.c_double)]


class pat_params(C.Structure):
    _fields_ = [("c", C.c_double), ("fs", C.c_double), ("t0", C.c_double), ("L", C.c_int32), ("U", C.c_int32),
                ("dl", C.c_int32), ("method", C.c_int32), ("q1", C.c_int32), ("q2", C.c_int32),
                ("flags", C.c_int32), ("np_planes", C.c_int32)]


class pat_system(C.Structure):
    _fields_ = [("rbf_kind", C.c_int32), ("eir_kind", C.c_int32), ("kappa", C.c_double), ("eir", C.c_double * 4)]


class pat_peaks(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("fp32_ffma_flops", "fp32_ffma2_flops", "fp64_dfma_flops", "sfu_rsqrt_ops")]


class pat_plan_info(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("N", "K", "L", "U", "UL", "dl", "method", "n_taps", "n_lo", "bin_lo",
                                         "bin_hi", "area_evals", "pair_bins", "quad_evals", "clipped_pairs",
                                         "conv_clipped")] + \
               [("dist_min", C.c_double), ("fwd_blocks", C.c_int64), ("adj_blocks", C.c_int64),
                ("tc_error", C.c_int64)]


EXPORTS = ["pat_system_kernel", "pat_system_kernel_dc", "pat_plan_create", "pat_plan_destroy", "pat_plan_get_info",
           "pat_workspace_bytes", "pat_forward", "pat_adjoint", "pat_forward_geometric", "pat_conv_forward",
           "pat_conv_adjoint", "pat_conv_split", "pat_conv_forward_split", "pat_conv_forward_split_withheld",
           "pat_plan_clear_tc_error", "pat_adjoint_geometric", "pat_forward_dc", "pat_recon", "pat_recon_batch",
           "pat_plan_autotune", "pat_forward_static", "pat_measure_peaks", "pat_last_error", "pat_version"]

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpat.so (building it first if needed); raises if it cannot."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"libpat.so not found at {path}")
        L = C.CDLL(path)
        vp, st = C.c_void_p, C.c_int
        L.pat_system_kernel.restype = st
        L.pat_system_kernel.argtypes = [C.POINTER(pat_system), C.c_double, C.c_double, C.c_int32, C.c_int32,
                                        C.c_int32, vp, vp]
        L.pat_system_kernel_dc.restype = st
        L.pat_system_kernel_dc.argtypes = L.pat_system_kernel.argtypes
        L.pat_forward_dc.restype = st
        L.pat_forward_dc.argtypes = [vp, vp, vp, vp, vp, C.c_size_t, vp]
        L.pat_plan_create.restype = st
        L.pat_plan_create.argtypes = [C.POINTER(vp), C.POINTER(pat_grid), vp, C.c_int32, C.POINTER(pat_params),
                                      C.c_double, vp, C.c_int32, C.c_int32, vp]
        L.pat_plan_destroy.restype = st
        L.pat_plan_destroy.argtypes = [vp]
        L.pat_plan_get_info.restype = st
        L.pat_plan_get_info.argtypes = [vp, C.POINTER(pat_plan_info)]
        L.pat_workspace_bytes.restype = C.c_size_t
        L.pat_workspace_bytes.argtypes = [vp, C.c_int32]
        for nm in ("pat_forward", "pat_adjoint", "pat_forward_geometric", "pat_adjoint_geometric"):
            getattr(L, nm).restype = st
            getattr(L, nm).argtypes = [vp, vp, vp, vp, C.c_size_t, vp]
        for nm in ("pat_conv_forward", "pat_conv_adjoint", "pat_conv_split", "pat_conv_forward_split",
                   "pat_conv_forward_split_withheld"):
            getattr(L, nm).restype = st
            getattr(L, nm).argtypes = [vp, vp, vp, vp]
        L.pat_plan_clear_tc_error.restype = st
        L.pat_plan_clear_tc_error.argtypes = [vp, vp]
        L.pat_forward_static.restype = st
        L.pat_forward_static.argtypes = [vp, vp, vp, vp]
        L.pat_recon.restype = st
        L.pat_recon.argtypes = [vp, vp, vp, C.c_int32, C.c_float, C.c_float, vp, C.c_size_t, vp]
        L.pat_recon_batch.restype = st
        L.pat_recon_batch.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, vp, vp, vp, vp, vp]
        L.pat_plan_autotune.restype = st
        L.pat_plan_autotune.argtypes = [vp, vp, vp, C.c_size_t, vp]
        L.pat_measure_peaks.restype = st
        L.pat_measure_peaks.argtypes = [C.POINTER(pat_peaks), vp]
        L.pat_last_error.restype = C.c_char_p
        L.pat_last_error.argtypes = []
        L.pat_version.restype = C.c_int32
        L.pat_version.argtypes = []
        _lib = L
        return L


def check(status):
    if status != PAT_OK:
        raise PatError(status, load().pat_last_error().decode())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# same-name wrappers (torch tensors in, status checked)
# ---------------------------------------------------------------------------
def pat_system_kernel(rbf_kind, kappa, eir_kind, eir, c, fs, U, n_lo, taps_dev, stream=None):
    sys = pat_system(int(rbf_kind), int(eir_kind), float(kappa), (C.c_double * 4)(*[float(v) for v in eir]))
    check(load().pat_system_kernel(C.byref(sys), float(c), float(fs), int(U), int(n_lo), int(taps_dev.numel()),
                                   _ptr(taps_dev), _stream(stream)))


def pat_system_kernel_dc(rbf_kind, kappa, eir_kind, eir, c, fs, U, n_lo, dtaps_dev, stream=None):
    sys = pat_system(int(rbf_kind), int(eir_kind), float(kappa), (C.c_double * 4)(*[float(v) for v in eir]))
    check(load().pat_system_kernel_dc(C.byref(sys), float(c), float(fs), int(U), int(n_lo), int(dtaps_dev.numel()),
                                      _ptr(dtaps_dev), _stream(stream)))


def pat_forward_dc(plan, x, dtaps, ds, ws, stream=None):
    check(load().pat_forward_dc(plan, _ptr(x), _ptr(dtaps), _ptr(ds), _ptr(ws), ws.numel(), _stream(stream)))


def pat_plan_create(n, origin, pitch, tx, c, fs, t0, L, U, dl, method, q1, q2, flags, kappa, taps, n_lo,
                    stream=None, np_planes=0):
    grid = pat_grid((C.c_int32 * 3)(*[int(v) for v in n]), 0, (C.c_double * 3)(*[float(v) for v in origin]),
                    float(pitch))
    par = pat_params(float(c), float(fs), float(t0), int(L), int(U), int(dl), int(method), int(q1), int(q2),
                     int(flags), int(np_planes))
    tx = np.ascontiguousarray(tx, dtype=np.float64)
    taps = np.ascontiguousarray(taps, dtype=np.float64)
    out = C.c_void_p()
    check(load().pat_plan_create(C.byref(out), C.byref(grid), tx.ctypes.data_as(C.c_void_p), int(tx.shape[0]),
                                 C.byref(par), float(kappa), taps.ctypes.data_as(C.c_void_p), int(taps.size),
                                 int(n_lo), _stream(stream)))
    return out


def pat_plan_destroy(plan):
    check(load().pat_plan_destroy(plan))


def pat_plan_get_info(plan):
    info = pat_plan_info()
    check(load().pat_plan_get_info(plan, C.byref(info)))
    return {f: getattr(info, f) for f, _ in pat_plan_info._fields_}


def pat_workspace_bytes(plan, op):
    return int(load().pat_workspace_bytes(plan, int(op)))


def pat_forward(plan, x, s, ws, stream=None):
    check(load().pat_forward(plan, _ptr(x), _ptr(s), _ptr(ws), ws.numel(), _stream(stream)))


def pat_adjoint(plan, s, z, ws, stream=None):
    check(load().pat_adjoint(plan, _ptr(s), _ptr(z), _ptr(ws), ws.numel(), _stream(stream)))


def pat_forward_geometric(plan, x, f, ws, stream=None):
    check(load().pat_forward_geometric(plan, _ptr(x), _ptr(f), _ptr(ws), ws.numel(), _stream(stream)))


def pat_adjoint_geometric(plan, v, z, ws, stream=None):
    check(load().pat_adjoint_geometric(plan, _ptr(v), _ptr(z), _ptr(ws), ws.numel(), _stream(stream)))


def pat_conv_forward(plan, f, s, stream=None):
    check(load().pat_conv_forward(plan, _ptr(f), _ptr(s), _stream(stream)))


def pat_conv_adjoint(plan, s, v, stream=None):
    check(load().pat_conv_adjoint(plan, _ptr(s), _ptr(v), _stream(stream)))


def pat_conv_split(plan, f, planes, stream=None):
    check(load().pat_conv_split(plan, _ptr(f), _ptr(planes), _stream(stream)))


def pat_conv_forward_split(plan, planes, s, stream=None):
    check(load().pat_conv_forward_split(plan, _ptr(planes), _ptr(s), _stream(stream)))


def pat_conv_forward_split_withheld(plan, planes, s, stream=None):
    check(load().pat_conv_forward_split_withheld(plan, _ptr(planes), _ptr(s), _stream(stream)))


def pat_plan_clear_tc_error(plan, stream=None):
    check(load().pat_plan_clear_tc_error(plan, _stream(stream)))


def pat_recon(plan, s, x, iters, lambda_R, step, ws, stream=None):
    check(load().pat_recon(plan, _ptr(s), _ptr(x), int(iters), float(lambda_R), float(step), _ptr(ws), ws.numel(),
                           _stream(stream)))


def pat_recon_batch(plans, s_list, x_list, iters, lambdas, steps, ws_list, stream=None):
    n = len(plans)
    P = (C.c_void_p * n)(*[p.value if isinstance(p, C.c_void_p) else p for p in plans])
    S = (C.c_void_p * n)(*[t.data_ptr() for t in s_list])
    X = (C.c_void_p * n)(*[t.data_ptr() for t in x_list])
    lam = (C.c_float * n)(*[float(v) for v in lambdas])
    stp = (C.c_float * n)(*[float(v) for v in steps]) if steps is not None else None
    WS = (C.c_void_p * n)(*[t.data_ptr() for t in ws_list])
    WB = (C.c_size_t * n)(*[t.numel() for t in ws_list])
    check(load().pat_recon_batch(P, n, S, X, int(iters), lam, stp, WS, WB, _stream(stream)))


def pat_plan_autotune(plan, x, ws, stream=None):
    check(load().pat_plan_autotune(plan, _ptr(x), _ptr(ws), ws.numel(), _stream(stream)))


def pat_forward_static(plan, x, s, stream=None):
    check(load().pat_forward_static(plan, _ptr(x), _ptr(s), _stream(stream)))


def pat_measure_peaks(stream=None):
    """Measured FP32 (FFMA, FFMA2), FP64 (DFMA) flop/s and SFU rsqrt op/s of
    the current device (dependent-chain kernels)."""
    out = pat_peaks()
    check(load().pat_measure_peaks(C.byref(out), _stream(stream)))
    return {f: getattr(out, f) for f, _ in pat_peaks._fields_}


def pat_version():
    return int(load().pat_version())
