"""FP64 CPU oracle of the photoacoustic operator A and its adjoint.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  It shares no code with the CUDA library: the C source
``pat_oracle.c`` restates the paper's steps on its own, and this module only
marshals numpy arrays to it through ctypes.

Functions take a workload-like object ``w`` with the attributes of
``Workload`` (n, origin, pitch, tx, c, fs, t0, L, U, dl, method, q1, q2) but do
not import the product package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pat_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libpat_oracle.so")
_lock = threading.Lock()
_lib = None

_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP64, OpenMP) into oracle/_build."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _OUT)
    return _OUT


def _opt_i64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp = C.c_void_p
            L.oracle_carlson_rf.restype = C.c_double
            L.oracle_carlson_rf.argtypes = [C.c_double] * 3
            L.oracle_carlson_rd.restype = C.c_double
            L.oracle_carlson_rd.argtypes = [C.c_double] * 3
            for nm in ("oracle_ellip_f", "oracle_ellip_e", "oracle_ellip_e_any"):
                getattr(L, nm).restype = C.c_double
                getattr(L, nm).argtypes = [C.c_double, C.c_double]
            L.oracle_pair_bin_areas.restype = C.c_int64
            L.oracle_pair_bin_areas.argtypes = [_D, _D, _D, _I32, C.POINTER(C.c_int64), _D, C.c_int64]
            L.oracle_pair_bin_areas_m.restype = C.c_int64
            L.oracle_pair_bin_areas_m.argtypes = [_D, _D, _D, _I32, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int64),
                                                  _D, C.c_int64]
            L.oracle_ellip_e_lut.restype = C.c_double
            L.oracle_ellip_e_lut.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int]
            L.oracle_lut_node.restype = C.c_double
            L.oracle_lut_node.argtypes = [C.c_int, C.c_int]
            L.oracle_pair_range.restype = C.c_int
            L.oracle_pair_range.argtypes = [_D, _D, _D]
            geo = [_I32, _D, C.c_double, _D, C.c_int, _D, _I32, C.c_int, C.c_int, C.c_int]
            L.oracle_geometric_forward.restype = C.c_int64
            L.oracle_geometric_forward.argtypes = geo + [vp, C.c_int64, _D, _D]
            L.oracle_geometric_adjoint.restype = C.c_int64
            L.oracle_geometric_adjoint.argtypes = geo + [_D, vp, C.c_int64, _D]
            L.oracle_conv_forward.restype = None
            L.oracle_conv_forward.argtypes = [_D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _D, _D]
            L.oracle_conv_adjoint.restype = None
            L.oracle_conv_adjoint.argtypes = [_D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _D, _D]
            L.oracle_forward.restype = C.c_int64
            L.oracle_forward.argtypes = geo + [_D, C.c_int, C.c_int, vp, C.c_int64, _D, _D, vp]
            L.oracle_adjoint.restype = C.c_int64
            L.oracle_adjoint.argtypes = geo + [_D, C.c_int, C.c_int, _D, vp, C.c_int64, _D, vp]
            L.oracle_system_kernel.restype = None
            L.oracle_system_kernel.argtypes = [C.c_int, C.c_double, C.c_int, _D, C.c_double, C.c_double, C.c_int,
                                               C.c_int, C.c_int, C.c_int, _D]
            L.oracle_h_value.restype = C.c_double
            L.oracle_h_value.argtypes = [C.c_int, C.c_double, C.c_int, _D, C.c_double, C.c_int, C.c_double]
            L.oracle_quad_points.restype = None
            L.oracle_quad_points.argtypes = [_D, C.c_int, C.c_int, _D, _D]
            L.oracle_num_threads.restype = C.c_int
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# --------------------------------------------------------------------------
def _geo_args(w):
    n = np.ascontiguousarray(np.asarray(w.n, dtype=np.int32))
    org = np.ascontiguousarray(np.asarray(w.origin, dtype=np.float64))
    tx = np.ascontiguousarray(np.asarray(w.tx, dtype=np.float64))
    tp = np.array([w.c, w.fs, w.t0], dtype=np.float64)
    ip = np.array([w.L, w.U, w.dl], dtype=np.int32)
    return [n, org, float(w.pitch), tx, int(tx.shape[0]), tp, ip, int(w.method), int(w.q1), int(w.q2)]


def _idx_args(vox_idx, N):
    if vox_idx is None:
        return None, N, None
    idx = _opt_i64(vox_idx)
    return idx.ctypes.data_as(C.c_void_p), int(idx.size), idx


def time_args(w):
    return np.array([w.c, w.fs, w.t0], dtype=np.float64), np.array([w.L, w.U, w.dl], dtype=np.int32)


def geometric_forward(w, x, vox_idx=None):
    """f = [K][UL] geometric signals (Alg. 2 / Alg. 3)."""
    N = int(np.prod(w.n))
    p, nv, keep = _idx_args(vox_idx, N)
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.zeros((w.tx.shape[0], w.U * w.L))
    d = lib().oracle_geometric_forward(*_geo_args(w), p, nv, x, f)
    return f, int(d)


def geometric_adjoint(w, v, vox_idx=None):
    N = int(np.prod(w.n))
    p, nv, keep = _idx_args(vox_idx, N)
    v = np.ascontiguousarray(v, dtype=np.float64)
    z = np.zeros(nv)
    d = lib().oracle_geometric_adjoint(*_geo_args(w), v, p, nv, z)
    return z, int(d)


def conv_forward(w, taps, f):
    taps = np.ascontiguousarray(taps, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    K = f.shape[0]
    s = np.zeros((K, w.L))
    lib().oracle_conv_forward(taps, taps.size, int(w.n_lo), int(w.U), int(w.L), K, f, s)
    return s


def conv_adjoint(w, taps, s):
    taps = np.ascontiguousarray(taps, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    K = s.shape[0]
    v = np.zeros((K, w.U * w.L))
    lib().oracle_conv_adjoint(taps, taps.size, int(w.n_lo), int(w.U), int(w.L), K, s, v)
    return v


def forward(w, taps, x, vox_idx=None):
    """s = A x, [K][L] (Alg. 1).  x has N entries, or one per vox_idx."""
    N = int(np.prod(w.n))
    p, nv, keep = _idx_args(vox_idx, N)
    taps = np.ascontiguousarray(taps, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    s = np.zeros((w.tx.shape[0], w.L))
    d = lib().oracle_forward(*_geo_args(w), taps, taps.size, int(w.n_lo), p, nv, x, s, None)
    return s, int(d)


def adjoint(w, taps, s, vox_idx=None):
    """z = A^T s (Alg. 5); z has N entries, or one per vox_idx."""
    N = int(np.prod(w.n))
    p, nv, keep = _idx_args(vox_idx, N)
    taps = np.ascontiguousarray(taps, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    z = np.zeros(nv)
    d = lib().oracle_adjoint(*_geo_args(w), taps, taps.size, int(w.n_lo), s, p, nv, z, None)
    return z, int(d)


def system_kernel(rbf_kind, kappa, eir_kind, eir_par, c, fs, U, n_lo, T, panels=3):
    """Discrete system kernel taps h-bar[n_lo .. n_lo + T) (Eq. def_bh)."""
    taps = np.zeros(T)
    lib().oracle_system_kernel(int(rbf_kind), float(kappa), int(eir_kind),
                               np.ascontiguousarray(eir_par, dtype=np.float64), float(c), float(fs), int(U),
                               int(n_lo), int(T), int(panels), taps)
    return taps


def taps_for(w, panels=3):
    return system_kernel(w.rbf_kind, w.kappa, w.eir_kind, w.eir_par, w.c, w.fs, w.U, w.n_lo, w.T, panels)


def h_value(rbf_kind, kappa, eir_kind, eir_par, c, t, panels=3):
    return lib().oracle_h_value(int(rbf_kind), float(kappa), int(eir_kind),
                                np.ascontiguousarray(eir_par, dtype=np.float64), float(c), int(panels), float(t))


def quad_points(tx_row, q1, q2):
    """The point method's Q1 x Q2 points of one element, [Q, 3], and their
    areas dq [Q] (Alg. 2, Sec. 3.2), point j = j1 q2 + j2."""
    pts = np.zeros(3 * q1 * q2)
    dq = np.zeros(q1 * q2)
    lib().oracle_quad_points(np.ascontiguousarray(tx_row, dtype=np.float64), int(q1), int(q2), pts, dq)
    return pts.reshape(-1, 3), dq


METHOD_SURFACE, METHOD_POINT, METHOD_TRAPEZOID, METHOD_LUT = 0, 1, 2, 3


def pair_bin_areas(tx_row, xi, w, method=METHOD_SURFACE, lut=(1000, 1000)):
    """(b_min, areas per fine bin) of one voxel-transducer pair; method
    METHOD_TRAPEZOID takes the trapezoidal arc integral for a cylinder,
    METHOD_LUT the elliptic closed form with E from lut = (N_s, N_m) tables."""
    tp, ip = time_args(w)
    q1, q2 = (int(lut[0]), int(lut[1])) if method == METHOD_LUT else (0, 0)
    tx_row = np.ascontiguousarray(tx_row, dtype=np.float64)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    cap = 1 << 16
    out = np.zeros(cap)
    bmin = C.c_int64(0)
    nb = lib().oracle_pair_bin_areas_m(tx_row, xi, tp, ip, int(method), q1, q2, C.byref(bmin), out, cap)
    if nb < 0:
        cap = -nb
        out = np.zeros(cap)
        nb = lib().oracle_pair_bin_areas_m(tx_row, xi, tp, ip, int(method), q1, q2, C.byref(bmin), out, cap)
    return int(bmin.value), out[:nb].copy()


def pair_range(tx_row, xi):
    out = np.zeros(2)
    nq = lib().oracle_pair_range(np.ascontiguousarray(tx_row, dtype=np.float64),
                                 np.ascontiguousarray(xi, dtype=np.float64), out)
    return float(out[0]), float(out[1]), int(nq)


def carlson_rf(x, y, z):
    return lib().oracle_carlson_rf(x, y, z)


def carlson_rd(x, y, z):
    return lib().oracle_carlson_rd(x, y, z)


def ellip_e(phi, m):
    return lib().oracle_ellip_e(phi, m)


def ellip_f(phi, m):
    return lib().oracle_ellip_f(phi, m)


def ellip_e_any(theta, nu):
    return lib().oracle_ellip_e_any(theta, nu)


def ellip_e_lut(theta, nu, ns=1000, nm=1000):
    """E(theta, nu) from the ns x nm lookup tables (Sec. 4.2.2), any nu >= 0."""
    return lib().oracle_ellip_e_lut(float(theta), float(nu), int(ns), int(nm))


def lut_node(n, N):
    """Node n (0-based) of the power-law grid of Eq. (LUT_sampling)."""
    return lib().oracle_lut_node(int(n), int(N))


# --------------------------------------------------------------------------
# Piecewise-Planes (Sec. 4.3): a cylindrical element replaced by n_planes
# planes tangent to it at the centres of equal angular sectors.
# --------------------------------------------------------------------------
def piecewise_planes(tx_row, n_planes):
    """Descriptor rows (16 doubles, plane layout) of the n_planes tangent
    planes of one cylindrical element: sector j of width 2 theta_max /
    n_planes has central angle theta_j; its plane touches the cylinder along
    the generator at theta_j, with half-width R dtheta / 2 across the
    generator and half-height Lz along the axis e1.  A planar row is
    returned unchanged (one plane)."""
    row = np.asarray(tx_row, dtype=np.float64)
    if int(row[0]) != 1:
        return row[None, :].copy()
    c0, e1, e2 = row[1:4], row[4:7], row[7:10]
    R, th, Lz = float(row[12]), float(row[13]), float(row[14])
    n = np.cross(e1, e2)
    dth = 2.0 * th / n_planes
    out = np.zeros((n_planes, row.size))
    for j in range(n_planes):
        tj = -th + (j + 0.5) * dth
        radial = np.cos(tj) * e2 + np.sin(tj) * n      # from the focal line to the surface
        tangent = -np.sin(tj) * e2 + np.cos(tj) * n    # along the arc
        out[j, 0] = 0.0
        out[j, 1:4] = c0 + R * radial
        out[j, 4:7] = tangent
        out[j, 7:10] = e1
        out[j, 10] = 0.5 * R * dth
        out[j, 11] = Lz
    return out


def piecewise_planes_forward(w, taps, x, n_planes, vox_idx=None):
    """s = A x with every cylindrical element replaced by its tangent planes:
    the planes' signals summed per element (the geometric coefficients add,
    and the convolution is linear)."""
    rows, owner = [], []
    for k, row in enumerate(w.tx):
        f = piecewise_planes(row, n_planes)
        rows.append(f)
        owner += [k] * len(f)
    wp = w.with_tx(np.concatenate(rows))
    sp, d = forward(wp, taps, x, vox_idx)
    s = np.zeros((w.tx.shape[0], w.L))
    np.add.at(s, np.asarray(owner), sp)
    return s, d


def piecewise_planes_adjoint(w, taps, s, n_planes, vox_idx=None):
    """The transpose: each element's signal replicated to its planes."""
    rows, owner = [], []
    for k, row in enumerate(w.tx):
        f = piecewise_planes(row, n_planes)
        rows.append(f)
        owner += [k] * len(f)
    wp = w.with_tx(np.concatenate(rows))
    return adjoint(wp, taps, np.asarray(s)[np.asarray(owner)], vox_idx)
