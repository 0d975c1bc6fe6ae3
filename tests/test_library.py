"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/pat.h declares; host-side argument checks return the
documented status without touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pat_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("pat_forward", "pat_adjoint", "pat_recon", "pat_plan_create", "pat_plan_destroy",
                 "pat_system_kernel", "pat_workspace_bytes", "pat_last_error"):
        assert need in names


def test_library_exports_every_declared_symbol():
    from paper_2609_29253_gb300 import _lib

    L = _lib.load()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert _lib.pat_version() == 100


def test_host_side_validation_without_gpu():
    """Null and invalid arguments are rejected before any CUDA call."""
    from paper_2609_29253_gb300 import _lib

    L = _lib.load()
    out = C.c_void_p()
    assert L.pat_plan_create(C.byref(out), None, None, 0, None, 0.0, None, 0, 0, None) == 1
    assert b"null" in L.pat_last_error()
    assert L.pat_workspace_bytes(None, 1) == 0
    assert L.pat_forward(None, None, None, None, 0, None) == 1
    assert L.pat_plan_destroy(None) == 0
    g = _lib.pat_grid((C.c_int32 * 3)(4, 4, 0), 0, (C.c_double * 3)(0, 0, 0), 1e-4)
    p = _lib.pat_params(1500.0, 40e6, 0.0, 16, 11, 11, 0, 0, 0, 0, 0)
    tx = (C.c_double * 16)(*([0.0] * 16))
    taps = (C.c_double * 4)(0, 1, -1, 0)
    assert L.pat_plan_create(C.byref(out), C.byref(g), tx, 1, C.byref(p), 1e-4, taps, 4, -1, None) == 1
    assert b"grid size" in L.pat_last_error()
    g.n[2] = 4
    p.dl = 12  # dl > U
    assert L.pat_plan_create(C.byref(out), C.byref(g), tx, 1, C.byref(p), 1e-4, taps, 4, -1, None) == 1
    p.dl = 11
    # e1, e2 = 0: not orthonormal
    assert L.pat_plan_create(C.byref(out), C.byref(g), tx, 1, C.byref(p), 1e-4, taps, 4, -1, None) == 1
    assert b"orthonormal" in L.pat_last_error()
    assert out.value is None
    # lookup tables need 2 .. 8192 nodes per axis
    p.method, p.q1, p.q2 = 3, 1, 1000
    assert L.pat_plan_create(C.byref(out), C.byref(g), tx, 1, C.byref(p), 1e-4, taps, 4, -1, None) == 1
    assert b"lookup tables" in L.pat_last_error()
    assert out.value is None
    assert L.pat_measure_peaks(None, None) == 1


def test_build_flags_target_sm103a():
    from paper_2609_29253_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
