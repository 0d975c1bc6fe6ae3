"""pat_forward_static: the forward operator for callers that cannot allocate
device memory (code where cudaMalloc is unavailable or forbidden, such as a
host callback or a plug-in that must not touch the allocator).  Its scratch
is a fixed array inside the library, so the call needs only the plan, x and s.

Checked through the C ABI against pat_forward (same kernels, caller-provided
workspace) on two calls in a row, within the tolerance of the GPU parity
tests, plus the size limit.  Collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2609_29253_gb300 import workloads as W  # noqa: E402

TOL = 1e-5  # rel L2, as for the surface method in test_gpu_parity


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def parts(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_29253_gb300 import _lib, api

    return _lib, api, oracle_mod


def _call_static(_lib, plan, x, s):
    L = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.pat_forward_static(plan.handle, C.c_void_p(x.data_ptr()), C.c_void_p(s.data_ptr()), stream)


@pytest.mark.parametrize("make,conv_tc", [(lambda: W.c1(), False),
                                          (lambda: W.small_cylinder(n_vox=12, n_angles=4, n_el=3), False),
                                          (lambda: W.small_cylinder(n_vox=12, n_angles=4, n_el=3), True)],
                         ids=["plane", "cylinder", "cylinder-tensor-core-conv"])
def test_static_forward_matches_forward(parts, make, conv_tc):
    """With conv_tc the scratch also holds f as BF16 hi and lo planes after
    the FP64 difference array, which the tensor-core convolution reads."""
    _lib, api, orc = parts
    w = make()
    plan = api.Plan(w, taps=orc.taps_for(w), conv_tc=conv_tc)
    x = torch.from_numpy(w.x.astype(np.float32)).cuda()
    s_ref = plan.forward(x).cpu().numpy()
    for _ in range(2):  # the scratch keeps the previous call's contents
        s = torch.full((w.K, w.L), float("nan"), dtype=torch.float32, device="cuda")
        assert _call_static(_lib, plan, x, s) == 0, _lib.load().pat_last_error()
        torch.cuda.synchronize()
        assert rel(s.cpu().numpy(), s_ref) <= TOL


def test_static_forward_rejects_oversize_plan(parts):
    _lib, api, orc = parts
    w = W.c1()
    w = w.with_tx(np.tile(w.tx, (50, 1)))  # 1600 positions: K (U L + 1) 8 bytes > 16 MiB
    plan = api.Plan(w, taps=orc.taps_for(w))
    assert _lib.pat_workspace_bytes(plan.handle, _lib.PAT_OP_FORWARD) > (16 << 20)
    x = torch.from_numpy(w.x.astype(np.float32)).cuda()
    s = torch.empty((w.K, w.L), dtype=torch.float32, device="cuda")
    assert _call_static(_lib, plan, x, s) == _lib.PAT_ERR_WORKSPACE
    assert b"fixed array" in _lib.load().pat_last_error()


def test_static_forward_rejects_tensor_core_f_beyond_limit(parts):
    """704 c1 positions: the difference array alone, K (U L + 1) 8 bytes,
    fits the fixed array; with the tensor-core convolution's f planes, K ld 4
    bytes more (ld = U L rounded up to a multiple of 8), it does not, and only
    that plan is rejected."""
    _lib, api, orc = parts
    w = W.c1()
    w = w.with_tx(np.tile(w.tx, (22, 1)))
    taps = orc.taps_for(w)
    plain = api.Plan(w, taps=taps)
    tc = api.Plan(w, taps=taps, conv_tc=True)
    assert _lib.pat_workspace_bytes(plain.handle, _lib.PAT_OP_FORWARD) <= (16 << 20)
    assert _lib.pat_workspace_bytes(tc.handle, _lib.PAT_OP_FORWARD) > (16 << 20)
    x = torch.from_numpy(w.x.astype(np.float32)).cuda()
    s = torch.empty((w.K, w.L), dtype=torch.float32, device="cuda")
    assert _call_static(_lib, plain, x, s) == 0, _lib.load().pat_last_error()
    torch.cuda.synchronize()
    assert _call_static(_lib, tc, x, s) == _lib.PAT_ERR_WORKSPACE
    assert b"K ld 4 bytes" in _lib.load().pat_last_error()
