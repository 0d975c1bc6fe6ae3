"""Speed-of-sound derivative of the forward operator on the GPU against
central finite differences of the FP64 oracle, through the C ABI.

c enters the operator through the bin radii r = c tau (the swept areas),
the weights U Fs / (c tau) of Eq. ui_area and the system kernel h-bar
(Eq. def_bh).  The bins of every pair (l_min, l_max of Eq. rmin_rmax, and
with dl > 1 the phase of the groups of Remark 1) change with c in discrete
steps, so the operator is piecewise smooth in c; the derivative is taken
between such steps.  Each test chooses its step eps so that no pair's bins
differ between c - eps, c and c + eps (checked pair by pair with the
oracle's distances), then compares

    pat_forward_dc   with   (A(c + eps) x - A(c - eps) x) / (2 eps)

and the gradient of a least-squares loss through torch.autograd with the
same difference of the oracle's loss.  x is sparse (a few seeded voxels), so
that few pairs constrain eps.  The quotient's own error has two sources:
the oracle's rounding (about 1e-14 of an element's area, divided by 2 eps),
which dominates for the plane, whose literal primitive loses digits when a
bound lies on the circle, so the plane cases take the largest safe eps; and
truncation where A'(r) has a square-root singularity (near r_min and r_max),
which dominates for the cylinder with dl = 1, whose bins resolve it, so that
case takes eps / 64.  Bounds (rel L2): 1e-3 for the plane with dl = 1 (the
quotient itself is good to about 2e-4 there), 2e-4 otherwise and for the
scalar gradient.  d h-bar / dc (device FP64 quadrature) against the
difference quotient of the oracle's taps: 1e-8 of its maximum.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2609_29253_gb300 import workloads as W  # noqa: E402

DC_TOL = {("plane", 1): 1e-3, ("plane", 11): 2e-4, ("cylinder", 1): 2e-4, ("cylinder", 11): 2e-4,
          ("cylinder_tiles", 11): 2e-4}
EPS_SCALE = {("plane", 1): 1.0, ("plane", 11): 1.0, ("cylinder", 1): 1 / 64, ("cylinder", 11): 1.0,
             ("cylinder_tiles", 11): 1.0}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_29253_gb300 import api as A

    return A


def _sparse(w, n_vox, seed):
    """x with n_vox seeded nonzero voxels (values in [0.5, 1))."""
    rng = np.random.default_rng(seed)
    x = np.zeros(w.N, dtype=np.float32)
    x[rng.choice(w.N, n_vox, replace=False)] = rng.uniform(0.5, 1.0, n_vox)
    return w.with_(x=x)


def _bins(orc, w, c):
    """(l_min, l_max) of every pair with x_i != 0 at speed of sound c (Eq. rmin_rmax)."""
    idx = np.flatnonzero(w.x)
    xs = W.voxel_centres(w.n, w.origin, w.pitch, idx)
    ufs = w.U * w.fs
    out = []
    for row in w.tx:
        for xi in xs:
            rmin, rmax, _ = orc.pair_range(row, xi)
            out.append((math.floor((rmin / c - w.t0) * ufs), math.ceil((rmax / c - w.t0) * ufs) - 1))
    return out


def _safe_eps(orc, w, eps=2e-3):
    b0 = _bins(orc, w, w.c)
    for _ in range(30):
        if _bins(orc, w, w.c + eps) == b0 and _bins(orc, w, w.c - eps) == b0:
            return eps
        eps *= 0.5
    pytest.fail("no step keeps every pair's bins")


def _oracle_s(orc, w, c, x):
    wc = w.with_(c=c)
    s, _ = orc.forward(wc, orc.taps_for(wc), x)
    return s


def test_system_kernel_dc(api, oracle_mod):
    for w in (W.c1(), W.small_cylinder(n_vox=4)):
        d = api.system_taps_dc(w).cpu().numpy()
        eps = 1e-2
        fd = (oracle_mod.taps_for(w.with_(c=w.c + eps)) - oracle_mod.taps_for(w.with_(c=w.c - eps))) / (2 * eps)
        assert np.abs(d - fd).max() <= 1e-8 * np.abs(fd).max(), np.abs(d - fd).max() / np.abs(fd).max()


@pytest.mark.parametrize("kind,dl", [("plane", 1), ("plane", 11), ("cylinder", 1), ("cylinder", 11),
                                     ("cylinder_tiles", 11)])
def test_forward_dc_matches_finite_differences(api, oracle_mod, kind, dl):
    """cylinder_tiles: a grid of 2 x 2 x 2 forward super-tiles, cut off in
    every axis (the derivative kernel's chunks and windows)."""
    if kind == "plane":
        w = W.c1(dl=dl).with_(n=(8, 8, 8), origin=W.centred_origin((8, 8, 8), 0.1e-3))
    elif kind == "cylinder":
        w = W.small_cylinder(n_vox=8, n_angles=3, n_el=3, dl=dl)
    else:
        n = (37, 45, 21)
        w = W.small_cylinder(n_vox=8, n_angles=3, n_el=3, dl=dl).with_(n=n, origin=W.centred_origin(n, 0.1e-3))
    w = _sparse(w, 12, seed=dl)
    eps = _safe_eps(oracle_mod, w) * EPS_SCALE[(kind, dl)]
    x32 = w.x.astype(np.float32)
    plan = api.Plan(w, taps=oracle_mod.taps_for(w))
    ds = plan.forward_dc(torch.from_numpy(x32).cuda()).cpu().numpy()
    x64 = x32.astype(np.float64)
    fd = (_oracle_s(oracle_mod, w, w.c + eps, x64) - _oracle_s(oracle_mod, w, w.c - eps, x64)) / (2 * eps)
    e = rel(ds, fd)
    print(f"{kind} dl={dl} eps={eps:.2e} rel L2 {e:.3e}")
    assert e <= DC_TOL[(kind, dl)], e


def test_autograd_speed_of_sound_gradient(api, oracle_mod):
    w = _sparse(W.small_cylinder(n_vox=8, n_angles=3, n_el=3, dl=11), 12, seed=3)
    eps = _safe_eps(oracle_mod, w)
    taps = oracle_mod.taps_for(w)
    plan = api.Plan(w, taps=taps)
    x32 = w.x.astype(np.float32)
    rng = np.random.default_rng(4)
    s0, _ = oracle_mod.forward(w, taps, x32.astype(np.float64))
    y = (s0 + 0.1 * np.abs(s0).max() * rng.standard_normal(s0.shape)).astype(np.float32)
    x = torch.from_numpy(x32).cuda().requires_grad_(True)
    c = torch.tensor(w.c, dtype=torch.float64, requires_grad=True)
    s = api.forward(plan, x, c)
    loss = 0.5 * ((s.double() - torch.from_numpy(y).cuda().double()) ** 2).sum()
    loss.backward()

    def oloss(cc):
        sc = _oracle_s(oracle_mod, w, cc, x32.astype(np.float64))
        return 0.5 * float(((sc - y.astype(np.float64)) ** 2).sum())

    g_fd = (oloss(w.c + eps) - oloss(w.c - eps)) / (2 * eps)
    g = float(c.grad)
    print(f"dloss/dc GPU {g:.6e} oracle FD {g_fd:.6e}")
    assert abs(g - g_fd) <= DC_TOL[("cylinder", 11)] * abs(g_fd)
    # the x-gradient is A^T (A x - y)
    gx = plan.adjoint((s.detach() - torch.from_numpy(y).cuda()).contiguous())
    assert torch.allclose(x.grad, gx, rtol=1e-4, atol=1e-6 * float(gx.abs().max()))


def test_forward_dc_c2_full_grid(api, oracle_mod):
    """The same check on the c2 system itself: the full 128^3 grid at 0.1 mm,
    the 128-element cylindrical array at U 11, dl 11, eight positions from
    two rotation angles (elements near both ends and the middle of the
    array), x with 12 seeded voxels anywhere in the grid."""
    w = W.c2(angles=[0.0, 37 * 2 * math.pi / 180], with_x=False)
    w = w.with_tx(w.tx[[3, 50, 90, 127, 128 + 10, 128 + 64, 128 + 100, 128 + 121]])
    w = _sparse(w, 12, seed=21)
    eps = _safe_eps(oracle_mod, w)
    x32 = w.x.astype(np.float32)
    plan = api.Plan(w, taps=oracle_mod.taps_for(w))
    ds = plan.forward_dc(torch.from_numpy(x32).cuda()).cpu().numpy()
    x64 = x32.astype(np.float64)
    fd = (_oracle_s(oracle_mod, w, w.c + eps, x64) - _oracle_s(oracle_mod, w, w.c - eps, x64)) / (2 * eps)
    e = rel(ds, fd)
    print(f"c2 full grid eps={eps:.2e} rel L2 {e:.3e}")
    assert e <= DC_TOL[("cylinder", 11)], e
