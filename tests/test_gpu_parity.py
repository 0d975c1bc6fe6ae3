"""GPU parity of the CUDA library against the FP64 oracle, through the C ABI.

Bars (rel L2 = |y - y_ref| / |y_ref| over the whole output):
  * surface method (closed-form areas), FP32: 1e-5 on s = A x and on
    z = A^T s, and on every stage (f, conv, correlation, gather);
  * point method: 5e-5 on s, because FP32 and FP64 distances put a
    contribution on different sides of a bin edge for a few points
    (flip-tolerant bound);
  * system kernel taps (device FP64 quadrature): 1e-12 of max |h-bar|;
  * dot-product test of the GPU pair (A, A^T): 1e-5.
Inputs are the seeded workloads; x is rounded to float32 once and the same
values feed both sides.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2609_29253_gb300 import workloads as W  # noqa: E402

SURF_TOL = 1e-5
POINT_TOL = 5e-5


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


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod


def _run(api, orc, w, check_stages=True, tol=SURF_TOL):
    taps = orc.taps_for(w)
    plan = api.Plan(w, taps=taps)
    x32 = w.x.astype(np.float32)
    xg = torch.from_numpy(x32).cuda()
    s = plan.forward(xg).cpu().numpy()
    s_ref, _ = orc.forward(w, taps, x32.astype(np.float64))
    assert rel(s, s_ref) <= tol, rel(s, s_ref)
    rng = np.random.default_rng(11)
    y = rng.standard_normal(s.shape).astype(np.float32)
    z = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    z_ref, _ = orc.adjoint(w, taps, y.astype(np.float64))
    assert rel(z, z_ref) <= tol, rel(z, z_ref)
    if check_stages:
        f = plan.forward_geometric(xg).cpu().numpy()
        f_ref, _ = orc.geometric_forward(w, x32.astype(np.float64))
        assert rel(f, f_ref) <= tol, rel(f, f_ref)
        s2 = plan.conv_forward(torch.from_numpy(f_ref.astype(np.float32)).cuda()).cpu().numpy()
        s2_ref = orc.conv_forward(w, taps, f_ref.astype(np.float32).astype(np.float64))
        assert rel(s2, s2_ref) <= 1e-6
        v = plan.conv_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
        v_ref = orc.conv_adjoint(w, taps, y.astype(np.float64))
        assert rel(v, v_ref) <= 1e-6
        z2 = plan.adjoint_geometric(torch.from_numpy(v_ref.astype(np.float32)).cuda()).cpu().numpy()
        z2_ref, _ = orc.geometric_adjoint(w, v_ref.astype(np.float32).astype(np.float64))
        assert rel(z2, z2_ref) <= tol, rel(z2, z2_ref)
    return plan, s, s_ref


def test_system_kernel_taps(api, orc):
    for w in (W.c1(), W.c2(n_angles=1, with_x=False)):
        t = api.system_taps(w)
        t_ref = orc.taps_for(w)
        assert np.abs(t - t_ref).max() <= 1e-12 * np.abs(t_ref).max()


@pytest.mark.parametrize("dl", [1, 11])
def test_plane_surface(api, orc, dl):
    _run(api, orc, W.c1(dl=dl))


def test_plane_point(api, orc):
    _run(api, orc, W.c1(method=W.METHOD_POINT, q=(16, 16)), tol=POINT_TOL)


@pytest.mark.parametrize("dl", [1, 11])
def test_cylinder_surface(api, orc, dl):
    _run(api, orc, W.small_cylinder(n_vox=12, n_angles=4, n_el=3, dl=dl))


@pytest.mark.parametrize("dl", [1, 11])
def test_cylinder_trapezoid(api, orc, dl):
    """The trapezoidal arc integral (Eq. trapezoid_Il) against the oracle's
    own trapezoidal areas, all stages, and its distance to the exact areas."""
    w = W.small_cylinder(n_vox=12, n_angles=4, n_el=3, dl=dl).with_(method=W.METHOD_TRAPEZOID)
    _, s, s_ref = _run(api, orc, w)
    s_ex, _ = orc.forward(w.with_(method=W.METHOD_SURFACE), orc.taps_for(w), w.x.astype(np.float32).astype(np.float64))
    assert 0.0 < rel(s_ref, s_ex) < 0.2


@pytest.mark.parametrize("dl,lut", [(1, (1000, 1000)), (11, (1000, 1000)), (11, (181, 263))])
def test_cylinder_lut(api, orc, dl, lut):
    """The paper's lookup tables (Sec. 4.2.2) against the oracle's own LUT
    areas, all stages: the paper's 1000 x 1000 tables, and small non-square
    ones (other cells, other index inversions); and the distance of the LUT
    operator to the exact one."""
    w = W.small_cylinder(n_vox=12, n_angles=4, n_el=3, dl=dl).with_(method=W.METHOD_LUT, q1=lut[0], q2=lut[1])
    _, s, s_ref = _run(api, orc, w)
    s_ex, _ = orc.forward(w.with_(method=W.METHOD_SURFACE, q1=0, q2=0), orc.taps_for(w),
                          w.x.astype(np.float32).astype(np.float64))
    assert 0.0 < rel(s_ref, s_ex) < 0.05


def _axis_rows(n_az=4, zc=(-1.3e-3, 0.0, 2.1e-3)):
    """Cylinders focused on the z axis (focal line = z axis), frames built from
    exact unit vectors, so that voxels on the axis have rho = 0 exactly."""
    a = W.C2_ARRAY
    e2s = [np.array(v, dtype=float) for v in ((1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0))][:n_az]
    return np.array([W.cylinder_row(np.array([0.0, 0.0, z]), np.array([0.0, 0.0, 1.0]), e2, a["R"], a["theta_max"],
                                    a["Lz"]) for z in zc for e2 in e2s])


def test_lut_on_the_focal_line(api, orc):
    """Voxels exactly on the focal line (rho = 0: E is never read) and next to
    it, LUT against the oracle's LUT."""
    n, pitch = 7, 2.0 ** -13  # exact pitch: the centre column lies on the axis in FP64 and in float-float
    w = W.small_cylinder(n_vox=n).with_tx(_axis_rows())
    w = w.with_(pitch=pitch, origin=W.centred_origin((n, n, n), pitch), t0=5.00037e-6, L=2048,
                method=W.METHOD_LUT, q1=1000, q2=1000)
    _run(api, orc, w, check_stages=False)


def test_lut_c2_geometry_reduced(api, orc):
    """The c2 element and rotation geometry on a coarse grid, LUT operator."""
    n = 16
    pitch = 12.8e-3 / n
    w = W.c2(angles=np.array([0.3, 1.7]), with_x=False)
    w = w.with_tx(w.tx[np.arange(0, 256, 8)]).with_(n=(n, n, n), pitch=pitch, origin=W.centred_origin((n, n, n), pitch))
    w = w.with_(x=W.blob_phantom(w.n, w.origin, pitch, 30, 1, sigma=(0.4e-3, 1.2e-3)), method=W.METHOD_LUT, q1=1000,
                q2=1000)
    _run(api, orc, w, check_stages=False)


@pytest.mark.parametrize("n_planes", [1, 8, 30])
def test_cylinder_piecewise_planes(api, orc, n_planes):
    """Piecewise-Planes (Sec. 4.3): the library's own tangent-plane expansion
    against the oracle's, A and A^T, each plane's signal summed into its
    element's row."""
    w = W.small_cylinder(n_vox=9, n_angles=3, n_el=2)
    taps = orc.taps_for(w)
    plan = api.Plan(w, taps=taps, piecewise_planes=n_planes)
    x32 = w.x.astype(np.float32)
    s = plan.forward(torch.from_numpy(x32).cuda()).cpu().numpy()
    s_ref, _ = orc.piecewise_planes_forward(w, taps, x32.astype(np.float64), n_planes)
    assert rel(s, s_ref) <= SURF_TOL, rel(s, s_ref)
    y = np.random.default_rng(6).standard_normal(s.shape).astype(np.float32)
    z = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    z_ref, _ = orc.piecewise_planes_adjoint(w, taps, y.astype(np.float64), n_planes)
    assert rel(z, z_ref) <= SURF_TOL, rel(z, z_ref)
    if n_planes == 30:  # the approximation itself, against the exact cylinder
        s_ex, _ = orc.forward(w, taps, x32.astype(np.float64))
        assert rel(s_ref, s_ex) < 0.2


def test_cylinder_point(api, orc):
    w = W.small_cylinder(n_vox=8, n_angles=3, n_el=2)
    _run(api, orc, w.with_(method=W.METHOD_POINT, q1=16, q2=4), tol=POINT_TOL)


def test_ragged_grid_and_many_tiles(api, orc):
    """Grid sizes that are not multiples of the 4x4x2 brick, several CTAs."""
    w = W.c1().with_(n=(13, 7, 5), origin=W.centred_origin((13, 7, 5), 0.1e-3))
    w = w.with_(x=W.uniform_phantom(13 * 7 * 5, 4))
    _run(api, orc, w)
    w2 = W.small_cylinder(n_vox=9, n_angles=2, n_el=2).with_(n=(9, 5, 11), origin=W.centred_origin((9, 5, 11), 0.1e-3))
    w2 = w2.with_(x=W.uniform_phantom(9 * 5 * 11, 5))
    _run(api, orc, w2)


def test_super_tiles_cut_off_in_every_axis(api, orc):
    """A grid of 2 x 2 x 2 forward super-tiles (32 x 32 x 16 voxels each)
    that the grid cuts off in every axis, cylinders and planes; the cylinder
    plan again after the autotuner has timed its forward chunkings.  As in
    the focal-line test, t0 is off the round values, so that no pair's r_min
    or r_max ties with a bin edge (the odd grid puts voxels on the focal
    line); the planes get the time window that holds all their pairs."""
    n = (37, 45, 21)
    w = W.small_cylinder(n_vox=8, n_angles=2, n_el=2).with_(n=n, origin=W.centred_origin(n, 0.1e-3), t0=6.00037e-6)
    w = w.with_(x=W.uniform_phantom(math.prod(n), 6))
    plan, _, s_ref = _run(api, orc, w, check_stages=False)
    x = torch.from_numpy(w.x.astype(np.float32)).cuda()
    shapes = plan.autotune(x)
    assert shapes["fwd_blocks"] % w.K == 0
    assert rel(plan.forward(x).cpu().numpy(), s_ref) <= SURF_TOL
    wp = W.c1().with_(n=n, origin=W.centred_origin(n, 0.1e-3), t0=4.00037e-6, L=512)
    _run(api, orc, wp.with_(x=W.uniform_phantom(math.prod(n), 7)), check_stages=False)


def test_more_elements_than_a_grid_dimension_holds(api, orc):
    """66,560 cylindrical positions, more than the 65,535 blocks of a CUDA
    grid's y or z extent, on a 2 x 2 x 2 grid: the forward chunks and the
    scan are indexed along one grid dimension.  Three rows of s against the
    oracle, one from each end and one from the middle."""
    a = W.C2_ARRAY
    tx = W.rotated_linear_cylinder_array(a["n_el"], a["el_pitch"], a["R"], a["theta_max"], a["Lz"], 520)
    n = (2, 2, 2)
    w = W.c2(angles=np.array([0.0]), with_x=False).with_tx(tx)
    w = w.with_(n=n, origin=W.centred_origin(n, 0.1e-3), t0=6.00037e-6, x=W.uniform_phantom(8, 3))
    assert w.K > 65535
    taps = orc.taps_for(w)
    plan = api.Plan(w, taps=taps)
    x32 = w.x.astype(np.float32)
    s = plan.forward(torch.from_numpy(x32).cuda()).cpu().numpy()
    ks = [0, 40001, w.K - 1]
    s_ref = np.stack([orc.forward(w.with_tx(w.tx[k:k + 1]), taps, x32.astype(np.float64))[0][0] for k in ks])
    assert rel(s[ks], s_ref) <= SURF_TOL, rel(s[ks], s_ref)


def test_voxels_on_and_near_the_focal_line(api, orc):
    """An odd grid centred on the focal line (voxels at rho = 0 and, after the
    frame rotation by pi, at rho ~ 1e-19 m) seen by the whole 128-element
    array, whose end elements see the axis voxels under a near-flat level
    curve (both branch points inside one short piece).  t0 is set off the
    round value 5 us so that no pair's r_min or r_max falls within 1e-5 of
    a bin edge: with round numbers (R - rho = 19.8 mm at 5 us) some fall
    exactly on one, and the oracle (FP64) and the kernel (float-float) then
    round the tie to different bins, which moves the whole first group of
    Remark 1."""
    a = W.C2_ARRAY
    tx = W.rotated_linear_cylinder_array(a["n_el"], a["el_pitch"], a["R"], a["theta_max"], a["Lz"], 2)
    w = W.c2(angles=np.array([0.0]), with_x=False).with_tx(tx)
    n = 7
    w = w.with_(n=(n, n, n), origin=W.centred_origin((n, n, n), 0.1e-3), t0=5.00037e-6, L=2048)
    w = w.with_(x=W.uniform_phantom(n ** 3, 9))
    plan, s, s_ref = _run(api, orc, w, check_stages=False)
    assert np.isfinite(s).all()


def test_single_voxel_and_single_transducer(api, orc):
    w = W.c1().with_(n=(1, 1, 1), origin=np.array([0.05e-3, -0.02e-3, 0.01e-3]), x=np.array([0.7], dtype=np.float32))
    w = w.with_tx(w.tx[:1])
    _run(api, orc, w)


def test_c2_geometry_reduced(api, orc):
    """The full c2 element and rotation geometry on a coarser grid of the same
    extent (20^3 voxels over 12.8 mm), 64 positions."""
    n = 20
    pitch = 12.8e-3 / n
    w = W.c2(angles=np.array([0.0, 1.1]), with_x=False)
    sel = np.arange(0, 256, 4)
    w = w.with_tx(w.tx[sel]).with_(n=(n, n, n), pitch=pitch, origin=W.centred_origin((n, n, n), pitch))
    w = w.with_(x=W.blob_phantom(w.n, w.origin, pitch, 40, 0, sigma=(0.4e-3, 1.2e-3)))
    _run(api, orc, w, check_stages=False)


def test_dot_product_gpu(api, orc):
    w = W.small_cylinder(n_vox=12, n_angles=4, n_el=3)
    plan = api.Plan(w, taps=orc.taps_for(w))
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(w.N, device="cuda", generator=g)
    y = torch.randn(w.K, w.L, device="cuda", generator=g)
    lhs = float((plan.forward(x).double() * y.double()).sum())
    rhs = float((x.double() * plan.adjoint(y.contiguous()).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_clipping_matches_oracle(api, orc):
    """Bins before t0 are dropped on both sides when clipping is allowed."""
    w = W.c1().with_(t0=6.3e-6, L=200)
    taps = orc.taps_for(w)
    from paper_2609_29253_gb300._lib import PatError

    with pytest.raises(PatError, match="PAT_ERR_WINDOW"):
        api.Plan(w, taps=taps)
    plan = api.Plan(w, taps=taps, allow_clip=True)
    assert plan.info["clipped_pairs"] > 0
    x32 = w.x.astype(np.float32)
    s = plan.forward(torch.from_numpy(x32).cuda()).cpu().numpy()
    s_ref, dropped = orc.forward(w, taps, x32.astype(np.float64))
    assert dropped > 0
    assert rel(s, s_ref) <= SURF_TOL
    y = np.random.default_rng(2).standard_normal(s.shape).astype(np.float32)
    z = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    z_ref, _ = orc.adjoint(w, taps, y.astype(np.float64))
    assert rel(z, z_ref) <= SURF_TOL


def test_geometry_error(api, orc):
    from paper_2609_29253_gb300._lib import PatError

    w = W.c1()
    tx = w.tx.copy()
    tx[0, 1:4] = np.array([0.0, 0.0, 0.8e-3])  # element inside the grid
    with pytest.raises(PatError, match="PAT_ERR_GEOMETRY"):
        api.Plan(w.with_tx(tx), taps=orc.taps_for(w))


def test_autograd_backward_is_adjoint(api, orc):
    w = W.c1()
    plan = api.Plan(w, taps=orc.taps_for(w))
    x = torch.from_numpy(w.x).cuda().requires_grad_(True)
    s = api.forward(plan, x)
    g = torch.randn_like(s)
    (s * g).sum().backward()
    z = plan.adjoint(g.contiguous())
    assert torch.allclose(x.grad, z)


def test_recon_decreases_objective(api, orc):
    w = W.c1().with_(n=(8, 8, 8), origin=W.centred_origin((8, 8, 8), 0.1e-3))
    plan = api.Plan(w, taps=orc.taps_for(w))
    xt = torch.from_numpy(W.uniform_phantom(512, 7)).cuda()
    s = plan.forward(xt)
    lam = 0.0

    def obj(x):
        r = plan.forward(x) - s
        return float(0.5 * (r.double() ** 2).sum() + 0.5 * lam * (x.double() ** 2).sum())

    x0 = torch.zeros(512, device="cuda")
    x5 = plan.recon(s, x0, iters=5, lambda_R=lam)
    x40 = plan.recon(s, x0, iters=40, lambda_R=lam)
    assert float(x40.min()) >= 0.0
    assert obj(x40) < obj(x5) < obj(x0)


@pytest.mark.parametrize("value", [float("nan"), float("inf")])
def test_non_finite_voxel_propagates(api, orc, value):
    """A NaN or infinite voxel value reaches the output as in FP64 arithmetic,
    on the cylinder forward (whose window is in fixed point) and on planes;
    the other outputs of a plan with finite x stay finite."""
    for w in (W.small_cylinder(n_vox=8, n_angles=2, n_el=3), W.c1().with_(n=(8, 8, 8), origin=W.centred_origin((8, 8, 8), 0.1e-3))):
        plan = api.Plan(w, taps=orc.taps_for(w))
        x = torch.rand(w.N, device="cuda", generator=torch.Generator(device="cuda").manual_seed(2))
        assert bool(torch.isfinite(plan.forward(x)).all())
        x[w.N // 2] = value
        s = plan.forward(x)
        assert not bool(torch.isfinite(s).all())


@pytest.mark.parametrize("k", [1e-22, 1e-12, 1e12, 1e22])
def test_forward_linearity_extreme_scales(api, orc, k):
    """A_geo (k x) = k A_geo x at extreme scales of x, on the cylinder forward
    (its window in fixed point with per-CTA scales from max |x|; for this
    element, 12.8 R Lz = 3.8e-5, a single FP32 power of two would overflow
    below max |x| = 1e-20) and on planes.  Compared on the fine-bin rows f
    (areas of order 1e-10..1e-8 per unit x), whose scaled values stay normal
    FP32 numbers; the convolved outputs are about 1e-16 per unit x and would
    underflow FP32 at the smallest k on any path."""
    for w in (W.small_cylinder(n_vox=8, n_angles=2, n_el=3), W.c1().with_(n=(8, 8, 8), origin=W.centred_origin((8, 8, 8), 0.1e-3))):
        plan = api.Plan(w, taps=orc.taps_for(w))
        x = torch.rand(w.N, device="cuda", generator=torch.Generator(device="cuda").manual_seed(4))
        f1 = plan.forward_geometric(x).double()
        fk = plan.forward_geometric(x * k).double() / k
        assert float(f1.norm()) > 0.0
        rel = float((fk - f1).norm() / f1.norm())
        assert rel <= 1e-6, (w.name, rel)
