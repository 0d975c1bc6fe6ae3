"""Pins of the oracle's whole operator A and adjoint A^T (Alg. 1, 3, 5, 7).

* Continuous model: for one voxel in front of a planar element, with a box
  EIR and the bump radial function, the exact sampled signal
  s[l] = F_s int_{t_l}^{t_{l+1}} int_Sigma h(t - r(x)/c) / r(x) dsigma dt
  (Prop. 1 with Eq. measurement and Eq. def_operatorS) is computed here with a
  dense midpoint rule over the element and exact time antiderivatives of h.
  The oracle's surface method must converge to it as O(1/U) (Prop. 3), and
  the point method must approach it as Q grows (Prop. 2).  A wrong factor
  (U F_s, 1/(c tau), 1/U, J0) or a shifted index cannot pass.
* <A x, y> = <x, A^T y> to rounding (App. G), for planes and cylinders, both
  methods and both area steps.
* Invariance under a common translation or a 90-degree rotation of grid and
  transducers (the model only depends on relative positions, Sec. 4).
"""
import math

import numpy as np
import pytest

from paper_2609_29253_gb300 import workloads as W

sp = pytest.importorskip("sympy")


def _bump_P1():
    """gamma1(u) with P1(y) = int_{-inf}^y G = c K^3 gamma1(y/K) on |y| <= K,
    K = kappa/c, where G = int g and g(s) = -1/2 c s (1 - (s/K)^2)^2."""
    u, s = sp.symbols("u s")
    gam = sp.integrate(-sp.Rational(1, 2) * s * (1 - s ** 2) ** 2, (s, -1, u))
    g1 = sp.integrate(gam.subs(u, s), (s, -1, u))
    return sp.lambdify(u, g1, "numpy"), float(g1.subs(u, 1))


G1, G1_END = _bump_P1()


def continuous_signal(row, xi, c, kappa, te, fs, t0, L, M=700):
    """Exact-in-time, dense-in-space sampled signal of one unit voxel."""
    K = kappa / c

    def P1(y):
        u = np.clip(y / K, -1.0, 1.0)
        out = c * K ** 3 * G1(u)
        out = np.where(y >= K, c * K ** 3 * G1_END, out)
        return np.where(y <= -K, 0.0, out)

    def H1(y):  # int_{-inf}^y h, h = e * g with e = 1 on [0, te]
        return P1(y) - P1(y - te)

    c0, e1, e2 = row[1:4], row[4:7], row[7:10]
    L1, L2 = row[10], row[11]
    g1 = -L1 + (np.arange(M) + 0.5) * 2 * L1 / M
    g2 = -L2 + (np.arange(M) + 0.5) * 2 * L2 / M
    P = c0[None, None, :] + g1[:, None, None] * e1[None, None, :] + g2[None, :, None] * e2[None, None, :]
    r = np.linalg.norm(P - xi[None, None, :], axis=2).ravel()
    dq = (2 * L1 / M) * (2 * L2 / M)
    tl = t0 + np.arange(L + 1) / fs
    out = np.zeros(L)
    for l in range(L):
        out[l] = fs * np.sum(dq / r * (H1(tl[l + 1] - r / c) - H1(tl[l] - r / c)))
    return out


def _one_voxel_workload(U, method=W.METHOD_SURFACE, q=(0, 0), dl=1):
    c, fs, t0, L = 1500.0, 40e6, 5.0e-6, 128
    kappa, te = 0.15e-3, 0.7e-6
    n_lo, T = W.tap_window(kappa, c, fs, U, te)
    p = np.array([0.2e-3, -1.0e-3, 9.0e-3])
    e1, e2 = W.facing_frame(p)
    row = W.plane_row(p, e1, e2, 0.5e-3, 0.4e-3)
    w = W.Workload(name="one voxel", n=(1, 1, 1), origin=np.array([0.1e-3, 0.05e-3, -0.2e-3]), pitch=0.1e-3,
                   tx=row[None, :], c=c, fs=fs, t0=t0, L=L, U=U, dl=dl, rbf_kind=W.RBF_BUMP, kappa=kappa,
                   eir_kind=W.EIR_BOX, eir_par=np.array([1.0, 0, 0, te]), n_lo=n_lo, T=T, method=method,
                   q1=q[0], q2=q[1], x=np.ones(1, dtype=np.float32))
    return w


@pytest.fixture(scope="module")
def cont_ref():
    w = _one_voxel_workload(11)
    return continuous_signal(w.tx[0], w.origin, w.c, w.kappa, w.eir_par[3], w.fs, w.t0, w.L)


def test_surface_method_converges_to_continuous_model(oracle_mod, cont_ref):
    errs = []
    for U in (5, 11, 41):
        w = _one_voxel_workload(U)
        s, d = oracle_mod.forward(w, oracle_mod.taps_for(w), np.ones(1))
        assert d == 0
        errs.append(np.abs(s[0] - cont_ref).max() / np.abs(cont_ref).max())
    # Prop. 3: error O(1 / U)
    assert errs[1] < 0.03
    assert errs[2] < errs[1] * 0.5
    assert errs[1] < errs[0] * 0.8
    assert errs[2] < 0.01


def test_point_method_converges_to_continuous_model(oracle_mod, cont_ref):
    errs = []
    for q in (4, 16, 64):
        w = _one_voxel_workload(41, W.METHOD_POINT, (q, q))
        s, d = oracle_mod.forward(w, oracle_mod.taps_for(w), np.ones(1))
        errs.append(np.abs(s[0] - cont_ref).max() / np.abs(cont_ref).max())
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.02


def test_point_method_converges_to_surface_method(oracle_mod):
    """Same U: the point method's f tends to the surface method's areas as Q grows."""
    w = W.c1(dl=1)
    taps = oracle_mod.taps_for(w)
    x = w.x.astype(np.float64)
    ref, _ = oracle_mod.forward(w, taps, x)
    errs = []
    for q in (8, 32):
        wp = w.with_(method=W.METHOD_POINT, q1=q, q2=q)
        s, _ = oracle_mod.forward(wp, taps, x)
        errs.append(np.linalg.norm(s - ref) / np.linalg.norm(ref))
    assert errs[1] < errs[0] * 0.5
    assert errs[1] < 5e-3


def _dot_case(oracle_mod, w, seed=0):
    rng = np.random.default_rng(seed)
    taps = oracle_mod.taps_for(w)
    x = rng.standard_normal(w.N)
    s, _ = oracle_mod.forward(w, taps, x)
    y = rng.standard_normal(s.shape)
    z, _ = oracle_mod.adjoint(w, taps, y)
    lhs, rhs = float((s * y).sum()), float((x * z).sum())
    scale = np.linalg.norm(s) * np.linalg.norm(y)
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)


@pytest.mark.parametrize("dl", [1, 11])
def test_dot_product_plane(oracle_mod, dl):
    w = W.c1(dl=dl).with_(n=(8, 8, 8), origin=W.centred_origin((8, 8, 8), 0.1e-3))
    _dot_case(oracle_mod, w)


def test_dot_product_point(oracle_mod):
    w = W.c1(method=W.METHOD_POINT, q=(8, 8)).with_(n=(8, 8, 8), origin=W.centred_origin((8, 8, 8), 0.1e-3))
    _dot_case(oracle_mod, w)


@pytest.mark.parametrize("dl", [1, 11])
def test_dot_product_cylinder(oracle_mod, dl):
    w = W.small_cylinder(n_vox=6, n_angles=3, n_el=2, dl=dl)
    _dot_case(oracle_mod, w)


def test_translation_invariance(oracle_mod):
    w = W.small_cylinder(n_vox=6, n_angles=2, n_el=2)
    taps = oracle_mod.taps_for(w)
    x = w.x.astype(np.float64)
    s0, _ = oracle_mod.forward(w, taps, x)
    d = np.array([0.31e-3, -0.22e-3, 0.13e-3])
    tx = w.tx.copy()
    tx[:, 1:4] += d
    s1, _ = oracle_mod.forward(w.with_(origin=w.origin + d, tx=tx), taps, x)
    assert np.abs(s1 - s0).max() <= 1e-9 * np.abs(s0).max()


def test_rotation_invariance(oracle_mod):
    w = W.c1().with_(n=(8, 8, 8), origin=W.centred_origin((8, 8, 8), 0.1e-3))
    w = w.with_(x=W.uniform_phantom(512, 3))
    taps = oracle_mod.taps_for(w)
    x = w.x.astype(np.float64)
    s0, _ = oracle_mod.forward(w, taps, x)
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    tx = w.tx.copy()
    for a in (1, 4, 7):
        tx[:, a:a + 3] = tx[:, a:a + 3] @ Rz.T
    n = 8
    xr = np.zeros((n, n, n))
    x3 = x.reshape(n, n, n)  # [iz, iy, ix]
    for iy in range(n):
        for ix in range(n):
            xr[:, ix, n - 1 - iy] = x3[:, iy, ix]  # (x, y) -> (-y, x)
    s1, _ = oracle_mod.forward(w.with_(tx=tx), taps, xr.ravel())
    assert np.abs(s1 - s0).max() <= 1e-9 * np.abs(s0).max()


def test_linearity(oracle_mod):
    w = W.c1().with_(n=(6, 6, 6), origin=W.centred_origin((6, 6, 6), 0.1e-3))
    taps = oracle_mod.taps_for(w)
    rng = np.random.default_rng(9)
    a, b = rng.standard_normal(216), rng.standard_normal(216)
    sa, _ = oracle_mod.forward(w, taps, a)
    sb, _ = oracle_mod.forward(w, taps, b)
    sab, _ = oracle_mod.forward(w, taps, 2.5 * a - b)
    assert np.abs(sab - (2.5 * sa - sb)).max() <= 1e-12 * np.abs(sab).max()


# ---------------------------------------------------------------------------
# Cylinder branch of the point method (Alg. 2 on the cylinder of
# Eq. cylinder_param, Sec. 4.2.1): its points must lie on the element and
# its areas must integrate known functions over the surface exactly (up to
# the midpoint rule's O(h^2)); the whole point operator must then converge
# to the surface method's (Prop. 2).
# ---------------------------------------------------------------------------
def _tilted_cylinder_row():
    rng = np.random.default_rng(3)
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    e1, e2 = q[:, 0], q[:, 1]
    return W.cylinder_row(np.array([1.1e-3, -0.4e-3, 0.7e-3]), e1, e2, 20e-3, math.asin(0.25), 0.15e-3)


def test_cylinder_points_lie_on_the_element(oracle_mod):
    row = _tilted_cylinder_row()
    c0, e1 = row[1:4], row[4:7]
    R, thmax, Lz = row[12], row[13], row[14]
    pts, dq = oracle_mod.quad_points(row, 12, 5)
    d = pts - c0
    along = d @ e1
    radial = d - along[:, None] * e1[None, :]
    # every point on the cylinder of radius R about the line c0 + t e1, within the strip
    assert np.abs(np.linalg.norm(radial, axis=1) - R).max() <= 1e-15 * R * 10
    assert np.abs(along).max() < Lz
    # the angular aperture: the points' directions from the axis stay within
    # theta_max of the element's centre direction e2
    e2 = row[7:10]
    cosang = radial @ e2 / R
    assert cosang.min() > math.cos(thmax)
    # the total area is the element's, R 2 theta_max 2 Lz
    assert dq.sum() == pytest.approx(R * 2 * thmax * 2 * Lz, rel=1e-14)
    assert np.all(dq > 0)


@pytest.mark.parametrize("q", [(16, 4), (64, 16)])
def test_cylinder_points_integrate_exactly(oracle_mod, q):
    """Sum dq f(q_j) against closed-form surface integrals: the midpoint rule
    is exact for functions affine in the angle and the height, and second
    order otherwise."""
    row = _tilted_cylinder_row()
    c0, e1, e2 = row[1:4], row[4:7], row[7:10]
    R, thmax, Lz = row[12], row[13], row[14]
    pts, dq = oracle_mod.quad_points(row, *q)
    d = pts - c0
    along = d @ e1
    radial = d - along[:, None] * e1[None, :]
    # angle about the axis measured from e2 in the plane normal to e1
    n = np.cross(e1, e2)
    ang = np.arctan2(radial @ n, radial @ e2)
    h1, h2 = 2 * thmax / q[0], 2 * Lz / q[1]
    # f = angle + height: odd on the symmetric element, integral 0
    assert abs(np.sum(dq * (ang + along / Lz))) <= 1e-12 * R * thmax * Lz
    # f = along^2: exact R 2 theta_max (2/3) Lz^3; the midpoint rule is short by R 2 theta_max 2 Lz h2^2 / 12
    exact = R * 2 * thmax * (2.0 / 3.0) * Lz ** 3
    mid = exact - R * 2 * thmax * 2 * Lz * h2 ** 2 / 12
    assert np.sum(dq * along ** 2) == pytest.approx(mid, rel=1e-12)
    # f = (x - c0) . e2 = R cos(angle): exact 2 R^2 sin(theta_max) 2 Lz; the
    # midpoint rule for cos on q1 cells gives the closed form below
    exact_cos = 2 * R * R * math.sin(thmax) * 2 * Lz
    mid_cos = R * R * 2 * Lz * h1 * sum(math.cos(-thmax + (j + 0.5) * h1) for j in range(q[0]))
    assert np.sum(dq * (d @ e2)) == pytest.approx(mid_cos, rel=1e-12)
    assert mid_cos == pytest.approx(exact_cos, rel=h1 ** 2)


def test_cylinder_point_method_converges_to_surface_method(oracle_mod):
    """Prop. 2 on the cylinder: at the same U, the point method's signals
    approach the surface method's as Q grows, at about the Q^-1 rate."""
    w = W.small_cylinder(n_vox=6, n_angles=2, n_el=2, dl=1)
    taps = oracle_mod.taps_for(w)
    x = w.x.astype(np.float64)
    ref, _ = oracle_mod.forward(w, taps, x)
    errs = []
    for q in (4, 8, 16, 32):
        wp = w.with_(method=W.METHOD_POINT, q1=q, q2=q)
        s, _ = oracle_mod.forward(wp, taps, x)
        errs.append(np.linalg.norm(s - ref) / np.linalg.norm(ref))
    # Q grows 4x per step: the quadrature term of Prop. 2 falls 4x (measured
    # 4.2x and 3.9x), until the O(1 / (U F_s)) term, the binning of each
    # point's 1/r against the surface method's 1/(c tau), is reached at
    # Q = 32^2 (2.3e-4 at U = 11)
    assert errs[1] < 0.3 * errs[0], errs
    assert errs[2] < 0.3 * errs[1], errs
    assert errs[3] < errs[2] and errs[3] < 5e-4, errs
