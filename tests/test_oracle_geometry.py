"""Pins of the oracle's swept areas |M_i^l| (Eq. def:bffi, Alg. 4, Sec. 4).

The reference here is the plain definition of the area, written from the 3-D
geometry and nothing else: for each abscissa along one side of the element
(x1 for a plane, theta for a cylinder) the length of the straight segment of
the element that lies within distance r of the voxel is a 1-D interval
computation, and the cumulative area |{x in Sigma : |x - x_i| < r}| is its
integral (Fubini), done by adaptive quadrature.  No separable form, quadrant,
clamp, primitive or elliptic function enters the reference, so a mistake in
any of them (a wrong fold, sign, clamp or branch) shows up as a mismatch.

Further pins: telescoped totals equal the element area, the on-axis piston
plateau f_i[l] = 2 pi c (Remark on the SIR), the focal-line cylinder formula,
Remark 1 (group areas are sums of fine areas), the bin range of
Eq. (rmin_rmax) against brute-force distances, and the limit R -> infinity of
a cylinder (its tangent plane).
"""
import math

import numpy as np
import pytest

from paper_2609_29253_gb300 import workloads as W

quad = pytest.importorskip("scipy.integrate").quad
brentq = pytest.importorskip("scipy.optimize").brentq


def _seg_len(h2, w1, half):
    """Length of {z in [-half, half] : (z - w1)^2 < h2}."""
    if h2 <= 0:
        return 0.0
    h = math.sqrt(h2)
    lo, hi = max(-half, w1 - h), min(half, w1 + h)
    return max(0.0, hi - lo)


def _element_slices(row):
    """For a descriptor, return (a, b, weight, base(t), axis, half) such that
    the element is { base(t) + z axis : t in [a, b], |z| <= half } with area
    element weight dt dz."""
    kind = int(row[0])
    c0, e1, e2 = row[1:4], row[4:7], row[7:10]
    n = np.cross(e1, e2)
    if kind == W.PLANE:
        L1, L2 = row[10], row[11]
        return -L1, L1, 1.0, (lambda t: c0 + t * e1), e2, L2
    R, thm, Lz = row[12], row[13], row[14]
    return -thm, thm, R, (lambda t: c0 + R * math.cos(t) * e2 + R * math.sin(t) * n), e1, Lz


def fubini_cumulative_area(row, xi, r):
    a, b, wgt, base, axis, half = _element_slices(row)

    def length(t):
        w = xi - base(t)
        w1 = float(w @ axis)
        A = float(w @ w) - w1 * w1
        return _seg_len(r * r - A, w1, half)

    # break points: where the disc boundary meets the segment ends or appears
    ts = np.linspace(a, b, 2001)

    def ev(t, s):
        w = xi - base(t)
        w1 = float(w @ axis)
        A = float(w @ w) - w1 * w1
        if s == 0:
            return r * r - A
        return r * r - A - (s * half - w1) ** 2

    pts = []
    for s in (0, -1, 1):
        vals = np.array([ev(t, s) for t in ts])
        for i in np.nonzero(np.sign(vals[:-1]) * np.sign(vals[1:]) < 0)[0]:
            pts.append(brentq(lambda t: ev(t, s), ts[i], ts[i + 1], xtol=1e-15))
    pts = sorted(set(pts))
    edges = [a] + [p for p in pts if a < p < b] + [b]
    tot = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        tot += quad(length, lo, hi, epsabs=1e-16, epsrel=1e-12, limit=400)[0]
    return wgt * tot


def element_area(row):
    if int(row[0]) == W.PLANE:
        return 4 * row[10] * row[11]
    return 4 * row[12] * row[13] * row[14]


def _cases():
    plane = W.fibonacci_planar(8, 10e-3, 0.5e-3, 0.7e-3)[3]
    cyl = W.rotated_linear_cylinder_array(1, 0.3e-3, 20e-3, math.asin(0.25), 0.15e-3, 1, angles=[0.3])[0]
    n_p = np.cross(plane[4:7], plane[7:10])
    rng = np.random.default_rng(7)
    cases = []
    # plane: voxel facing the element centre, off-axis inside the aperture, outside the aperture
    cases.append(("plane-centre", plane, plane[1:4] + 9e-3 * n_p))
    cases.append(("plane-inside", plane, plane[1:4] + 8e-3 * n_p + 0.2e-3 * plane[4:7] - 0.3e-3 * plane[7:10]))
    cases.append(("plane-outside", plane, plane[1:4] + 7e-3 * n_p + 2.0e-3 * plane[4:7] + 1.1e-3 * plane[7:10]))
    # cylinder: near focus, off-focus in front, sideways, behind the axis, within the element's z range
    e1, e2 = cyl[4:7], cyl[7:10]
    n_c = np.cross(e1, e2)
    c0 = cyl[1:4]
    cases.append(("cyl-focus", cyl, c0 + 0.05e-3 * e2 + 0.02e-3 * n_c + 0.4e-3 * e1))
    cases.append(("cyl-front", cyl, c0 + 6e-3 * e2 + 1e-3 * n_c + 1.0e-3 * e1))
    cases.append(("cyl-side", cyl, c0 + 0.5e-3 * e2 + 7e-3 * n_c - 2.0e-3 * e1))
    cases.append(("cyl-behind", cyl, c0 - 5e-3 * e2 + 0.3e-3 * n_c + 0.1e-3 * e1))
    cases.append(("cyl-inz", cyl, c0 + 3e-3 * e2 - 2e-3 * n_c + 0.05e-3 * e1))
    cases.append(("cyl-rand", cyl, c0 + rng.uniform(-8e-3, 8e-3, 3) * np.array([1, 1, 0.5])))
    return cases


CASES = _cases()


@pytest.mark.parametrize("name,row,xi", CASES, ids=[c[0] for c in CASES])
def test_area_against_fubini(oracle_mod, name, row, xi):
    w = W.c1(dl=1)
    b0, area = oracle_mod.pair_bin_areas(row, xi, w)
    assert area.size > 0
    ufs = w.U * w.fs
    cum = np.cumsum(area)
    total = element_area(row)
    # cumulative area up to the upper edge of every k-th bin
    step = max(1, area.size // 40)
    for j in list(range(0, area.size, step)) + [area.size - 1]:
        r = w.c * (w.t0 + (b0 + j + 1) / ufs)
        ref = fubini_cumulative_area(row, xi, r)
        # The literal primitive of Eq. (plane_primitive) takes sqrt(rho^2 - u^2) of a
        # rounding-size difference when a bound lies on the circle, which costs
        # FP64 about half its digits (~1e-8 of the area); a wrong branch, fold,
        # sign or term costs orders of magnitude more.
        assert abs(cum[j] - ref) <= 1e-6 * total, (name, j, cum[j], ref)


@pytest.mark.parametrize("name,row,xi", CASES, ids=[c[0] for c in CASES])
def test_total_is_element_area(oracle_mod, name, row, xi):
    for dl in (1, 11):
        w = W.c1(dl=dl)
        _, area = oracle_mod.pair_bin_areas(row, xi, w)
        assert area.sum() == pytest.approx(element_area(row), rel=1e-12)


@pytest.mark.parametrize("name,row,xi", CASES, ids=[c[0] for c in CASES])
def test_groups_are_sums_of_fine_areas(oracle_mod, name, row, xi):
    """Remark 1: the area over Delta-l consecutive bins is the sum of the fine
    areas; groups start at the pair's first bin and the last one is clipped."""
    w1 = W.c1(dl=1)
    wU = W.c1(dl=11)
    b1, a1 = oracle_mod.pair_bin_areas(row, xi, w1)
    bU, aU = oracle_mod.pair_bin_areas(row, xi, wU)
    assert b1 == bU and a1.size == aU.size
    for g in range(0, a1.size, 11):
        sl = slice(g, min(g + 11, a1.size))
        assert aU[sl].sum() == pytest.approx(a1[sl].sum(), rel=1e-11, abs=1e-14 * element_area(row))
        assert np.allclose(aU[sl], aU[sl][0])  # split evenly


@pytest.mark.parametrize("name,row,xi", CASES, ids=[c[0] for c in CASES])
def test_range_against_brute_force(oracle_mod, name, row, xi):
    a, b, wgt, base, axis, half = _element_slices(row)
    t = np.linspace(a, b, 801)
    z = np.linspace(-half, half, 41)
    P = np.array([base(tt) for tt in t])
    d = np.linalg.norm(P[:, None, :] + z[None, :, None] * axis[None, None, :] - xi[None, None, :], axis=2)
    rmin, rmax, nq = oracle_mod.pair_range(row, xi)
    assert nq >= 1
    span = d.max() - d.min()
    assert rmin <= d.min() + 1e-15 and rmin >= d.min() - 1e-3 * span
    assert rmax >= d.max() - 1e-15 and rmax <= d.max() + 1e-3 * span


def test_on_axis_piston_plateau(oracle_mod):
    """Voxel on the axis of a planar element: every bin whose annulus lies in the
    rectangle has f_i[l] = U Fs |M| / (c tau_mid) = 2 pi c exactly."""
    w = W.c1(dl=1)
    row = W.plane_row(np.zeros(3), np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), 0.6e-3, 0.5e-3)
    a3 = 9.3e-3
    xi = np.array([0.0, 0.0, a3])
    b0, area = oracle_mod.pair_bin_areas(row, xi, w)
    ufs = w.U * w.fs
    checked = 0
    for j, A in enumerate(area):
        b = b0 + j
        r_lo = w.c * (w.t0 + b / ufs)
        r_hi = w.c * (w.t0 + (b + 1) / ufs)
        if r_lo >= a3 and math.sqrt(r_hi ** 2 - a3 ** 2) <= 0.5e-3:
            f = ufs * A / (w.c * (w.t0 + (b + 0.5) / ufs))
            # FP64 square-root conditioning of the literal primitive, as above
            assert f == pytest.approx(2 * math.pi * w.c, rel=1e-7)
            checked += 1
    assert checked >= 3


def test_focal_line_cylinder(oracle_mod):
    """rho = 0: |M^l| = 2 R theta_max |{v in [v1, v2] : R^2 + v^2 in [r_l^2, r_{l+1}^2)}|."""
    w = W.c1(dl=1).with_(t0=13.0e-6)
    R, thm, Lz = 20e-3, math.asin(0.25), 0.15e-3
    row = W.cylinder_row(np.zeros(3), np.array([0, 0, 1.0]), np.array([1.0, 0, 0]), R, thm, Lz)
    for a3 in (0.0, 0.1e-3, 0.6e-3):
        xi = np.array([0.0, 0.0, a3])
        b0, area = oracle_mod.pair_bin_areas(row, xi, w)
        ufs = w.U * w.fs
        for j, A in enumerate(area):
            b = b0 + j
            r_lo = w.c * (w.t0 + b / ufs)
            r_hi = w.c * (w.t0 + (b + 1) / ufs)
            # |v| range with R^2 + v^2 in [r_lo^2, r_hi^2)
            vlo = math.sqrt(max(0.0, r_lo ** 2 - R ** 2))
            vhi = math.sqrt(max(0.0, r_hi ** 2 - R ** 2))
            v1, v2 = -Lz - a3, Lz - a3
            meas = max(0.0, min(v2, vhi) - max(v1, vlo)) + max(0.0, min(v2, -vlo) - max(v1, -vhi))
            assert A == pytest.approx(2 * R * thm * meas, rel=1e-9, abs=1e-20)


def test_cylinder_tends_to_the_tangent_plane(oracle_mod):
    """R -> infinity at fixed arc half-width w and half-height Lz: the
    cylinder's group areas tend to those of its tangent plane (half sizes w
    and Lz) at first order in 1/R (the arc's sagitta w^2 / 2R)."""
    w_arc, Lz, d = 0.5e-3, 0.5e-3, 4.0e-3
    wl = W.small_cylinder(n_vox=4, L=2048).with_(t0=0.0)
    e1, e2 = np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])
    errs = []
    for R in (0.05, 0.5, 5.0):
        c0 = -R * e2  # the surface passes through the origin
        cyl = W.cylinder_row(c0, e1, e2, R, w_arc / R, Lz)
        pla = W.plane_row(np.zeros(3), np.cross(e1, e2), e1, w_arc, Lz)
        xi = np.array([-d, 0.13e-3, -0.21e-3])  # on the concave side, off the element's centre
        b0, a_c = oracle_mod.pair_bin_areas(cyl, xi, wl)
        b1, a_p = oracle_mod.pair_bin_areas(pla, xi, wl)
        lo, hi = min(b0, b1), max(b0 + len(a_c), b1 + len(a_p))
        ac = np.zeros(hi - lo)
        ap = np.zeros(hi - lo)
        ac[b0 - lo:b0 - lo + len(a_c)] = a_c
        ap[b1 - lo:b1 - lo + len(a_p)] = a_p
        # compare cumulative areas (robust to a one-bin shift of the range)
        errs.append(np.abs(np.cumsum(ac) - np.cumsum(ap)).max() / (4 * w_arc * Lz))
    print("cumulative-area error vs tangent plane", errs)
    assert errs[0] / errs[1] > 5 and errs[1] / errs[2] > 5, errs
    assert errs[2] < 1e-3, errs
