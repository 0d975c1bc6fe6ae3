"""Pins of the oracle's lookup-table variant of the cylinder's arc integral
(Sec. 4.2.2: E~(s, m) = E(arcsin s, m) and F~(s, m) = F(arcsin s, m) on the
power-law grid of Eq. LUT_sampling, bilinear interpolation, the
reciprocal-modulus transformation of Eq. reciprocal_modulus for nu > 1),
each fixed by something other than the oracle's own formulas:

  * at the nodes of the paper's grid, written out here from Eq. LUT_sampling
    (1-based n), the tables return scipy's incomplete integrals to rounding,
    so the oracle's grid is the paper's;
  * between the nodes the error against scipy is that of bilinear
    interpolation: second order in the grid step (halving the step divides
    it by about 4);
  * for nu > 1 the table value matches direct quadrature of
    sqrt(1 - nu sin^2 t) over [0, theta] (the integral of Eq. cyl_Il itself,
    no elliptic-integral routine involved);
  * the telescoped group areas of a pair sum to the element area R 2
    theta_max 2 Lz, whatever the tables hold;
  * on the focal line (rho = 0) E is never evaluated: LUT and exact areas
    agree to rounding;
  * the LUT areas converge to the exact ones at second order as the tables
    grow, and the LUT operator passes its own dot-product test.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import ellipeinc, ellipkinc

from paper_2609_29253_gb300 import workloads as W


def _paper_node(n, N, eps=1e-16):
    """Eq. LUT_sampling, n = 1 .. N."""
    return (1 - eps) * (1 - (1 - (n - 1) / (N - 1)) ** 4)


def test_grid_is_the_papers(oracle_mod):
    for N in (7, 100, 1000):
        for n in (1, 2, N // 3, N - 1, N):
            assert oracle_mod.lut_node(n - 1, N) == pytest.approx(_paper_node(n, N), rel=1e-15, abs=1e-300)


def test_tables_exact_at_the_nodes(oracle_mod):
    N = 100
    rng = np.random.default_rng(0)
    for _ in range(40):
        n, k = rng.integers(1, N + 1, 2)
        s, m = _paper_node(n, N), _paper_node(k, N)
        if s > 0.999 and m > 0.999:
            continue  # the log-singular corner: scipy itself loses digits there
        ref = ellipeinc(math.asin(s), m)
        # nu <= 1 branch: E~(sin theta, nu) with theta = arcsin s
        assert oracle_mod.ellip_e_lut(math.asin(s), m, N, N) == pytest.approx(ref, rel=1e-12, abs=1e-15)


def test_interpolation_error_is_second_order(oracle_mod):
    rng = np.random.default_rng(1)
    pts = [(rng.uniform(0.0, 0.97), rng.uniform(0.0, 0.97)) for _ in range(300)]
    errs = []
    for N in (100, 200, 400):
        e = 0.0
        for s, m in pts:
            th = math.asin(s)
            e = max(e, abs(oracle_mod.ellip_e_lut(th, m, N, N) - ellipeinc(th, m)))
        errs.append(e)
    assert errs[0] > 1e-9
    assert errs[0] / errs[1] >= 3.0 and errs[1] / errs[2] >= 3.0, errs
    # at the paper's size the tables are good to about 1e-6 in this range
    e1000 = max(abs(oracle_mod.ellip_e_lut(math.asin(s), m, 1000, 1000) - ellipeinc(math.asin(s), m)) for s, m in pts)
    assert e1000 < 1e-6, e1000


@pytest.mark.parametrize("nu", [1.3, 2.0, 7.5, 60.0])
def test_reciprocal_modulus_branch_against_quadrature(oracle_mod, nu):
    th_max = math.asin(1.0 / math.sqrt(nu))  # nu sin^2(theta) <= 1 (Lemma 6)
    for f in (0.1, 0.5, 0.9, 0.999):
        th = f * th_max
        ref, _ = quad(lambda t: math.sqrt(max(0.0, 1.0 - nu * math.sin(t) ** 2)), 0.0, th, epsabs=1e-14,
                      epsrel=1e-13, limit=200)
        got = oracle_mod.ellip_e_lut(th, nu, 1000, 1000)
        # the interpolation error of E~ and F~ (about 1e-7) scaled by sqrt(nu)
        assert abs(got - ref) <= 2e-6 * math.sqrt(nu), (th, got, ref)
    # and F~ agrees with scipy's F through the same transformation
    m = 1.0 / nu
    s = 0.6
    e = math.sqrt(nu) * (ellipeinc(math.asin(s), m) - (1 - m) * ellipkinc(math.asin(s), m))
    assert abs(oracle_mod.ellip_e_lut(math.asin(s / math.sqrt(nu)), nu, 1000, 1000) - e) <= 2e-6 * math.sqrt(nu)


def _cyl(Lz=0.15e-3, R=20e-3):
    a = W.C2_ARRAY
    return W.cylinder_row(np.array([0.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0]), R,
                          a["theta_max"], Lz)


@pytest.mark.parametrize("dl", [1, 11])
def test_lut_total_is_the_element_area(oracle_mod, dl):
    w = W.small_cylinder(n_vox=4, dl=dl, L=2048)
    Lz = 0.15e-3
    row = _cyl(Lz)
    total = 20e-3 * 2 * W.C2_ARRAY["theta_max"] * 2 * Lz
    rng = np.random.default_rng(3)
    for _ in range(6):
        xi = np.array([rng.uniform(-3e-3, 3e-3), rng.uniform(-3e-3, 3e-3), rng.uniform(-1e-3, 1e-3)])
        _, lu = oracle_mod.pair_bin_areas(row, xi, w, method=oracle_mod.METHOD_LUT, lut=(200, 200))
        assert abs(lu.sum() - total) <= 1e-10 * total


def test_lut_exact_on_focal_line(oracle_mod):
    w = W.small_cylinder(n_vox=4, L=2048)
    row = _cyl()
    for z in (0.0, 0.05e-3, 0.4e-3, 2e-3):
        xi = np.array([0.0, 0.0, z])
        b0, ex = oracle_mod.pair_bin_areas(row, xi, w)
        b1, lu = oracle_mod.pair_bin_areas(row, xi, w, method=oracle_mod.METHOD_LUT, lut=(50, 50))
        assert b0 == b1 and np.abs(lu - ex).max() <= 1e-12 * np.abs(ex).max()


def test_lut_areas_converge_to_exact(oracle_mod):
    w = W.small_cylinder(n_vox=4, dl=11, L=2048)
    tx = W.c2(n_angles=3, with_x=False).tx
    rng = np.random.default_rng(0)
    pairs = [(tx[rng.integers(len(tx))], rng.uniform(-6e-3, 6e-3, 3)) for _ in range(16)]
    exact = [oracle_mod.pair_bin_areas(row, xi, w) for row, xi in pairs]
    errs = []
    for N in (250, 500, 1000):
        num = den = 0.0
        for (row, xi), (b0, ex) in zip(pairs, exact):
            b1, lu = oracle_mod.pair_bin_areas(row, xi, w, method=oracle_mod.METHOD_LUT, lut=(N, N))
            assert b0 == b1
            num += float(np.sum((lu - ex) ** 2))
            den += float(np.sum(ex ** 2))
        errs.append(math.sqrt(num / den))
    assert errs[0] / errs[1] >= 3.0 and errs[1] / errs[2] >= 2.5, errs
    assert errs[2] < 3e-3, errs


def test_lut_operator_dot_product(oracle_mod):
    w = W.small_cylinder(n_vox=6, n_angles=2, n_el=2).with_(method=oracle_mod.METHOD_LUT, q1=300, q2=300)
    taps = oracle_mod.taps_for(w)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(w.N)
    y = rng.standard_normal((w.K, w.L))
    s, _ = oracle_mod.forward(w, taps, x)
    z, _ = oracle_mod.adjoint(w, taps, y)
    lhs, rhs = float((s * y).sum()), float((x * z).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    s_ex, _ = oracle_mod.forward(w.with_(method=0, q1=0, q2=0), taps, x)
    d = np.linalg.norm(s - s_ex) / np.linalg.norm(s_ex)
    assert 0 < d < 2e-2, d
