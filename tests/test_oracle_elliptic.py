"""Pins of the oracle's elliptic integrals (Sec. 4.2.1, App. F).

The oracle's Carlson R_F / R_D, E and F are checked against mpmath (an
independent arbitrary-precision library), against special values
(E(t, 0) = t, E(t, 1) = sin t), and the arc-integral identity of Lemma 6 is
checked against direct numerical integration of sqrt(2 R rho cos u + b).
"""
import math

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")
mp.mp.dps = 30  # the default 15 digits is not enough near the singularity of F


def test_carlson_against_mpmath(oracle_mod):
    rng = np.random.default_rng(0)
    for _ in range(300):
        x, y, z = rng.random(3) * 4.0
        assert oracle_mod.carlson_rf(x, y, z) == pytest.approx(float(mp.elliprf(x, y, z)), rel=1e-13)
        assert oracle_mod.carlson_rd(x, y, z) == pytest.approx(float(mp.elliprd(x, y, z)), rel=1e-13)
    # degenerate first arguments
    assert oracle_mod.carlson_rf(0.0, 0.5, 1.0) == pytest.approx(float(mp.elliprf(0, 0.5, 1)), rel=1e-13)
    assert oracle_mod.carlson_rd(0.0, 0.5, 1.0) == pytest.approx(float(mp.elliprd(0, 0.5, 1)), rel=1e-13)


def test_incomplete_e_f_against_mpmath(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(300):
        phi = rng.random() * math.pi / 2
        m = rng.random()
        assert oracle_mod.ellip_e(phi, m) == pytest.approx(float(mp.ellipe(phi, m)), abs=1e-14)
        assert oracle_mod.ellip_f(phi, m) == pytest.approx(float(mp.ellipf(phi, m)), abs=1e-14)
    # near the logarithmic singularity of F at (pi/2, 1)
    for m in (1 - 1e-6, 1 - 1e-10):
        phi = math.pi / 2 - 1e-7
        assert oracle_mod.ellip_f(phi, m) == pytest.approx(float(mp.ellipf(phi, m)), rel=1e-12)


def test_special_values(oracle_mod):
    for t in np.linspace(0, math.pi / 2, 17):
        assert oracle_mod.ellip_e(t, 0.0) == pytest.approx(t, abs=1e-15)
        assert oracle_mod.ellip_e(t, 1.0) == pytest.approx(math.sin(t), abs=1e-15)
        assert oracle_mod.ellip_e_any(t, 0.0) == pytest.approx(t, abs=1e-15)


def test_reciprocal_modulus_against_mpmath(oracle_mod):
    """E(t, nu) with nu > 1 and nu sin^2 t <= 1 (Eq. reciprocal_modulus)."""
    rng = np.random.default_rng(2)
    for _ in range(300):
        nu = 1.0 + rng.random() * 50.0
        tmax = math.asin(math.sqrt(1.0 / nu))
        t = tmax * rng.random()
        ref = mp.ellipe(t, nu)
        assert abs(mp.im(ref)) < 1e-20
        assert oracle_mod.ellip_e_any(t, nu) == pytest.approx(float(mp.re(ref)), abs=1e-14)
    # at the end point nu sin^2 t = 1
    for nu in (1.5, 4.0, 100.0):
        t = math.asin(math.sqrt(1.0 / nu))
        assert oracle_mod.ellip_e_any(t, nu) == pytest.approx(float(mp.re(mp.ellipe(t, nu))), abs=1e-12)


def test_lemma6_arc_integral_against_quadrature(oracle_mod):
    """int_a^b sqrt(2 R rho cos u + b) du = 2 sqrt(2 R rho + b) [E(b/2, nu) - E(a/2, nu)]."""
    from scipy.integrate import quad

    rng = np.random.default_rng(3)
    R = 20e-3
    for _ in range(40):
        rho = rng.uniform(0.5e-3, 15e-3)
        r = rng.uniform(R - rho + 1e-4, R + rho + 5e-3)
        bb = r * r - rho * rho - R * R
        # largest u with a real integrand on [0, pi]
        cu = -bb / (2 * R * rho)
        umax = math.pi if cu <= -1 else math.acos(min(1.0, cu))
        a, b = sorted(rng.random(2) * umax)
        num = quad(lambda u: math.sqrt(max(0.0, 2 * R * rho * math.cos(u) + bb)), a, b, epsabs=0, epsrel=1e-13,
                   limit=200)[0]
        q = 2 * R * rho + bb
        nu = 4 * R * rho / q
        cf = 2 * math.sqrt(q) * (oracle_mod.ellip_e_any(b / 2, nu) - oracle_mod.ellip_e_any(a / 2, nu))
        assert cf == pytest.approx(num, rel=1e-9, abs=1e-15)
