"""Pins of the oracle's trapezoidal arc integral (Eq. trapezoid_Il: the level
curve between (alpha, Psi(alpha)) and (beta, Psi(beta)) replaced by its
chord), each fixed by the geometry rather than by the formula:

  * on the focal line (rho = 0) every level curve is flat, so the chord is
    the curve: trapezoidal and exact areas agree to rounding;
  * when the sphere has passed the whole element every bound is clamped, so
    the telescoped sum of a pair's areas is the element's area R 2 theta_max
    2 Lz exactly, whatever the rule did in between;
  * the chord error shrinks with the strip: for a voxel near the focal zone,
    halving Lz (the element's width along the axis) cuts the error of the
    pair's group areas against the exact ones (rel L2, dl = U) by at least
    3x (second order in the chord length; far from the focus the chords
    span strongly curved arcs and the rate is lower);
  * the trapezoidal operator is a linear operator like the exact one, and
    its oracle transpose passes the dot-product test.
"""
import numpy as np
import pytest

from paper_2609_29253_gb300 import workloads as W


def _cyl(Lz=0.15e-3, R=20e-3):
    a = W.C2_ARRAY
    return W.cylinder_row(np.array([0.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0]), R,
                          a["theta_max"], Lz)


def _w(dl=1):
    return W.small_cylinder(n_vox=4, dl=dl, L=2048)


def test_trapezoid_exact_on_focal_line(oracle_mod):
    w = _w()
    row = _cyl()
    for z in (0.0, 0.05e-3, 0.4e-3, 2e-3):
        xi = np.array([0.0, 0.0, z])
        b0, ex = oracle_mod.pair_bin_areas(row, xi, w)
        b1, tr = oracle_mod.pair_bin_areas(row, xi, w, method=oracle_mod.METHOD_TRAPEZOID)
        assert b0 == b1 and len(ex) == len(tr)
        assert np.abs(tr - ex).max() <= 1e-12 * np.abs(ex).max()


@pytest.mark.parametrize("dl", [1, 11])
def test_trapezoid_total_is_the_element_area(oracle_mod, dl):
    w = _w(dl)
    Lz = 0.15e-3
    row = _cyl(Lz)
    total = 20e-3 * 2 * W.C2_ARRAY["theta_max"] * 2 * Lz
    rng = np.random.default_rng(3)
    for _ in range(6):
        xi = np.array([rng.uniform(-3e-3, 3e-3), rng.uniform(-3e-3, 3e-3), rng.uniform(-1e-3, 1e-3)])
        b, tr = oracle_mod.pair_bin_areas(row, xi, w, method=oracle_mod.METHOD_TRAPEZOID)
        assert abs(tr.sum() - total) <= 1e-10 * total


def test_trapezoid_error_is_second_order_in_the_strip_width(oracle_mod):
    w = _w(11)
    xi = np.array([2.3e-3, -1.1e-3, 0.37e-3])
    errs = []
    for Lz in (0.4e-3, 0.2e-3, 0.1e-3, 0.05e-3):
        row = _cyl(Lz)
        b0, ex = oracle_mod.pair_bin_areas(row, xi, w)
        b1, tr = oracle_mod.pair_bin_areas(row, xi, w, method=oracle_mod.METHOD_TRAPEZOID)
        assert b0 == b1
        errs.append(np.linalg.norm(tr - ex) / np.linalg.norm(ex))
    assert errs[0] > 0
    assert all(errs[i] / errs[i + 1] >= 3.0 for i in range(3)), errs


def test_trapezoid_operator_dot_product(oracle_mod):
    w = W.small_cylinder(n_vox=6, n_angles=2, n_el=2).with_(method=2)
    taps = oracle_mod.taps_for(w)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(w.N)
    y = rng.standard_normal((w.K, w.L))
    s, _ = oracle_mod.forward(w, taps, x)
    z, _ = oracle_mod.adjoint(w, taps, y)
    lhs, rhs = float((s * y).sum()), float((x * z).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # and it differs from the exact operator, but not by much on this thin strip
    s_ex, _ = oracle_mod.forward(w.with_(method=0), taps, x)
    d = np.linalg.norm(s - s_ex) / np.linalg.norm(s_ex)
    assert 0 < d < 1e-2, d
