"""Pins of the oracle's Piecewise-Planes decomposition (Sec. 4.3: the
cylindrical aperture cut into N_p equal angular sectors, each replaced by its
tangent plane), fixed by geometry:

  * every plane touches the cylinder: its centre lies at distance R from the
    focal line, its in-plane directions are orthonormal and perpendicular to
    the radius there, and it spans the sector's chord direction;
  * the planes' total area is the cylinder's, R 2 theta_max 2 Lz (the sector
    width R dtheta is the arc length);
  * the swept areas of the planes converge to the cylinder's as N_p grows
    (the surfaces converge): the error of a pair's summed planar per-bin
    areas (dl = 1) against the exact cylinder areas falls at least 2x per
    doubling of N_p and 10x from N_p = 8 to 64 (between first and second
    order: the planes' edges cross bins where the cylinder's arc does not);
  * the piecewise-planes operator and its transpose pass the dot-product test.
"""
import numpy as np

from paper_2609_29253_gb300 import workloads as W


def _cyl():
    a = W.C2_ARRAY
    return W.cylinder_row(np.array([0.0, 0.0, 1e-3]), np.array([0.0, 0.0, 1.0]),
                          np.array([np.cos(0.3), np.sin(0.3), 0.0]), a["R"], a["theta_max"], a["Lz"])


def test_planes_touch_the_cylinder(oracle_mod):
    row = _cyl()
    P = oracle_mod.piecewise_planes(row, 30)
    c0, e1 = row[1:4], row[4:7]
    for p in P:
        c, u, v = p[1:4], p[4:7], p[7:10]
        d = c - c0 - np.dot(c - c0, e1) * e1
        assert abs(np.linalg.norm(d) - row[12]) <= 1e-15
        assert abs(np.dot(u, u) - 1) < 1e-14 and abs(np.dot(v, v) - 1) < 1e-14 and abs(np.dot(u, v)) < 1e-14
        assert abs(np.dot(u, d)) < 1e-15 and abs(np.dot(v, d)) < 1e-15
    area = sum(4 * p[10] * p[11] for p in P)
    assert abs(area - row[12] * 2 * row[13] * 2 * row[14]) <= 1e-14 * area


def test_planes_converge_to_the_cylinder(oracle_mod):
    row = _cyl()
    # dl = 1: per-bin areas (with dl > 1 each plane's groups would start at
    # its own l_min, a different partition from the cylinder's)
    w = W.small_cylinder(n_vox=4, dl=1, L=2048)
    xi = np.array([1.7e-3, -0.9e-3, 1.2e-3])
    b0, ex = oracle_mod.pair_bin_areas(row, xi, w)
    errs = []
    for npl in (8, 16, 32, 64):
        tot = np.zeros(len(ex) + 400)
        for p in oracle_mod.piecewise_planes(row, npl):
            b, a = oracle_mod.pair_bin_areas(p, xi, w)
            off = b - b0 + 200
            tot[off:off + len(a)] += a
        errs.append(np.linalg.norm(tot[200:200 + len(ex)] - ex) / np.linalg.norm(ex))
    assert all(errs[i] / errs[i + 1] >= 2.0 for i in range(3)), errs
    assert errs[3] <= errs[0] / 10, errs


def test_piecewise_planes_dot_product(oracle_mod):
    w = W.small_cylinder(n_vox=5, n_angles=2, n_el=2)
    taps = oracle_mod.taps_for(w)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(w.N)
    y = rng.standard_normal((w.K, w.L))
    s, _ = oracle_mod.piecewise_planes_forward(w, taps, x, 6)
    z, _ = oracle_mod.piecewise_planes_adjoint(w, taps, y, 6)
    lhs, rhs = float((s * y).sum()), float((x * z).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
