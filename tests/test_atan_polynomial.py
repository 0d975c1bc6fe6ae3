"""Pin of the planar geometry kernels' own first-quadrant arctangent (no GPU needed).

The plane's primitive (Sec. 4.1, Eq. plane_primitive) takes arcsin(u / rho) at
the two clamped bounds; the kernels form the difference of the two arcsines
as one angle, atan_q1(cross, dot) with cross, dot >= 0.  atan_q1 computes
t = min / max (reciprocal, then one Newton step on the quotient), z = t^2,
arctan(t) = t + t z q(z) with a degree-8 polynomial q read here from the CUDA
source (`kAt1` .. `kAt9`), and pi/2 - arctan(t) when y > x.  This test
evaluates that sequence in FP32 (every fused multiply-add formed exactly in
FP64 and rounded once; the reciprocal, approximate on the device, taken
correctly rounded and off by one and two ulps either way, which the Newton
step on the quotient absorbs) and checks the bound the source
states, 1.5e-7 relative to the angle (about 1.3 ulp; CUDA documents 2 ulp for
atan2f), against math.atan2 on a dense set of
first-quadrant directions, plus the fit's own 2e-8 in FP64 and the exact
ends (0 at y = 0, pi/2 at x = 0).
"""
import math
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2609_29253_gb300", "csrc",
                   "pat_geom.cuh")


def _coeffs():
    found = dict((int(k), float(v)) for k, v in re.findall(r"kAt(\d) = (-?\d+\.\d*(?:e-?\d+)?)f", open(SRC).read()))
    assert sorted(found) == list(range(1, 10)), found
    return [float(np.float32(found[k])) for k in range(1, 10)]


F = np.float32


def _fma(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def _atan_q1(y, x, c, rcp_ulps=0):
    y, x = F(y), F(x)
    mx, mn = F(max(max(x, y), F(1e-30))), F(min(x, y))
    rc = F(1.0 / np.float64(mx))
    for _ in range(abs(rcp_ulps)):  # the hardware reciprocal is approximate: try it off by an ulp or two
        rc = np.nextafter(rc, F(np.inf) if rcp_ulps > 0 else F(0))
    t = F(np.float64(mn) * np.float64(rc))
    t = _fma(rc, _fma(-t, mx, mn), t)
    z = F(np.float64(t) * np.float64(t))
    q = F(c[8])
    for k in range(7, -1, -1):
        q = _fma(q, z, c[k])
    a = _fma(F(np.float64(t) * np.float64(z)), q, t)
    return F(np.float64(F(1.57079637)) - np.float64(a)) if y > x else a


def test_first_quadrant_arctangent_within_stated_bound():
    c = _coeffs()
    rng = np.random.default_rng(0)
    ang = np.concatenate([np.linspace(0.0, math.pi / 2, 20001), rng.uniform(0, math.pi / 2, 20000),
                          np.geomspace(1e-9, 1e-2, 500), math.pi / 2 - np.geomspace(1e-9, 1e-2, 500)])
    worst = 0.0
    for i, th in enumerate(ang):
        r = 10.0 ** ((i % 7) - 3)  # scale-free
        y, x = F(r * math.sin(th)), F(r * math.cos(th))
        if y == 0 and x == 0:
            continue
        exact = math.atan2(float(y), float(x))
        for ulps in ((0, -2, -1, 1, 2) if i % 5 == 0 else (0,)):
            got = float(_atan_q1(y, x, c, ulps))
            if exact == 0.0:
                assert got == 0.0
                continue
            worst = max(worst, abs(got - exact) / exact)
    assert worst <= 1.5e-7, worst
    assert float(_atan_q1(0.0, 1.0, c)) == 0.0
    assert float(_atan_q1(1.0, 0.0, c)) == float(F(1.57079637))


def test_arctangent_fit_in_fp64():
    c = np.array(_coeffs())
    z = np.linspace(1e-12, 1.0, 100001)
    t = np.sqrt(z)
    approx = t * (1.0 + z * np.polyval(c[::-1], z))
    assert np.max(np.abs(approx / np.arctan(t) - 1.0)) <= 2e-8
