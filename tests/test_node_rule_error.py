"""Truncation error of the Gauss-Legendre rules of the exact cylinder path.

The kernels integrate the accumulated angle along the element's axial
coordinate over an unclamped piece (Fubini along v, Sec. 4.2.1, the integral
form of Eq. cyl_Il): in the shifted variable t = v - vc, with
4 R rho S(t) = q' - t (2 vc + t) and X = 1 - S, the angle is
u(t) = 2 arcsin(sqrt(S)), accumulated as u on quadrants on the u = 0 side of
pi/2 and as pi - u = 2 arcsin(sqrt(X)) on those on the u = pi side.  u has
square-root branch points where S = 0 (v_s = sqrt(q' + vc^2)) and where
X = 0 (v_f = sqrt(vc^2 - qf') when qf' = 4 R rho - q' < vc^2, else the pair
v = +-i sqrt(qf' - vc^2)).  With the piece [v_a, v_b] = vc + [a, a + L] the
distances are d_s = v_s - v_b and d_f = v_a - v_f, or the distance from v_a
to the complex pair.  The operator's kernels take 2 nodes when both are at
least 8 L, 4 nodes from 1 L to 8 L (closer: a substitution); the design
bounds the relative error of the piece integral by 1.1e-7 for that 2-node
rule (the worst case sits on the u = pi side of a reflected quadrant; about
1.6 times the FP32 error of a node's angle from the arcsine polynomial alone,
6.4e-8) and by 1.5e-8 for the 4-node rule.  The speed-of-sound derivative's
kernels (cyl_F) keep 2, 3 or 4 nodes above 13 L, 3 L and 1 L, bounded by
1.6e-8.  These tests check those claims over c2-like geometries (R 20 mm,
rho 0.5-8 mm, vc 0.5-10 mm, L 0.1-0.3 mm, q' swept across the range where
the piece is unclamped) against an adaptive quadrature of the same
integrand, analytic on the piece (good to ~1e-14).
No kernel code is involved: the nodes come from numpy's Legendre routine.
"""
import math

import numpy as np
import pytest

integrate = pytest.importorskip("scipy.integrate")

R = 20e-3
RHO = (0.5e-3, 1e-3, 3e-3, 8e-3)
VC = (0.5e-3, 2e-3, 10e-3)
LEN = (0.1e-3, 0.15e-3, 0.3e-3)


def _rule(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1.0) / 2.0, w / 2.0


def _samples():
    """(4 R rho, q', vc, L, d / L, low side) for pieces [0, L] in t that stay
    inside one side of pi/2 (0 < S < 1/2 or 1/2 < S < 1 at both ends), with q'
    on a geometric sweep toward each branch point; d is the smaller of d_s and
    d_f, low side whether the accumulated angle is u (else pi - u)."""
    out = []
    for rho in RHO:
        four = 4.0 * R * rho
        for vc in VC:
            for L in LEN:
                c_end = L * (2.0 * vc + L)  # t (2 vc + t) at t = L; 0 at t = 0
                # S(0) = q'/four, S(L) = (q' - c_end)/four: sweep q' over (c_end, four)
                for frac in np.concatenate([np.geomspace(1e-4, 0.5, 40), 1.0 - np.geomspace(1e-4, 0.5, 40)]):
                    qp = c_end + frac * (four - c_end)
                    S0, S1 = qp / four, (qp - c_end) / four
                    if not (0.0 < S1 < S0 < 1.0) or (S1 < 0.5 < S0):
                        continue
                    vs = math.sqrt(qp + vc * vc)
                    ds = vs - (vc + L)
                    qf = four - qp
                    if qf < vc * vc:
                        df = vc - math.sqrt(vc * vc - qf)
                    else:
                        df = math.sqrt(qf)  # |v_a - i sqrt(qf - vc^2)| with v_a = vc: sqrt(vc^2 + qf - vc^2)
                    out.append((four, qp, vc, L, min(ds, df) / L, S0 <= 0.5))
    return out


SAMPLES = _samples()


def _rel_error(n, four, qp, vc, L, low_side):
    x, w = _rule(n)

    def acc(t):
        S = (qp - t * (2.0 * vc + t)) / four
        u = 2.0 * np.arcsin(np.sqrt(np.clip(S, 0.0, 1.0)))
        return u if low_side else math.pi - u

    ref, _ = integrate.quad(lambda t: float(acc(t)), 0.0, L, epsabs=0.0, epsrel=1e-13, limit=200)
    got = L * float(np.sum(w * acc(x * L)))
    return abs(got - ref) / abs(ref)


def _worst(n, dmin, dmax):
    errs = [_rel_error(n, four, qp, vc, L, low) for four, qp, vc, L, d, low in SAMPLES if dmin <= d < dmax]
    return (max(errs) if errs else None), len(errs)


def test_two_node_rule_from_8L():
    worst, count = _worst(2, 8.0, math.inf)
    assert count > 200, count
    assert worst <= 1.1e-7, worst


def test_four_node_rule_from_1L_to_8L():
    worst, count = _worst(4, 1.0, 8.0)
    assert count > 50, count
    assert worst <= 1.5e-8, worst


def test_derivative_kernel_rules():
    for n, lo, hi in ((4, 1.0, 3.0), (3, 3.0, 13.0), (2, 13.0, math.inf)):
        worst, count = _worst(n, lo, hi)
        assert count > 50, (n, count)
        assert worst <= 1.6e-8, (n, worst)


def test_two_nodes_would_not_hold_at_5L():
    """The threshold is not loose: between 5 L and 6 L the 2-node rule exceeds
    the bound several times (so a wrong node or weight would not hide behind a
    margin)."""
    worst, count = _worst(2, 5.0, 6.0)
    assert count > 0
    assert worst > 3 * 1.1e-7, worst


def _subst(near, a, b, ts, tf, f):
    """6 Gauss-Legendre nodes in tau after t = t_s - c tau^2 (near: the S = 0
    branch point at or beyond b) or t = t_f + c tau^2 (the X = 0 one at or
    before a), tau over [t0, 1] so that the map covers exactly [a, b]."""
    x, w = _rule(6)
    if near:
        c = ts - a
        t0 = math.sqrt((ts - b) / c)
    else:
        c = b - tf
        t0 = math.sqrt((a - tf) / c)
    tau = t0 + (1.0 - t0) * x
    t = ts - c * tau**2 if near else tf + c * tau**2
    return float(np.sum(w * 2.0 * c * tau * (1.0 - t0) * f(t)))


def test_substitution_rule_within_L():
    """Branch points closer than L: the substitution at the near one, or with
    both within L the piece halved at its midpoint, each half taking its own
    end's substitution.  The truncation error of the rule itself (FP64
    emulation) stays below 1e-10 of the piece integral, branch point on the
    piece's end included; the kernels' FP32 rounding comes on top of it."""
    worst, count = 0.0, 0
    for rho in RHO:
        four = 4.0 * R * rho
        for vc in VC:
            for L in LEN:
                a, b = 0.0, L
                for side in ("s", "f"):
                    for k in np.linspace(0.0, 0.99, 12):
                        if side == "s":
                            t = b + k * L
                            qp = t * (2.0 * vc + t)  # S = 0 at t
                        else:
                            t = a - k * L
                            if t + vc < 0.0:
                                continue  # v_f >= 0 on a folded quadrant
                            qp = four + t * (2.0 * vc + t)  # X = 0 at t
                        S0, S1 = qp / four, (qp - L * (2.0 * vc + L)) / four
                        if not (-1e-15 <= S1 < S0 <= 1.0 + 1e-15) or (S1 < 0.5 < S0):
                            continue
                        ts = max(math.sqrt(qp + vc * vc) - vc, b)
                        qf = four - qp
                        hasf = qf < vc * vc
                        tf = min(math.sqrt(max(0.0, vc * vc - qf)) - vc, a) if hasf else -vc
                        near, far = ts - b < L, hasf and a - tf < L
                        if not (near or far):
                            continue
                        low = S0 <= 0.5

                        def f(tt, four=four, qp=qp, vc=vc, low=low):
                            S = (qp - tt * (2.0 * vc + tt)) / four
                            u = 2.0 * np.arcsin(np.sqrt(np.clip(S, 0.0, 1.0)))
                            return u if low else math.pi - u

                        if near and far:
                            m = 0.5 * (a + b)
                            got = _subst(False, a, m, ts, tf, f) + _subst(True, m, b, ts, tf, f)
                        else:
                            got = _subst(near, a, b, ts, tf, f)
                        ref, _ = integrate.quad(lambda tt: float(f(tt)), a, b, epsabs=0.0, epsrel=1e-13, limit=500)
                        worst = max(worst, abs(got - ref) / abs(ref))
                        count += 1
    assert count > 300, count
    assert worst <= 1e-10, worst
