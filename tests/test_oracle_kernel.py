"""Pins of the oracle's system kernel, convolution and downsampling
(Prop. 1, Eq. def_bh, Eq. discrete_conv, App. D, App. G).

* With a box EIR and the bump radial function every quantity is a piecewise
  polynomial, so h-bar[n] and the sampled response S(h * 1_bin) have exact
  rational values; they are computed here from antiderivatives of
  g(t) = -1/2 c t phi(|c t|) with Python fractions, independently of the
  oracle's Gauss-Legendre quadrature and of its discrete convolution loop.
* sum_n h-bar[n] = int h = (int e)(int g) = 0 because g is odd.
* The oracle's convolution + downsampling equals numpy.convolve followed by
  block means; its transpose passes the dot-product test.
* The Gaussian-modulated sine of the benchmark input recipe has the stated
  -6 dB fractional bandwidth.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_2609_29253_gb300 import workloads as W

sp = pytest.importorskip("sympy")

C = 1500
KAPPA = Fr(3, 20000)  # 0.15 mm
TE = Fr(7, 10 ** 7)  # box EIR support 0.7 us
A0 = Fr(1, 1)
U = 11
FS = 40 * 10 ** 6
DELTA = Fr(1, U * FS)


def _poly_antiderivs():
    """Coefficients (ascending, Fractions) of G(y) = int_{-k/c}^y g and of the
    antiderivatives Q1 = int G, Q2 = int Q1, P2 = int y G(y), all on the
    support [-k/c, k/c] of g (they vanish at -k/c)."""
    y, s = sp.symbols("y s")
    k = sp.Rational(KAPPA.numerator, KAPPA.denominator)
    g = -sp.Rational(1, 2) * C * s * (1 - (C * s / k) ** 2) ** 2
    lo = -k / C
    G = sp.integrate(g, (s, lo, y))
    Q1 = sp.integrate(G.subs(y, s), (s, lo, y))
    Q2 = sp.integrate(Q1.subs(y, s), (s, lo, y))
    P2 = sp.integrate((s * G.subs(y, s)), (s, lo, y))

    def coeffs(expr):
        p = sp.Poly(sp.expand(expr), y)
        cs = p.all_coeffs()[::-1]
        return [Fr(int(sp.fraction(cc)[0]), int(sp.fraction(cc)[1])) for cc in cs]

    return coeffs(G), coeffs(Q1), coeffs(Q2), coeffs(P2)


GC, Q1C, Q2C, P2C = _poly_antiderivs()
KC = KAPPA / C


def _ev(cs, y):
    acc = Fr(0)
    for c in reversed(cs):
        acc = acc * y + c
    return acc


def _G(y):
    return _ev(GC, y) if -KC <= y <= KC else Fr(0)


def _P1(y):  # int_{-inf}^y G
    if y <= -KC:
        return Fr(0)
    if y >= KC:
        return _ev(Q1C, KC)
    return _ev(Q1C, y)


def _P2y(y):  # int_{-inf}^y t G(t) dt
    if y <= -KC:
        return Fr(0)
    if y >= KC:
        return _ev(P2C, KC)
    return _ev(P2C, y)


def _Q2(y):  # int_{-inf}^y P1
    if y <= -KC:
        return Fr(0)
    if y >= KC:
        return _ev(Q2C, KC) + _ev(Q1C, KC) * (y - KC)
    return _ev(Q2C, y)


def _tri_G(a):
    """int_{-D}^{D} (D - |s|) G(a + s) ds, exactly."""
    D = DELTA
    # s in [0, D]: y = a + s, weight D + a - y ; s in [-D, 0]: weight D - a + y
    right = (D + a) * (_P1(a + D) - _P1(a)) - (_P2y(a + D) - _P2y(a))
    left = (D - a) * (_P1(a) - _P1(a - D)) + (_P2y(a) - _P2y(a - D))
    return right + left


def exact_hbar(n):
    # h(t) = A0 [G(t) - G(t - Te)]
    return A0 * (_tri_G(n * DELTA) - _tri_G(n * DELTA - TE)) / DELTA


def exact_sampled_bin(l, b0):
    """F_s int_{t_l}^{t_{l+1}} int_{tau_b0}^{tau_b0+1} h(t - t') dt' dt (t0 = 0)."""
    a, b = l * U * DELTA, (l + 1) * U * DELTA
    c, d = b0 * DELTA, (b0 + 1) * DELTA

    def dbl(shift):  # int_a^b int_c^d G(t - t' - shift) dt' dt
        return (_Q2(b - c - shift) - _Q2(a - c - shift) - _Q2(b - d - shift) + _Q2(a - d - shift))

    return FS * A0 * (dbl(Fr(0)) - dbl(TE))


def _box_w():
    kappa, te = float(KAPPA), float(TE)
    n_lo, T = W.tap_window(kappa, C, FS, U, te)
    par = np.array([float(A0), 0.0, 0.0, te])
    return kappa, te, n_lo, T, par


def test_taps_exact_box_eir(oracle_mod):
    kappa, te, n_lo, T, par = _box_w()
    taps = oracle_mod.system_kernel(W.RBF_BUMP, kappa, W.EIR_BOX, par, C, FS, U, n_lo, T)
    ref = np.array([float(exact_hbar(n_lo + t)) for t in range(T)])
    assert np.abs(ref).max() > 0
    assert np.abs(taps - ref).max() <= 1e-12 * np.abs(ref).max()
    # the window of Sec. 2.6 holds the whole support
    assert ref[0] == 0.0 and ref[-1] == 0.0


def test_taps_sum_to_zero(oracle_mod):
    w = W.c1()
    taps = oracle_mod.taps_for(w)
    assert abs(taps.sum()) <= 1e-13 * np.abs(taps).sum()
    kappa, te, n_lo, T, par = _box_w()
    t2 = oracle_mod.system_kernel(W.RBF_CONE, kappa, W.EIR_BOX, par, C, FS, U, n_lo, T)
    assert abs(t2.sum()) <= 1e-13 * np.abs(t2).sum()


def test_taps_quadrature_converged(oracle_mod):
    w = W.c1()
    a = oracle_mod.system_kernel(w.rbf_kind, w.kappa, w.eir_kind, w.eir_par, w.c, w.fs, w.U, w.n_lo, w.T, panels=2)
    b = oracle_mod.system_kernel(w.rbf_kind, w.kappa, w.eir_kind, w.eir_par, w.c, w.fs, w.U, w.n_lo, w.T, panels=6)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_sampling_identity_app_d(oracle_mod):
    """A(one fine bin) = S(h * 1_[tau_b, tau_b+1)) exactly (App. D)."""
    kappa, te, n_lo, T, par = _box_w()
    taps = oracle_mod.system_kernel(W.RBF_BUMP, kappa, W.EIR_BOX, par, C, FS, U, n_lo, T)
    L = 24

    class Wl:
        pass

    w = Wl()
    w.U, w.L, w.n_lo = U, L, n_lo
    for b0 in (60, 61, 70, 71 + 3 * U):
        f = np.zeros((1, U * L))
        f[0, b0] = 1.0
        s = oracle_mod.conv_forward(w, taps, f)[0]
        ref = np.array([float(exact_sampled_bin(l, b0)) for l in range(L)])
        assert np.abs(ref).max() > 0
        assert np.abs(s - ref).max() <= 1e-12 * np.abs(ref).max(), b0


def test_conv_matches_numpy(oracle_mod):
    w = W.c1()
    rng = np.random.default_rng(5)
    taps = rng.standard_normal(w.T)
    f = rng.standard_normal((3, w.UL))
    s = oracle_mod.conv_forward(w, taps, f)
    for k in range(3):
        full = np.convolve(f[k], taps)  # full[m'] = sum_t taps[t] f[m' - t]
        sU = np.zeros(w.UL)
        for m in range(w.UL):
            j = m - w.n_lo
            if 0 <= j < full.size:
                sU[m] = full[j]
        ref = sU.reshape(w.L, w.U).mean(axis=1)
        assert np.allclose(s[k], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_conv_adjoint_is_transpose(oracle_mod):
    w = W.c1()
    rng = np.random.default_rng(6)
    taps = rng.standard_normal(w.T)
    f = rng.standard_normal((2, w.UL))
    y = rng.standard_normal((2, w.L))
    lhs = (oracle_mod.conv_forward(w, taps, f) * y).sum()
    rhs = (f * oracle_mod.conv_adjoint(w, taps, y)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_eir_bandwidth():
    fc = 5e6
    par = W.gauss_sine_eir(fc, 0.8)
    s, tc = par[1], par[2]
    dt = 1e-10
    t = np.arange(0, par[3], dt)
    e = np.exp(-((t - tc) ** 2) / (2 * s * s)) * np.sin(2 * math.pi * fc * (t - tc))
    nfft = 1 << 20
    spec = np.abs(np.fft.rfft(e, nfft))
    fr = np.fft.rfftfreq(nfft, dt)
    band = fr[spec >= 0.5 * spec.max()]
    # the image at -fc and the +-4 sigma truncation move the edges by ~0.3 %
    assert (band.max() - band.min()) / fc == pytest.approx(0.8, rel=1e-2)
    assert fr[np.argmax(spec)] == pytest.approx(fc, rel=1e-2)


# ---------------------------------------------------------------------------
# Gaussian-modulated sine EIR (the one every benchmark system uses).  The
# references below are built in this file from Prop. 1, g(t) = -1/2 c t
# phi(|c t|), with h = e * g, the pulse e(t) = exp(-(t - tc)^2 / (2 s^2))
# sin(2 pi fc (t - tc)) on [0, Te] (whose bandwidth test_eir_bandwidth pins),
# and Eq. (def_bh) for the taps, integrated by scipy's adaptive
# Gauss-Kronrod quadrature, not by the oracle's fixed Gauss-Legendre panels.
# ---------------------------------------------------------------------------
def _gauss_sine_ref():
    integ = pytest.importorskip("scipy.integrate")
    w = W.c1()
    fc, s, tc, te = (float(v) for v in w.eir_par)
    c, kappa = float(w.c), float(w.kappa)

    def phi(r):  # bump radial function (1 - r^2 / kappa^2)^2 on [0, kappa)
        r = abs(r)
        return (1.0 - (r / kappa) ** 2) ** 2 if r < kappa else 0.0

    def g(t):
        return -0.5 * c * t * phi(c * t)

    def e(t):
        if t < 0.0 or t > te:
            return 0.0
        return math.exp(-((t - tc) ** 2) / (2.0 * s * s)) * math.sin(2.0 * math.pi * fc * (t - tc))

    kc = kappa / c

    def h(t):
        a, b = max(0.0, t - kc), min(te, t + kc)
        if not b > a:
            return 0.0
        pts = [t] if a < t < b else None
        val, _ = integ.quad(lambda tp: e(tp) * g(t - tp), a, b, points=pts, epsabs=0.0, epsrel=1e-13, limit=200)
        return val

    return w, integ, h, kc, te


def test_h_gauss_sine_eir_vs_adaptive_quadrature(oracle_mod):
    w, _, h, kc, te = _gauss_sine_ref()
    ts = np.linspace(-kc, te + kc, 29)[1:-1]
    ts = np.concatenate([ts, [0.5 * kc, te - 0.3 * kc, w.eir_par[2]]])
    ref = np.array([h(t) for t in ts])
    got = np.array([oracle_mod.h_value(w.rbf_kind, w.kappa, W.EIR_GAUSS_SINE, w.eir_par, w.c, t) for t in ts])
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(got - ref).max() <= 1e-11 * scale
    # outside the support [-kappa/c, Te + kappa/c] the response vanishes
    for t in (-1.01 * kc, te + 1.01 * kc):
        assert oracle_mod.h_value(w.rbf_kind, w.kappa, W.EIR_GAUSS_SINE, w.eir_par, w.c, t) == 0.0


def test_taps_gauss_sine_eir_vs_adaptive_quadrature(oracle_mod):
    """h-bar[n] = (1/D) int_{-D}^{D} (D - |s|) h(n D + s) ds (Eq. def_bh)."""
    w, integ, h, _, _ = _gauss_sine_ref()
    taps = oracle_mod.taps_for(w)
    D = 1.0 / (w.U * w.fs)
    peak = int(np.argmax(np.abs(taps)))
    picks = sorted({1, 7, peak - 40, peak, peak + 13, w.T // 2, w.T - 3})
    for t in picks:
        n = w.n_lo + t
        val, _ = integ.quad(lambda sv: (D - abs(sv)) * h(n * D + sv), -D, D, points=[0.0], epsabs=0.0, epsrel=1e-12,
                            limit=100)
        assert abs(taps[t] - val / D) <= 1e-11 * np.abs(taps).max(), (t, taps[t], val / D)
