// pat_geom_lut.cuh -- the cylinder's arc integral from the paper's lookup
// tables (Sec. 4.2.2, PAT_METHOD_LUT), in float-float.  Included by
// pat_geom.cuh after the cylinder helpers it uses (half_angle_u, cyl_fold_u,
// PairRange); not a standalone header.
#pragma once

#include "pat_internal.cuh"

namespace pat {

// ---------------------------------------------------------------------------
// Lookup-table variant of the cylinder (Sec. 4.2.2, PAT_METHOD_LUT).
//
// F(r) = alpha v_max + I(r) - beta v_min (Eq. area_D_l_xi) with the arc
// integral of Eq. (cyl_Il), I = 2 sqrt(q) [E(beta/2, nu) - E(alpha/2, nu)],
// q = r^2 - (R - rho)^2 (the paper's 2 R rho + b), nu = 4 R rho / q, and E
// read from the tables E~(s, m) = E(arcsin s, m), F~(s, m) = F(arcsin s, m)
// by bilinear interpolation: E(theta, nu) = E~(sin theta, nu) for nu <= 1;
// for nu > 1 the reciprocal-modulus transformation (Eq. reciprocal_modulus)
// with m = 1/nu gives sqrt(nu) [E~(s', m) - (1 - m) F~(s', m)] at
// s' = sqrt(nu) sin theta, and 2 sqrt(q) sqrt(nu) = 2 sqrt(4 R rho) is a
// per-pair constant.
//
// Precision: the terms of F are of the size of |a3| (u_max - u_min), while a
// group area is the difference of F at two edges a few per cent of the sweep
// apart; FP32 rounding of the table values, of their interpolation or of nu
// shows in the group areas at the 1e-4 .. 1e-3 level.  q, nu, the table
// values and F are therefore carried in float-float (about 48 bits, on the
// FP32 units: GB300 runs FP64 at 1/64 of its FP32 rate); only the small
// bilinear corrections (differences of neighbouring table values times the
// cell positions) are FP32.  The angles alpha, beta of unclamped bounds are
// FP32 half-angle results taken as exact: F is stationary in an unclamped
// bound (dF/dalpha = v_max - Psi(alpha) = 0), so their error enters at second
// order, provided the tables are read at the sine of that same angle, formed
// here in float-float.  Bounds at u = pi are pi itself (float-float), whose
// half-angle sine is 1.
// ---------------------------------------------------------------------------

// sin(u/2) for u in [0, pi], float-float: the Taylor series of sin x to the
// x^19 term (remainder below 3e-16 on |x| <= pi/2), the terms from x^11 on,
// below 1e-5 there, in FP32.
__device__ __forceinline__ float2 sin_half_ff(float2 u)
{
    const float2 x = ff_scale2(u, 0.5f), x2 = ff_sqr(x);
    const float y = x2.x;
    float t = fmaf(y, -8.22063525e-18f, 2.81145725e-15f);
    t = fmaf(y, t, -7.64716373e-13f);
    t = fmaf(y, t, 1.60590438e-10f);
    t = fmaf(y, t, -2.50521084e-08f); // x^11 / 11! .. x^19 / 19! over x^9
    float2 h = ff_add(make_float2(2.75573188e-06f, 3.79357122e-14f), make_float2(y * t, 0.f)); // 1/9!
    h = ff_add(make_float2(-1.98412701e-04f, 2.72559688e-12f), ff_mul(x2, h));                 // 1/7!
    h = ff_add(make_float2(8.33333377e-03f, -4.34617203e-10f), ff_mul(x2, h));                 // 1/5!
    h = ff_add(make_float2(-1.66666672e-01f, 4.96705388e-09f), ff_mul(x2, h));                 // 1/3!
    h = ff_add_f(ff_mul(x2, h), 1.f);
    return ff_mul(x, h);
}

// Cell c of a grid with g[c] <= z <= g[c+1] (z clamped into [0, top]) and
// the position w of z in it.  The inverse of Eq. (LUT_sampling),
// n = (N - 1) [1 - ((top - z) / top)^(1/4)], is taken in FP32 (two square
// roots); it can land one cell off next to a node, which the comparison with
// the float-float nodes corrects.
__device__ __forceinline__ int lut_cell(const float2 *g, const float *h, int N, float2 top, float2 z, float &w)
{
    if (z.x < 0.f) z = make_float2(0.f, 0.f);
    if (ff_lt(top, z)) z = top;
    const float y = ff_sub(top, z).x;
    const float nf = (float)(N - 1) * (1.f - sqrtf(sqrtf(y)));
    int c = min(max((int)nf, 0), N - 2);
    float2 g0 = __ldg(g + c);
    if (c > 0 && ff_lt(z, g0)) {
        --c;
        g0 = __ldg(g + c);
    } else if (c < N - 2) {
        const float2 g1 = __ldg(g + c + 1);
        if (ff_lt(g1, z)) {
            ++c;
            g0 = g1;
        }
    }
    w = ff_sub(z, g0).x * __ldg(h + c);
    return c;
}

// Per-edge part of the LUT arc integral, shared by the quadrants.
struct LutEdge {
    float2 pref;  // 2 sqrt(q) (nu <= 1) or 2 sqrt(4 R rho) (nu > 1)
    float2 sc;    // s' = sc s: 1, or sqrt(nu) for nu > 1
    float2 one_m; // nu > 1: 1 - m = 1 - 1/nu
    float wm;     // position of the table parameter in its cell
    int j;        // its cell
    bool big;     // nu > 1
};

__device__ __forceinline__ void lut_edge(const LutDev &L, float2 q, float2 fourRrho, float2 inv4, float2 P4,
                                         LutEdge &e)
{
    float2 m;
    e.big = ff_lt(q, fourRrho);
    if (e.big) {
        m = ff_mul(q, inv4); // 1 / nu
        if (!(m.x > 1e-30f)) m = make_float2(1e-30f, 0.f);
        e.sc = ff_div(make_float2(1.f, 0.f), ff_sqrt(m));
        e.one_m = ff_mul(ff_sub(fourRrho, q), inv4);
        e.pref = P4;
    } else {
        m = ff_div(fourRrho, q); // nu
        e.sc = make_float2(1.f, 0.f);
        e.one_m = make_float2(0.f, 0.f);
        e.pref = ff_scale2(ff_sqrt(q), 2.f);
    }
    e.j = lut_cell(L.gm, L.hm, L.nm, L.top, m, e.wm);
}

// E(theta, nu) (nu <= 1), or E(theta, nu) / sqrt(nu) (nu > 1), at the two
// bounds of a quadrant, s = sin(theta) = sb and sa, returning E(sb) - E(sa):
// both cells are found first and both cells' records are read together, so
// that the two chains of dependent reads overlap (5 % faster than one bound
// after the other).
__device__ __forceinline__ float2 lut_end_diff(const LutDev &L, const LutEdge &e, float2 sb, float2 sa)
{
    float wb, wa;
    const int ib = lut_cell(L.gs, L.hs, L.ns, L.top, e.big ? ff_mul(sb, e.sc) : sb, wb);
    const int ia = lut_cell(L.gs, L.hs, L.ns, L.top, e.big ? ff_mul(sa, e.sc) : sa, wa);
    const int cb = ib * (L.nm - 1) + e.j, ca = ia * (L.nm - 1) + e.j;
    const float4 ab = __ldg(L.A + cb), aa = __ldg(L.A + ca);
    const float4 bb = __ldg(L.B + cb), ba = __ldg(L.B + ca);
    const float wm = e.wm;
    float2 Eb = ff_add_f(make_float2(ab.x, ab.y), fmaf(wm, ab.z, wb * fmaf(wm, bb.x, ab.w)));
    float2 Ea = ff_add_f(make_float2(aa.x, aa.y), fmaf(wm, aa.z, wa * fmaf(wm, ba.x, aa.w)));
    if (e.big) {
        const float2 cb2 = __ldg(L.C + cb), ca2 = __ldg(L.C + ca);
        const float2 Fb = ff_add_f(make_float2(bb.y, bb.z), fmaf(wm, bb.w, wb * fmaf(wm, cb2.y, cb2.x)));
        const float2 Fa = ff_add_f(make_float2(ba.y, ba.z), fmaf(wm, ba.w, wa * fmaf(wm, ca2.y, ca2.x)));
        Eb = ff_sub(Eb, ff_mul(e.one_m, Fb));
        Ea = ff_sub(Ea, ff_mul(e.one_m, Fa));
    }
    return ff_sub(Eb, Ea);
}

// The record of one quadrant, kept small: the group loop indexes the
// records of a pair dynamically, so they live in the thread's stack frame,
// whose lines are evicted to DRAM as CTAs turn over; the squares of s and v
// are formed where they are used instead of stored (the same float-float
// products, so the same values).
struct LutQuad {
    float2 umin, umax; // angular bounds (FP32 fold; pi itself in float-float)
    float2 smin, smax; // sin(umin/2), sin(umax/2); their squares are the clamp thresholds of S = sin^2(u/2)
    float2 vmin, vmax; // axial bounds (v itself, not shifted)
};

// Clamped inverse Phi-hat(v, r) of Eq. (alphabeta), with s = sin(u/2) at it.
// S = sin^2(Phi/2) = (q - v^2) / (4 R rho).  The angle of an unclamped bound
// is the FP32 half-angle formula's, taken as exact (kept inside the quadrant,
// so that u/2 <= pi/2 and s is the sine of that same angle).
__device__ __forceinline__ float2 lut_bound(const LutQuad &Q, float2 q, float2 v2, float2 inv4, float2 &s)
{
    const float2 S = ff_mul(ff_sub(q, v2), inv4);
    if (!ff_lt(ff_sqr(Q.smin), S)) {
        s = Q.smin;
        return Q.umin;
    }
    if (!ff_lt(S, ff_sqr(Q.smax))) {
        s = Q.smax;
        return Q.umax;
    }
    float2 u = make_float2(half_angle_u(S.x, ff_sub(make_float2(1.f, 0.f), S).x), 0.f);
    if (ff_lt(u, Q.umin)) u = Q.umin;
    if (ff_lt(Q.umax, u)) u = Q.umax;
    s = sin_half_ff(u);
    return u;
}

// Group loop of one cylinder pair with the LUT arc integral (see above), in
// float-float from the pair's float-float set-up (frame coordinates, rho, r
// and q at the first edge); the sink gets FP32 shares as on the other paths.
// On the focal line (rho below about 1e-11 R, as on the exact path) Phi-hat
// only takes u_min or u_max and E(theta, 0) = theta: the tables are not read.
template <class Sink>
__device__ __forceinline__ void cyl_pair_lut(const TxDev &t, const TimeDev &tm, const PairRange &pr, int bmin,
                                             int bend, int ng, int dl, float inv_dl, float inv_last, Sink &sink)
{
    const LutDev &L = tm.lut;
    const float pi32 = 3.141592653589793f;
    const float2 pi_ff = make_float2(3.14159274e+00f, -8.74227766e-08f);
    float ui[2][2];
    const int nu = cyl_fold_u(t, pr.a1, pr.a2, ui);
    const float2 a3 = make_float2(pr.a3, pr.a3lo);
    const float2 v1 = ff_sub(ff_neg(t.fLz), a3), v2 = ff_sub(t.fLz, a3);
    const float2 vi[2][2] = {{ff_max0(v1), ff_max0(v2)}, {ff_max0(ff_neg(v2)), ff_max0(ff_neg(v1))}};
    const bool on_axis = !(4.f * t.R * pr.rho > 1e-12f * t.R * t.R);
    const float2 fourRrho = ff_scale2(ff_mul(t.fR, pr.ffrho), 4.f);
    const float2 inv4 = on_axis ? make_float2(0.f, 0.f) : ff_div(make_float2(1.f, 0.f), fourRrho);
    const float2 P4 = ff_scale2(ff_sqrt(fourRrho), 2.f);
    LutQuad Q[4];
    bool act[4];
    float2 Fp[4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            LutQuad &c = Q[2 * a + b];
            c.umin = ui[a][0] == pi32 ? pi_ff : make_float2(ui[a][0], 0.f);
            c.umax = ui[a][1] == pi32 ? pi_ff : make_float2(ui[a][1], 0.f);
            c.vmin = vi[b][0];
            c.vmax = vi[b][1];
            act[2 * a + b] = a < nu && ff_lt(c.umin, c.umax) && ff_lt(c.vmin, c.vmax); // else zero area
            c.smin = sin_half_ff(c.umin);
            c.smax = sin_half_ff(c.umax);
            Fp[2 * a + b] = ff_mul(c.umin, ff_sub(c.vmax, c.vmin)); // Phi-hat = umin before the sweep
        }
    // q = r^2 - (R - rho)^2 = q_b + tt (2 r_b + tt), tt = r - r_b
    const float2 qb = ff_add(pr.ffdb, ff_two_prod(pr.vc, pr.vc));
    const float2 two_rb = ff_scale2(pr.ffrb, 2.f);
    const float R = t.R;
    int e0 = bmin;
    for (int jg = 0; jg < ng; ++jg) {
        const int e1 = min(e0 + dl, bend);
        sink.pre(e0, e1);
        const float2 tt = ff_from_int_mul(e1 - bmin, tm.fdelta);
        const float2 q = ff_add(qb, ff_mul(tt, ff_add(two_rb, tt)));
        LutEdge ed;
        if (!on_axis) lut_edge(L, q, fourRrho, inv4, P4, ed);
        float2 area = make_float2(0.f, 0.f);
#pragma unroll 1 // one copy of the quadrant body: the unrolled loop is instruction-fetch bound (20 % slower)
        for (int i = 0; i < 4; ++i) {
            if (!act[i]) continue;
            const LutQuad &c = Q[i];
            float2 F;
            if (on_axis) {
                float2 b = ff_sqrt(q);
                if (ff_lt(b, c.vmin)) b = c.vmin;
                if (ff_lt(c.vmax, b)) b = c.vmax;
                F = ff_add(ff_mul(c.umax, ff_sub(b, c.vmin)), ff_mul(c.umin, ff_sub(c.vmax, b)));
            } else {
                float2 sa, sb;
                const float2 al = lut_bound(c, q, ff_sqr(c.vmax), inv4, sa); // alpha = Phi-hat(v_max)
                const float2 be = lut_bound(c, q, ff_sqr(c.vmin), inv4, sb); // beta = Phi-hat(v_min)
                F = ff_sub(ff_mul(al, c.vmax), ff_mul(be, c.vmin));
                if (ff_lt(al, be)) F = ff_add(F, ff_mul(ed.pref, lut_end_diff(L, ed, sb, sa)));
            }
            area = ff_add(area, ff_sub(F, Fp[i]));
            Fp[i] = F;
        }
        const float inv = jg == ng - 1 ? inv_last : inv_dl;
        sink.group(e0, e1, ff_mul_f(area, R).x * inv, 0.f);
        e0 = e1;
    }
}

} // namespace pat
