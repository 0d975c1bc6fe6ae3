/*
 * pat_oracle.c -- plain FP64 CPU oracle of the matrix-free photoacoustic
 * operator A (surface method and point method) and of its adjoint A^T.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA library; the two meet only
 * through the seeded input generators.
 *
 * Every step follows the paper (Do, Escande, Chaux, Gateau, Lee, "Scalable
 * photoacoustic tomography implementations accounting for the spatial impulse
 * response of transducers") in its order and notation; the functions cite the
 * section, equation or algorithm they restate.  Bins are 0-based: fine bin b
 * is the paper's l = b + 1, i.e. the interval [tau_b, tau_{b+1}) with
 * tau_b = t0 + b / (U Fs).
 *
 * Pinned by tests/test_oracle_*.py (see the header of each test module):
 *   - Carlson R_F, R_D and E, F (also for parameter > 1) against mpmath;
 *   - areas |M_i^l| of planes and cylinders against a 1-D Fubini integration
 *     of the area definition built from 3-D geometry (no closed form);
 *   - telescoped totals equal to the aperture area, on-axis piston plateau
 *     f_i[l] = 2 pi c, focal-line cylinder formula;
 *   - system-kernel taps against exact rational integration (box EIR), and
 *     h = e * g and the taps of the Gaussian-modulated sine EIR against
 *     adaptive Gauss-Kronrod quadrature of Prop. 1 and Eq. (def_bh);
 *   - the cylinder's point-method quadrature: points on the surface of
 *     Eq. (cylinder_param), areas summing to R 2 theta_max 2 Lz, midpoint
 *     sums of closed-form integrands, Q^-1 convergence to the surface
 *     method (Prop. 2);
 *   - the discrete convolution identity of the sampling operator (App. D);
 *   - the trapezoidal arc integral (Eq. trapezoid_Il): exact on the focal
 *     line (flat level curves), exact group totals, convergence to the exact
 *     areas as the strip narrows, its own dot-product test;
 *   - the lookup tables of E and F (Sec. 4.2.2): interpolated values against
 *     scipy's incomplete integrals within the bilinear error bound, second
 *     order in the grid step, the reciprocal-modulus branch against direct
 *     quadrature of the integrand, exact group totals, operator convergence
 *     to the exact areas as the tables grow, its own dot-product test;
 *   - the whole chain against the continuous model (Prop. 1 + Eq. 3,4) at
 *     growing U (Prop. 3), the point method against the surface method at
 *     growing Q (Prop. 2), translation/rotation invariance and the
 *     dot-product test <A x, y> = <x, A^T y> (App. G).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PLANE 0
#define OR_CYLINDER 1
#define OR_METHOD_SURFACE 0
#define OR_METHOD_POINT 1
#define OR_METHOD_TRAPEZOID 2 /* surface method, Eq. (trapezoid_Il) for the cylinder arc integral */
#define OR_METHOD_LUT 3       /* surface method, Eq. (cyl_Il) with E from the lookup tables of Sec. 4.2.2 */

/* Transducer descriptor: 16 doubles
 *   [0] kind, [1..3] c0, [4..6] e1, [7..9] e2,
 *   [10] L1, [11] L2 (plane half sizes),
 *   [12] R, [13] theta_max, [14] Lz (cylinder, c0 on the focal line). */
#define TXS 16

typedef struct {
    double c, fs, t0;
    int L, U, dl;
} otime;

static otime mk_time(const double *tp, const int *ip)
{
    otime t;
    t.c = tp[0];
    t.fs = tp[1];
    t.t0 = tp[2];
    t.L = ip[0];
    t.U = ip[1];
    t.dl = ip[2];
    return t;
}

/* ------------------------------------------------------------------------ */
/* Carlson symmetric integrals by the duplication theorem (DLMF 19.26.18,    */
/* series of DLMF 19.36.1 and 19.36.2; B. C. Carlson, Numer. Algorithms 10,  */
/* 1995).  FP64, iterated until the relative spread is below 1e-4 so that    */
/* the fifth-order series is exact to far below double rounding.             */
/* ------------------------------------------------------------------------ */
static double carlson_rf(double x, double y, double z)
{
    for (int it = 0; it < 200; ++it) {
        double A = (x + y + z) / 3.0;
        double X = 1.0 - x / A, Y = 1.0 - y / A, Z = 1.0 - z / A;
        double dev = fmax(fabs(X), fmax(fabs(Y), fabs(Z)));
        if (dev < 1e-4) {
            double E2 = X * Y - Z * Z;
            double E3 = X * Y * Z;
            return (1.0 - E2 / 10.0 + E3 / 14.0 + E2 * E2 / 24.0 - 3.0 * E2 * E3 / 44.0) / sqrt(A);
        }
        double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
        double lam = sx * sy + sy * sz + sz * sx;
        x = 0.25 * (x + lam);
        y = 0.25 * (y + lam);
        z = 0.25 * (z + lam);
    }
    return NAN;
}

static double carlson_rd(double x, double y, double z)
{
    double sum = 0.0, fac = 1.0;
    for (int it = 0; it < 200; ++it) {
        double A = (x + y + 3.0 * z) / 5.0;
        double X = 1.0 - x / A, Y = 1.0 - y / A, Z = 1.0 - z / A;
        double dev = fmax(fabs(X), fmax(fabs(Y), fabs(Z)));
        if (dev < 1e-4) {
            double XY = X * Y, Z2 = Z * Z;
            double E2 = XY - 6.0 * Z2;
            double E3 = (3.0 * XY - 8.0 * Z2) * Z;
            double E4 = 3.0 * (XY - Z2) * Z2;
            double E5 = XY * Z2 * Z;
            double ser = 1.0 - 3.0 * E2 / 14.0 + E3 / 6.0 + 9.0 * E2 * E2 / 88.0 - 3.0 * E4 / 22.0
                         - 9.0 * E2 * E3 / 52.0 + 3.0 * E5 / 26.0;
            return 3.0 * sum + fac * ser / (A * sqrt(A));
        }
        double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
        double lam = sx * sy + sy * sz + sz * sx;
        sum += fac / (sz * (z + lam));
        fac *= 0.25;
        x = 0.25 * (x + lam);
        y = 0.25 * (y + lam);
        z = 0.25 * (z + lam);
    }
    return NAN;
}

/* Incomplete integrals of the first and second kind, parameter m in [0,1],
 * amplitude phi in [0, pi/2] (DLMF 19.25.5, 19.25.9). */
static double ellip_f(double phi, double m)
{
    double s = sin(phi), c = cos(phi);
    if (s == 0.0) return 0.0;
    /* 1 - m sin^2 = cos^2 + (1 - m) sin^2, free of cancellation near (pi/2, 1) */
    return s * carlson_rf(c * c, c * c + (1.0 - m) * s * s, 1.0);
}

static double ellip_e(double phi, double m)
{
    double s = sin(phi), c = cos(phi);
    if (s == 0.0) return 0.0;
    if (m == 1.0) return s; /* E(phi,1) = sin(phi) */
    double y = c * c + (1.0 - m) * s * s;
    return s * carlson_rf(c * c, y, 1.0) - (m / 3.0) * s * s * s * carlson_rd(c * c, y, 1.0);
}

/* E(theta, nu) for any nu >= 0 with nu sin^2(theta) <= 1: the definition of
 * Eq. (cyl_Il) for nu <= 1, the reciprocal-modulus transformation of
 * Eq. (reciprocal_modulus) for nu > 1. */
static double ellip_e_any(double theta, double nu)
{
    if (nu <= 1.0) return ellip_e(theta, nu);
    double sn = sqrt(nu) * sin(theta);
    if (sn > 1.0) sn = 1.0; /* Lemma 6 keeps it <= 1; rounding may not */
    double tt = asin(sn);
    double m = 1.0 / nu;
    double corr = (m == 1.0 || sn == 0.0) ? 0.0 : (1.0 - m) * ellip_f(tt, m);
    return sqrt(nu) * (ellip_e(tt, m) - corr);
}

double oracle_carlson_rf(double x, double y, double z) { return carlson_rf(x, y, z); }
double oracle_carlson_rd(double x, double y, double z) { return carlson_rd(x, y, z); }
double oracle_ellip_f(double phi, double m) { return ellip_f(phi, m); }
double oracle_ellip_e(double phi, double m) { return ellip_e(phi, m); }
double oracle_ellip_e_any(double theta, double nu) { return ellip_e_any(theta, nu); }

/* ------------------------------------------------------------------------ */
/* Pair geometry (Sec. 4: separable form, four-quadrant decomposition).      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double umin, umax, vmin, vmax;
} oquad;

typedef struct {
    int kind;
    double a[3];     /* voxel in the transducer frame */
    double rho, thi; /* cylinder: polar coordinates of the voxel */
    double R;
    double J0;
    int nq;
    oquad q[4];
    double rmin, rmax;
} opair;

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static double psi_of(const opair *p, double u)
{
    if (p->kind == OR_PLANE) return u * u + p->a[2] * p->a[2]; /* Sec. 4.1 */
    return p->rho * p->rho + p->R * p->R - 2.0 * p->R * p->rho * cos(u); /* Sec. 4.2.1 */
}

/* Wrap an angle into (-pi, pi]. */
static double wrap_pi(double x)
{
    while (x > M_PI) x -= 2.0 * M_PI;
    while (x <= -M_PI) x += 2.0 * M_PI;
    return x;
}

static void add_quads(opair *p, int nu, const double (*ui)[2], const double v1, const double v2)
{
    /* v intervals of Eq. (uvminmax) */
    double vi[2][2] = {{fmax(v1, 0.0), fmax(v2, 0.0)}, {fmax(-v2, 0.0), fmax(-v1, 0.0)}};
    for (int a = 0; a < nu; ++a)
        for (int b = 0; b < 2; ++b) {
            if (!(ui[a][1] > ui[a][0]) || !(vi[b][1] > vi[b][0])) continue; /* degenerate: zero area */
            oquad *q = &p->q[p->nq++];
            q->umin = ui[a][0];
            q->umax = ui[a][1];
            q->vmin = vi[b][0];
            q->vmax = vi[b][1];
        }
}

static void pair_setup(const double *tx, const double *x, opair *p)
{
    const double *c0 = tx + 1, *e1 = tx + 4, *e2 = tx + 7;
    double n[3], d[3] = {x[0] - c0[0], x[1] - c0[1], x[2] - c0[2]};
    cross3(e1, e2, n);
    p->kind = (int)tx[0];
    p->nq = 0;
    if (p->kind == OR_PLANE) {
        /* Eq. (plane_param): frame (e1, e2, e1 x e2) centred at c0 */
        p->a[0] = dot3(e1, d);
        p->a[1] = dot3(e2, d);
        p->a[2] = dot3(n, d);
        p->J0 = 1.0;
        p->R = 0.0;
        double L1 = tx[10], L2 = tx[11];
        double u1 = -L1 - p->a[0], u2 = L1 - p->a[0];
        double v1 = -L2 - p->a[1], v2 = L2 - p->a[1];
        double ui[2][2] = {{fmax(u1, 0.0), fmax(u2, 0.0)}, {fmax(-u2, 0.0), fmax(-u1, 0.0)}};
        add_quads(p, 2, (const double(*)[2])ui, v1, v2);
    } else {
        /* Eq. (cylinder_param): frame (e2, e1 x e2, e1) centred at the focal-line point c0 */
        p->a[0] = dot3(e2, d);
        p->a[1] = dot3(n, d);
        p->a[2] = dot3(e1, d);
        p->R = tx[12];
        p->J0 = p->R;
        double thmax = tx[13], Lz = tx[14];
        p->rho = sqrt(p->a[0] * p->a[0] + p->a[1] * p->a[1]);
        p->thi = atan2(p->a[1], p->a[0]);
        double u1 = wrap_pi(-thmax - p->thi), u2 = wrap_pi(thmax - p->thi);
        double ui[2][2];
        int nu;
        /* Eq. (folded_intervals) */
        if (u1 < 0.0 && 0.0 < u2) {
            ui[0][0] = 0.0; ui[0][1] = -u1;
            ui[1][0] = 0.0; ui[1][1] = u2;
            nu = 2;
        } else if (u2 < u1) {
            ui[0][0] = u1; ui[0][1] = M_PI;
            ui[1][0] = -u2; ui[1][1] = M_PI;
            nu = 2;
        } else if (0.0 <= u1) {
            ui[0][0] = u1; ui[0][1] = u2;
            nu = 1;
        } else {
            ui[0][0] = -u2; ui[0][1] = -u1;
            nu = 1;
        }
        add_quads(p, nu, (const double(*)[2])ui, -Lz - p->a[2], Lz - p->a[2]);
    }
    /* Eq. (closedform_rminrmax): corner radii of each quadrant, then min / max */
    p->rmin = INFINITY;
    p->rmax = 0.0;
    for (int i = 0; i < p->nq; ++i) {
        const oquad *q = &p->q[i];
        double r0 = sqrt(psi_of(p, q->umin) + q->vmin * q->vmin);
        double r1 = sqrt(psi_of(p, q->umax) + q->vmax * q->vmax);
        if (r0 < p->rmin) p->rmin = r0;
        if (r1 > p->rmax) p->rmax = r1;
    }
}

/* Clamped inverse Phi-hat(v, r) of Sec. 4 (three cases). */
static double phi_hat(const opair *p, const oquad *q, double v, double r)
{
    double xx = r * r - v * v;
    if (xx <= psi_of(p, q->umin)) return q->umin;
    if (xx >= psi_of(p, q->umax)) return q->umax;
    if (p->kind == OR_PLANE) return sqrt(xx - p->a[2] * p->a[2]); /* Sec. 4.1 */
    double arg = (p->rho * p->rho + p->R * p->R - xx) / (2.0 * p->R * p->rho); /* Sec. 4.2.1 */
    if (arg > 1.0) arg = 1.0;
    if (arg < -1.0) arg = -1.0;
    return acos(arg);
}

/* ------------------------------------------------------------------------ */
/* Lookup tables (Sec. 4.2.2): E~(s, m) = E(arcsin s, m) and                 */
/* F~(s, m) = F(arcsin s, m) on the power-law grid of Eq. (LUT_sampling),    */
/* g_n = (1 - eps) [1 - (1 - n / (N - 1))^4], n = 0 .. N - 1 (0-based), for  */
/* both s and m, eps = 1e-16; a query is interpolated bilinearly in the cell */
/* that holds it.  The tables of one (N_s, N_m) are built once, from the     */
/* Carlson forms above, and kept.                                            */
/* ------------------------------------------------------------------------ */
#define OR_LUT_EPS 1e-16

typedef struct {
    int ns, nm;
    double *gs, *gm; /* grid nodes of s and m */
    double *E, *F;   /* [ns][nm] */
} olut;

static olut g_lut = {0, 0, NULL, NULL, NULL, NULL};

static double lut_node(int n, int N)
{
    double x = 1.0 - (double)n / (double)(N - 1);
    return (1.0 - OR_LUT_EPS) * (1.0 - x * x * x * x);
}

/* Not thread-safe: called before any parallel region. */
static const olut *lut_get(int ns, int nm)
{
    if (ns < 2 || nm < 2) return NULL;
    if (g_lut.ns == ns && g_lut.nm == nm) return &g_lut;
    free(g_lut.gs);
    free(g_lut.gm);
    free(g_lut.E);
    free(g_lut.F);
    g_lut.ns = ns;
    g_lut.nm = nm;
    g_lut.gs = (double *)malloc(sizeof(double) * (size_t)ns);
    g_lut.gm = (double *)malloc(sizeof(double) * (size_t)nm);
    g_lut.E = (double *)malloc(sizeof(double) * (size_t)ns * (size_t)nm);
    g_lut.F = (double *)malloc(sizeof(double) * (size_t)ns * (size_t)nm);
    for (int i = 0; i < ns; ++i) g_lut.gs[i] = lut_node(i, ns);
    for (int j = 0; j < nm; ++j) g_lut.gm[j] = lut_node(j, nm);
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < ns; ++i) {
        double phi = asin(g_lut.gs[i]);
        for (int j = 0; j < nm; ++j) {
            g_lut.E[(size_t)i * nm + j] = ellip_e(phi, g_lut.gm[j]);
            g_lut.F[(size_t)i * nm + j] = ellip_f(phi, g_lut.gm[j]);
        }
    }
    return &g_lut;
}

/* Cell c with g[c] <= z <= g[c+1] (z clamped into [g_0, g_{N-1}]), from the
 * inverse of Eq. (LUT_sampling), n = (N - 1) [1 - (1 - z / (1 - eps))^(1/4)]
 * (two square roots), then moved by whole cells until it holds z; *w is the
 * position of z in the cell. */
static int lut_cell(const double *g, int N, double z, double *w)
{
    if (z < 0.0) z = 0.0;
    if (z > g[N - 1]) z = g[N - 1];
    double y = 1.0 - z / (1.0 - OR_LUT_EPS);
    double x = 1.0 - sqrt(sqrt(y > 0.0 ? y : 0.0));
    int c = (int)floor(x * (double)(N - 1));
    if (c < 0) c = 0;
    if (c > N - 2) c = N - 2;
    while (c < N - 2 && z > g[c + 1]) ++c;
    while (c > 0 && z < g[c]) --c;
    *w = (z - g[c]) / (g[c + 1] - g[c]);
    return c;
}

static double lut_bilinear(const olut *t, const double *T, double s, double m)
{
    double ws, wm;
    int i = lut_cell(t->gs, t->ns, s, &ws);
    int j = lut_cell(t->gm, t->nm, m, &wm);
    const double *r0 = T + (size_t)i * t->nm + j, *r1 = r0 + t->nm;
    return (1.0 - ws) * ((1.0 - wm) * r0[0] + wm * r0[1]) + ws * ((1.0 - wm) * r1[0] + wm * r1[1]);
}

/* E(theta, nu) from the tables: E~(sin theta, nu) for nu <= 1; for nu > 1 the
 * reciprocal-modulus transformation of Eq. (reciprocal_modulus) with
 * sin(theta~) = sqrt(nu) sin(theta), on E~ and F~ at parameter 1 / nu. */
static double ellip_e_lut(const olut *t, double theta, double nu)
{
    if (nu <= 1.0) return lut_bilinear(t, t->E, sin(theta), nu);
    double sn = sqrt(nu) * sin(theta);
    if (sn > 1.0) sn = 1.0; /* Lemma 6 keeps it <= 1; rounding may not */
    double m = 1.0 / nu;
    return sqrt(nu) * (lut_bilinear(t, t->E, sn, m) - (1.0 - m) * lut_bilinear(t, t->F, sn, m));
}

double oracle_ellip_e_lut(double theta, double nu, int ns, int nm)
{
    const olut *t = lut_get(ns, nm);
    return t ? ellip_e_lut(t, theta, nu) : NAN;
}

double oracle_lut_node(int n, int N) { return lut_node(n, N); }

/* I(r) = integral of Psi(u, r) over [alpha, beta]: Eq. (plane_primitive) for
 * the plane, Eq. (cyl_Il) with Lemma 6 for the cylinder, E exact or (lut not
 * NULL) from the lookup tables.  On the focal line (rho = 0) E(theta, 0) =
 * theta and I is (beta - alpha) sqrt(q) in both cases. */
static double arc_integral(const opair *p, double alpha, double beta, double r, const olut *lut)
{
    if (!(beta > alpha)) return 0.0;
    if (p->kind == OR_PLANE) {
        double rho2 = r * r - p->a[2] * p->a[2];
        if (rho2 <= 0.0) return 0.0;
        double rho = sqrt(rho2);
        double ub[2] = {alpha, beta}, F[2];
        for (int i = 0; i < 2; ++i) {
            double u = ub[i];
            double w = rho2 - u * u;
            double s = u / rho;
            if (w < 0.0) w = 0.0;
            if (s > 1.0) s = 1.0;
            if (s < -1.0) s = -1.0;
            F[i] = 0.5 * (u * sqrt(w) + rho2 * asin(s));
        }
        return F[1] - F[0];
    }
    double R = p->R, rho = p->rho;
    double b = r * r - rho * rho - R * R;
    double q = 2.0 * R * rho + b;
    if (q <= 0.0) return 0.0; /* Lemma 6: degenerate, integral vanishes */
    if (rho == 0.0) return (beta - alpha) * sqrt(q);
    double nu = 4.0 * R * rho / q;
    if (lut) return 2.0 * sqrt(q) * (ellip_e_lut(lut, 0.5 * beta, nu) - ellip_e_lut(lut, 0.5 * alpha, nu));
    return 2.0 * sqrt(q) * (ellip_e_any(0.5 * beta, nu) - ellip_e_any(0.5 * alpha, nu));
}

/* Trapezoidal approximation of I_l (Eq. trapezoid_Il): the level curve
 * between (alpha, Psi(alpha)) and (beta, Psi(beta)) replaced by its chord,
 * Psi(u, r) = sqrt(r^2 - psi(u)) the height at angle u.  Used for the
 * cylinder only; a plane keeps its closed form. */
static double arc_integral_trapezoid(const opair *p, double alpha, double beta, double r)
{
    if (!(beta > alpha)) return 0.0;
    if (p->kind == OR_PLANE) return arc_integral(p, alpha, beta, r, NULL);
    double ha = r * r - psi_of(p, alpha), hb = r * r - psi_of(p, beta);
    return 0.5 * (beta - alpha) * (sqrt(ha > 0.0 ? ha : 0.0) + sqrt(hb > 0.0 ? hb : 0.0));
}

/* Group areas of one pair (Alg. 4 with the coarser area grid of Remark 1).
 * Bins [b_min, b_max] from Eq. (rmin_rmax); group j covers the fine bins
 * [b_min + j dl, min(b_min + (j+1) dl, b_max + 1)).  Returns the number of
 * groups written into areas[] (grown on demand).  method: the I_l of
 * OR_METHOD_SURFACE (exact), OR_METHOD_TRAPEZOID or OR_METHOD_LUT (tables
 * lut). */
static int pair_group_areas(const opair *p, const otime *tm, int64_t *bmin_out, int64_t *bmax_out,
                            double **areas, int *cap, int method, const olut *lut)
{
    const double ufs = (double)tm->U * tm->fs;
    int64_t bmin = (int64_t)floor((p->rmin / tm->c - tm->t0) * ufs);
    int64_t bmax = (int64_t)ceil((p->rmax / tm->c - tm->t0) * ufs) - 1;
    if (p->nq == 0 || bmax < bmin) {
        *bmin_out = 0;
        *bmax_out = -1;
        return 0;
    }
    int64_t nb = bmax - bmin + 1;
    int ng = (int)((nb + tm->dl - 1) / tm->dl);
    if (ng > *cap) {
        *cap = ng + 64;
        *areas = (double *)realloc(*areas, sizeof(double) * (size_t)(*cap));
    }
    /* stored (alpha, beta, I) per quadrant, initialised to (u_min, u_min, 0) */
    double al[4], be[4], Il[4];
    for (int i = 0; i < p->nq; ++i) {
        al[i] = p->q[i].umin;
        be[i] = p->q[i].umin;
        Il[i] = 0.0;
    }
    for (int j = 0; j < ng; ++j) {
        int64_t e1 = bmin + (int64_t)(j + 1) * tm->dl;
        if (e1 > bmax + 1) e1 = bmax + 1;
        double r = tm->c * (tm->t0 + (double)e1 / ufs); /* edge c tau at the group's upper end */
        double area = 0.0;
        for (int i = 0; i < p->nq; ++i) {
            const oquad *q = &p->q[i];
            double a = phi_hat(p, q, q->vmax, r); /* Eq. (alphabeta) */
            double bb = phi_hat(p, q, q->vmin, r);
            double I = method == OR_METHOD_TRAPEZOID ? arc_integral_trapezoid(p, a, bb, r)
                       : arc_integral(p, a, bb, r, method == OR_METHOD_LUT ? lut : NULL);
            /* Eq. (area_D_l_xi) and Eq. (swept_u) */
            area += p->J0 * ((a - al[i]) * q->vmax + I - Il[i] - (bb - be[i]) * q->vmin);
            al[i] = a;
            be[i] = bb;
            Il[i] = I;
        }
        (*areas)[j] = area;
    }
    *bmin_out = bmin;
    *bmax_out = bmax;
    return ng;
}

static void voxel_pos(const int *n, const double *origin, double pitch, int64_t i, double *x)
{
    int64_t ix = i % n[0], iy = (i / n[0]) % n[1], iz = i / ((int64_t)n[0] * n[1]);
    x[0] = origin[0] + pitch * (double)ix;
    x[1] = origin[1] + pitch * (double)iy;
    x[2] = origin[2] + pitch * (double)iz;
}

/* Exported: the pair's bin range and per-fine-bin areas |M_i^l| (each group
 * area split evenly over its fine bins, Remark 1).  out_area has room for
 * cap entries; returns the number of fine bins or -needed when too small.
 * method: OR_METHOD_SURFACE, or OR_METHOD_TRAPEZOID for Eq. (trapezoid_Il). */
int64_t oracle_pair_bin_areas_m(const double *tx, const double *x, const double *tp, const int *ip, int method,
                                int q1, int q2, int64_t *b_min, double *out_area, int64_t cap)
{
    otime tm = mk_time(tp, ip);
    opair p;
    pair_setup(tx, x, &p);
    double *areas = NULL;
    int acap = 0;
    int64_t bmin, bmax;
    const olut *lut = method == OR_METHOD_LUT ? lut_get(q1, q2) : NULL;
    int ng = pair_group_areas(&p, &tm, &bmin, &bmax, &areas, &acap, method, lut);
    int64_t nb = bmax - bmin + 1;
    *b_min = bmin;
    if (nb > cap) {
        free(areas);
        return -nb;
    }
    for (int j = 0; j < ng; ++j) {
        int64_t e0 = bmin + (int64_t)j * tm.dl, e1 = e0 + tm.dl;
        if (e1 > bmax + 1) e1 = bmax + 1;
        for (int64_t b = e0; b < e1; ++b) out_area[b - bmin] = areas[j] / (double)(e1 - e0);
    }
    free(areas);
    return nb < 0 ? 0 : nb;
}

int64_t oracle_pair_bin_areas(const double *tx, const double *x, const double *tp, const int *ip,
                              int64_t *b_min, double *out_area, int64_t cap)
{
    return oracle_pair_bin_areas_m(tx, x, tp, ip, OR_METHOD_SURFACE, 0, 0, b_min, out_area, cap);
}

/* Exported: r_min, r_max of Eq. (rmin_rmax) and the quadrant count. */
int oracle_pair_range(const double *tx, const double *x, double *out)
{
    opair p;
    pair_setup(tx, x, &p);
    out[0] = p.rmin;
    out[1] = p.rmax;
    return p.nq;
}

/* ------------------------------------------------------------------------ */
/* Point-detector quadrature (Sec. 3.2): Q1 x Q2 cell centres of D, with     */
/* Delta q_j = J0 * cell area.                                               */
/* ------------------------------------------------------------------------ */
static void quad_point(const double *tx, int q1, int q2, int j1, int j2, double *pt, double *dq)
{
    const double *c0 = tx + 1, *e1 = tx + 4, *e2 = tx + 7;
    double n[3];
    cross3(e1, e2, n);
    if ((int)tx[0] == OR_PLANE) {
        double L1 = tx[10], L2 = tx[11];
        double x1 = -L1 + (j1 + 0.5) * 2.0 * L1 / q1;
        double x2 = -L2 + (j2 + 0.5) * 2.0 * L2 / q2;
        for (int d = 0; d < 3; ++d) pt[d] = c0[d] + x1 * e1[d] + x2 * e2[d];
        *dq = (2.0 * L1 / q1) * (2.0 * L2 / q2);
    } else {
        double R = tx[12], thmax = tx[13], Lz = tx[14];
        double th = -thmax + (j1 + 0.5) * 2.0 * thmax / q1;
        double z = -Lz + (j2 + 0.5) * 2.0 * Lz / q2;
        for (int d = 0; d < 3; ++d) pt[d] = c0[d] + R * cos(th) * e2[d] + R * sin(th) * n[d] + z * e1[d];
        *dq = R * (2.0 * thmax / q1) * (2.0 * Lz / q2);
    }
}

/* Exported for the tests: the Q1 x Q2 points (pts[3 j], j = j1 q2 + j2) and
 * their areas dq[j] of one element, as Alg. 2 uses them. */
void oracle_quad_points(const double *tx, int q1, int q2, double *pts, double *dq)
{
    for (int j1 = 0; j1 < q1; ++j1)
        for (int j2 = 0; j2 < q2; ++j2) {
            const int j = j1 * q2 + j2;
            quad_point(tx, q1, q2, j1, j2, pts + 3 * (size_t)j, dq + j);
        }
}

/* ------------------------------------------------------------------------ */
/* Geometric assembly: f_k (Alg. 2 / Alg. 3) and its transpose (Alg. 6 / 7). */
/* ------------------------------------------------------------------------ */
/* f: [K][U L], overwritten.  x holds n_vox values for the voxels vox_idx
 * (vox_idx == NULL: all N voxels, x[i]).  Returns the number of dropped
 * contributions (bins outside [0, UL)). */
int64_t oracle_geometric_forward(const int *n, const double *origin, double pitch, const double *tx, int K,
                                 const double *tp, const int *ip, int method, int q1, int q2,
                                 const int64_t *vox_idx, int64_t n_vox, const double *x, double *f)
{
    otime tm = mk_time(tp, ip);
    const int64_t UL = (int64_t)tm.U * tm.L;
    const double ufs = (double)tm.U * tm.fs;
    int64_t dropped = 0;
    const olut *lut = method == OR_METHOD_LUT ? lut_get(q1, q2) : NULL; /* q1 x q2 = N_s x N_m */
    if (!vox_idx) n_vox = (int64_t)n[0] * n[1] * n[2];
    memset(f, 0, sizeof(double) * (size_t)UL * (size_t)K);
    for (int k = 0; k < K; ++k) {
        const double *t = tx + (size_t)k * TXS;
        double *fk = f + (size_t)k * UL;
#pragma omp parallel reduction(+ : dropped)
        {
            double *loc = (double *)calloc((size_t)UL, sizeof(double));
            double *areas = NULL;
            int acap = 0;
#pragma omp for schedule(dynamic, 16)
            for (int64_t v = 0; v < n_vox; ++v) {
                double xv = x[v];
                if (xv == 0.0) continue;
                int64_t i = vox_idx ? vox_idx[v] : v;
                double xi[3];
                voxel_pos(n, origin, pitch, i, xi);
                if (method == OR_METHOD_POINT) {
                    /* Alg. 2 */
                    for (int j1 = 0; j1 < q1; ++j1)
                        for (int j2 = 0; j2 < q2; ++j2) {
                            double pt[3], dq;
                            quad_point(t, q1, q2, j1, j2, pt, &dq);
                            double d[3] = {pt[0] - xi[0], pt[1] - xi[1], pt[2] - xi[2]};
                            double r = sqrt(dot3(d, d));
                            int64_t b = (int64_t)floor((r / tm.c - tm.t0) * ufs);
                            if (b < 0 || b >= UL) {
                                dropped++;
                                continue;
                            }
                            loc[b] += ufs * xv * dq / r;
                        }
                } else {
                    /* Alg. 3 with Remark 1 */
                    opair p;
                    pair_setup(t, xi, &p);
                    int64_t bmin, bmax;
                    int ng = pair_group_areas(&p, &tm, &bmin, &bmax, &areas, &acap, method, lut);
                    for (int j = 0; j < ng; ++j) {
                        int64_t e0 = bmin + (int64_t)j * tm.dl, e1 = e0 + tm.dl;
                        if (e1 > bmax + 1) e1 = bmax + 1;
                        double share = areas[j] / (double)(e1 - e0);
                        for (int64_t b = e0; b < e1; ++b) {
                            if (b < 0 || b >= UL) {
                                dropped++;
                                continue;
                            }
                            double tau_mid = tm.t0 + ((double)b + 0.5) / ufs;
                            loc[b] += ufs * xv * share / (tm.c * tau_mid); /* Eq. (ui_area) */
                        }
                    }
                }
            }
#pragma omp critical
            for (int64_t b = 0; b < UL; ++b) fk[b] += loc[b];
            free(loc);
            free(areas);
        }
    }
    return dropped;
}

/* z: [n_vox] (vox_idx == NULL: all N voxels), overwritten; v: [K][U L]. */
int64_t oracle_geometric_adjoint(const int *n, const double *origin, double pitch, const double *tx, int K,
                                 const double *tp, const int *ip, int method, int q1, int q2, const double *v,
                                 const int64_t *vox_idx, int64_t n_vox, double *z)
{
    otime tm = mk_time(tp, ip);
    const int64_t UL = (int64_t)tm.U * tm.L;
    const double ufs = (double)tm.U * tm.fs;
    int64_t dropped = 0;
    const olut *lut = method == OR_METHOD_LUT ? lut_get(q1, q2) : NULL; /* q1 x q2 = N_s x N_m */
    if (!vox_idx) n_vox = (int64_t)n[0] * n[1] * n[2];
#pragma omp parallel reduction(+ : dropped)
    {
        double *areas = NULL;
        int acap = 0;
#pragma omp for schedule(dynamic, 4)
        for (int64_t vv = 0; vv < n_vox; ++vv) {
            int64_t i = vox_idx ? vox_idx[vv] : vv;
            double xi[3];
            voxel_pos(n, origin, pitch, i, xi);
            double zi = 0.0;
            for (int k = 0; k < K; ++k) {
                const double *t = tx + (size_t)k * TXS;
                const double *vk = v + (size_t)k * UL;
                if (method == OR_METHOD_POINT) {
                    /* Alg. 6 */
                    for (int j1 = 0; j1 < q1; ++j1)
                        for (int j2 = 0; j2 < q2; ++j2) {
                            double pt[3], dq;
                            quad_point(t, q1, q2, j1, j2, pt, &dq);
                            double d[3] = {pt[0] - xi[0], pt[1] - xi[1], pt[2] - xi[2]};
                            double r = sqrt(dot3(d, d));
                            int64_t b = (int64_t)floor((r / tm.c - tm.t0) * ufs);
                            if (b < 0 || b >= UL) {
                                dropped++;
                                continue;
                            }
                            zi += ufs * dq * vk[b] / r;
                        }
                } else {
                    /* Alg. 7 with the coarser-grid gather of App. G */
                    opair p;
                    pair_setup(t, xi, &p);
                    int64_t bmin, bmax;
                    int ng = pair_group_areas(&p, &tm, &bmin, &bmax, &areas, &acap, method, lut);
                    for (int j = 0; j < ng; ++j) {
                        int64_t e0 = bmin + (int64_t)j * tm.dl, e1 = e0 + tm.dl;
                        if (e1 > bmax + 1) e1 = bmax + 1;
                        double acc = 0.0;
                        for (int64_t b = e0; b < e1; ++b) {
                            if (b < 0 || b >= UL) {
                                dropped++;
                                continue;
                            }
                            double tau_mid = tm.t0 + ((double)b + 0.5) / ufs;
                            acc += vk[b] / (tm.c * tau_mid);
                        }
                        zi += ufs * areas[j] / (double)(e1 - e0) * acc;
                    }
                }
            }
            z[vv] = zi;
        }
        free(areas);
    }
    return dropped;
}

/* ------------------------------------------------------------------------ */
/* Discrete convolution and downsampling (Eq. discrete_conv, App. D) and     */
/* their transposes (App. G).  h-bar[n] = taps[n - n_lo], n in [n_lo, n_lo+T) */
/* ------------------------------------------------------------------------ */
void oracle_conv_forward(const double *taps, int T, int n_lo, int U, int L, int K, const double *f, double *s)
{
    const int64_t UL = (int64_t)U * L;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < K; ++k) {
        const double *fk = f + (size_t)k * UL;
        double *sk = s + (size_t)k * L;
        for (int l = 0; l < L; ++l) {
            double acc = 0.0;
            for (int j = 0; j < U; ++j) {
                int64_t m = (int64_t)U * l + j; /* fine index of s^U */
                double sU = 0.0;
                for (int t = 0; t < T; ++t) {
                    int64_t b = m - (n_lo + t); /* h-bar[m - b] f[b] */
                    if (b < 0 || b >= UL) continue;
                    sU += taps[t] * fk[b];
                }
                acc += sU;
            }
            sk[l] = acc / U; /* Eq. (def_downsampling) */
        }
    }
}

void oracle_conv_adjoint(const double *taps, int T, int n_lo, int U, int L, int K, const double *s, double *v)
{
    const int64_t UL = (int64_t)U * L;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < K; ++k) {
        const double *sk = s + (size_t)k * L;
        double *vk = v + (size_t)k * UL;
        /* up = downsampling transpose: each sample replicated over its U fine bins, / U */
        for (int64_t b = 0; b < UL; ++b) {
            double acc = 0.0;
            for (int t = 0; t < T; ++t) {
                int64_t m = b + n_lo + t; /* correlation with h-bar^- : sum_m h-bar[m - b] up[m] */
                if (m < 0 || m >= UL) continue;
                acc += taps[t] * sk[m / U] / U;
            }
            vk[b] = acc;
        }
    }
}

/* Whole operator, Alg. 1: geometric assembly then convolution + downsampling. */
int64_t oracle_forward(const int *n, const double *origin, double pitch, const double *tx, int K, const double *tp,
                       const int *ip, int method, int q1, int q2, const double *taps, int T, int n_lo,
                       const int64_t *vox_idx, int64_t n_vox, const double *x, double *s, double *f_out)
{
    otime tm = mk_time(tp, ip);
    const int64_t UL = (int64_t)tm.U * tm.L;
    double *f = f_out ? f_out : (double *)malloc(sizeof(double) * (size_t)UL * (size_t)K);
    int64_t d = oracle_geometric_forward(n, origin, pitch, tx, K, tp, ip, method, q1, q2, vox_idx, n_vox, x, f);
    oracle_conv_forward(taps, T, n_lo, tm.U, tm.L, K, f, s);
    if (!f_out) free(f);
    return d;
}

/* Whole adjoint, Alg. 5. */
int64_t oracle_adjoint(const int *n, const double *origin, double pitch, const double *tx, int K, const double *tp,
                       const int *ip, int method, int q1, int q2, const double *taps, int T, int n_lo, const double *s,
                       const int64_t *vox_idx, int64_t n_vox, double *z, double *v_out)
{
    otime tm = mk_time(tp, ip);
    const int64_t UL = (int64_t)tm.U * tm.L;
    double *v = v_out ? v_out : (double *)malloc(sizeof(double) * (size_t)UL * (size_t)K);
    oracle_conv_adjoint(taps, T, n_lo, tm.U, tm.L, K, s, v);
    int64_t d = oracle_geometric_adjoint(n, origin, pitch, tx, K, tp, ip, method, q1, q2, v, vox_idx, n_vox, z);
    if (!v_out) free(v);
    return d;
}

/* ------------------------------------------------------------------------ */
/* System kernel (Prop. 1 and Eq. def_bh).                                   */
/*   g(t) = -1/2 c t phi(|c t|),  h = e * g,                                 */
/*   h-bar[n] = U Fs int_0^D int_0^D h(t - t' + n D) dt dt',  D = 1/(U Fs),  */
/* evaluated as (1/D) int_{-D}^{D} (D - |s|) h(n D + s) ds (the measure of   */
/* {(t, t') in [0,D]^2 : t - t' = s} is D - |s|).  Nested composite          */
/* Gauss-Legendre quadrature split at every kink.                            */
/* rbf kinds: 0 bump (1 - r^2/k^2)^2, 1 cone 1 - r/k, 2 Wendland (1 - r/k)^2. */
/* eir kinds: 0 exp(-(t-tc)^2 / (2 s^2)) sin(2 pi fc (t - tc)) on [0, Te],   */
/*            par = {fc, s, tc, Te};  1 box par[0] on [0, Te].               */
/* ------------------------------------------------------------------------ */
#define GLN 20
static double gl_x[GLN], gl_w[GLN];
static int gl_ready = 0;

static void gl_init(void)
{
    if (gl_ready) return;
    /* Newton iteration on the Legendre polynomial P_20 (three-term recurrence) */
    for (int i = 0; i < GLN; ++i) {
        double x = cos(M_PI * (i + 0.75) / (GLN + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= GLN; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = GLN * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

typedef struct {
    int rbf;
    double kappa;
    int eir;
    double ep[4];
    double c;
    int panels;
} okern;

static double rbf_val(int kind, double kappa, double r)
{
    r = fabs(r);
    if (r >= kappa) return 0.0;
    double q = r / kappa;
    if (kind == 0) return (1.0 - q * q) * (1.0 - q * q);
    if (kind == 1) return 1.0 - q;
    return (1.0 - q) * (1.0 - q);
}

static double g_val(const okern *k, double t)
{
    double ct = k->c * t;
    return -0.5 * ct * rbf_val(k->rbf, k->kappa, fabs(ct)); /* Prop. 1 */
}

static double e_val(const okern *k, double t)
{
    if (t < 0.0 || t > k->ep[3]) return 0.0;
    if (k->eir == 0) {
        double d = t - k->ep[2];
        return exp(-d * d / (2.0 * k->ep[1] * k->ep[1])) * sin(2.0 * M_PI * k->ep[0] * d);
    }
    return k->ep[0];
}

static double gl_piece(double a, double b, int panels, double (*fn)(const okern *, double, double),
                       const okern *k, double p)
{
    double acc = 0.0, w = (b - a) / panels;
    for (int q = 0; q < panels; ++q) {
        double mid = a + (q + 0.5) * w;
        for (int i = 0; i < GLN; ++i) acc += gl_w[i] * fn(k, mid + 0.5 * w * gl_x[i], p);
    }
    return acc * 0.5 * w;
}

static double inner_integrand(const okern *k, double tp, double t) { return e_val(k, tp) * g_val(k, t - tp); }

/* h(t) = int e(t') g(t - t') dt' over [max(0, t - kappa/c), min(Te, t + kappa/c)], split at t' = t. */
static double h_val(const okern *k, double t)
{
    double kc = k->kappa / k->c;
    double a = fmax(0.0, t - kc), b = fmin(k->ep[3], t + kc);
    if (!(b > a)) return 0.0;
    if (t > a && t < b) return gl_piece(a, t, k->panels, inner_integrand, k, t) + gl_piece(t, b, k->panels, inner_integrand, k, t);
    return gl_piece(a, b, k->panels, inner_integrand, k, t);
}

static int cmpd(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

void oracle_system_kernel(int rbf_kind, double kappa, int eir_kind, const double *eir_par, double c, double fs, int U,
                          int n_lo, int T, int panels, double *taps)
{
    gl_init();
    okern k;
    k.rbf = rbf_kind;
    k.kappa = kappa;
    k.eir = eir_kind;
    memcpy(k.ep, eir_par, sizeof(k.ep));
    k.c = c;
    k.panels = panels > 0 ? panels : 3;
    const double D = 1.0 / ((double)U * fs), kc = kappa / c, Te = k.ep[3];
    const double kinks[6] = {-kc, 0.0, kc, Te - kc, Te, Te + kc};
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < T; ++t) {
        double nD = (double)(n_lo + t) * D;
        double bp[9];
        int nb = 0;
        bp[nb++] = -D;
        bp[nb++] = 0.0;
        bp[nb++] = D;
        for (int i = 0; i < 6; ++i) {
            double s = kinks[i] - nD;
            if (s > -D && s < D && s != 0.0) bp[nb++] = s;
        }
        qsort(bp, (size_t)nb, sizeof(double), cmpd);
        double acc = 0.0;
        for (int p = 0; p + 1 < nb; ++p) {
            double a = bp[p], b = bp[p + 1];
            if (!(b > a)) continue;
            double w = (b - a) / k.panels;
            for (int q = 0; q < k.panels; ++q) {
                double mid = a + (q + 0.5) * w;
                for (int i = 0; i < GLN; ++i) {
                    double s = mid + 0.5 * w * gl_x[i];
                    acc += 0.5 * w * gl_w[i] * (D - fabs(s)) * h_val(&k, nD + s);
                }
            }
        }
        taps[t] = acc / D;
    }
}

/* Exported continuous kernels for the tests. */
double oracle_h_value(int rbf_kind, double kappa, int eir_kind, const double *eir_par, double c, int panels, double t)
{
    gl_init();
    okern k;
    k.rbf = rbf_kind;
    k.kappa = kappa;
    k.eir = eir_kind;
    memcpy(k.ep, eir_par, sizeof(k.ep));
    k.c = c;
    k.panels = panels > 0 ? panels : 3;
    return h_val(&k, t);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
