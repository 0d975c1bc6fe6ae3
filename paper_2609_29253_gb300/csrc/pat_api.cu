// pat_api.cu -- the C ABI of include/pat.h: plans, validation, workspaces and
// the enqueueing of the kernels of pat_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pat.h"
#include "pat_conv_tc.cuh"
#include "pat_kernels.cuh"

using namespace pat;

struct pat_plan {
    int device;
    int K;
    long long N;
    pat_grid grid;
    pat_params params;
    double kappa;
    GridDev g;
    TimeDev tm;
    TxDev *tx;
    double *taps;
    float *W;
    int T, nW, n_lo;
    int Kf;         // elements after the piecewise-planes expansion (== K without it)
    int *rows;      // per element: its signal row
    int fwd_bpc;    // forward geometric kernel: bricks per CTA (super-tile-major order)
    int fwd_bpc0;   // the chunking the plan-time scan sized fwd_span for (fwd_bpc divides it)
    int adj_wpb;    // warps (voxel bricks) per CTA of the adjoint gather
    int fwd_span;   // forward window length (edges): the largest over its CTAs
    int smem_optin;
    int kind_all;   // PAT_PLANE / PAT_CYLINDER if every element has it, else kKindAny
    double *scal; // device scalars for pat_recon
    // PAT_FLAG_CONV_TC: tensor-core convolution tables and error word
    bool tc;
    TcGeometry tcg;
    uint8_t *tc_fwd_tab, *tc_adj_tab, *tc_fwd2_tab; // FP32-input forward, adjoint, split-plane forward
    int *tc_err;
    // PAT_METHOD_LUT: the tables of E~ and F~ with their node arrays (one allocation)
    void *lut_buf;
    pat_plan_info info;
};

static thread_local std::string g_err;

static pat_status fail(pat_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                                      \
    do {                                                                                                              \
        cudaError_t e_ = (call);                                                                                      \
        if (e_ != cudaSuccess) return fail(PAT_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,  \
                                           __LINE__);                                                                 \
    } while (0)

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

extern "C" const char *pat_last_error(void) { return g_err.c_str(); }

extern "C" int32_t pat_version(void) { return 100; }

// ---------------------------------------------------------------------------
extern "C" pat_status pat_system_kernel(const pat_system *sys, double c, double fs, int32_t U, int32_t n_lo,
                                        int32_t n_taps, double *taps_dev, void *stream)
{
    g_err.clear();
    if (!sys || !taps_dev) return fail(PAT_ERR_INVALID_ARG, "pat_system_kernel: null pointer");
    if (n_taps < 1 || U < 1 || !(c > 0) || !(fs > 0) || !(sys->kappa > 0) || !(sys->eir[3] > 0))
        return fail(PAT_ERR_INVALID_ARG, "pat_system_kernel: sizes and parameters must be positive");
    if (sys->rbf_kind < PAT_RBF_BUMP || sys->rbf_kind > PAT_RBF_WENDLAND)
        return fail(PAT_ERR_INVALID_ARG, "pat_system_kernel: unknown rbf_kind %d", sys->rbf_kind);
    if (sys->eir_kind != PAT_EIR_GAUSS_SINE && sys->eir_kind != PAT_EIR_BOX)
        return fail(PAT_ERR_INVALID_ARG, "pat_system_kernel: unknown eir_kind %d", sys->eir_kind);
    if (sys->eir_kind == PAT_EIR_GAUSS_SINE && !(sys->eir[1] > 0))
        return fail(PAT_ERR_INVALID_ARG, "pat_system_kernel: Gaussian width must be positive");
    CK(launch_taps(sys->rbf_kind, sys->eir_kind, sys->kappa, c, sys->eir, (double)U * fs, n_lo, n_taps, taps_dev,
                   (cudaStream_t)stream));
    return PAT_OK;
}

extern "C" pat_status pat_system_kernel_dc(const pat_system *sys, double c, double fs, int32_t U, int32_t n_lo,
                                           int32_t n_taps, double *dtaps_dev, void *stream)
{
    g_err.clear();
    if (!sys || !dtaps_dev) return fail(PAT_ERR_INVALID_ARG, "pat_system_kernel_dc: null pointer");
    if (n_taps < 1 || U < 1 || !(c > 0) || !(fs > 0) || !(sys->kappa > 0) || !(sys->eir[3] > 0))
        return fail(PAT_ERR_INVALID_ARG, "pat_system_kernel_dc: sizes and parameters must be positive");
    if (sys->rbf_kind < PAT_RBF_BUMP || sys->rbf_kind > PAT_RBF_WENDLAND)
        return fail(PAT_ERR_INVALID_ARG, "pat_system_kernel_dc: unknown rbf_kind %d", sys->rbf_kind);
    if (sys->eir_kind != PAT_EIR_GAUSS_SINE && sys->eir_kind != PAT_EIR_BOX)
        return fail(PAT_ERR_INVALID_ARG, "pat_system_kernel_dc: unknown eir_kind %d", sys->eir_kind);
    if (sys->eir_kind == PAT_EIR_GAUSS_SINE && !(sys->eir[1] > 0))
        return fail(PAT_ERR_INVALID_ARG, "pat_system_kernel_dc: Gaussian width must be positive");
    CK(launch_taps(sys->rbf_kind, sys->eir_kind, sys->kappa, c, sys->eir, (double)U * fs, n_lo, n_taps, dtaps_dev,
                   (cudaStream_t)stream, true));
    return PAT_OK;
}

// ---------------------------------------------------------------------------
static pat_status validate(const pat_grid *grid, const pat_transducer *tx, int K, const pat_params *p, double kappa,
                           const double *taps, int n_taps)
{
    if (!grid || !tx || !p || !taps) return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: null pointer");
    if (K < 1) return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: K must be >= 1");
    for (int d = 0; d < 3; ++d)
        if (grid->n[d] < 1) return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: grid size must be >= 1");
    if (!(grid->pitch > 0)) return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: pitch must be > 0");
    if (!(p->c > 0) || !(p->fs > 0) || !(p->t0 >= 0))
        return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: need c > 0, fs > 0, t0 >= 0");
    if (p->L < 1 || p->U < 1 || p->dl < 1 || p->dl > p->U)
        return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: need L >= 1, U >= 1, 1 <= dl <= U");
    if ((long long)p->L * p->U >= (1LL << 30)) return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: U L too large");
    if (p->method != PAT_METHOD_SURFACE && p->method != PAT_METHOD_POINT && p->method != PAT_METHOD_TRAPEZOID &&
        p->method != PAT_METHOD_LUT)
        return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: unknown method %d", p->method);
    if (p->method == PAT_METHOD_POINT && (p->q1 < 1 || p->q2 < 1))
        return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: point method needs q1, q2 >= 1");
    if (p->method == PAT_METHOD_LUT && (p->q1 < 2 || p->q2 < 2 || p->q1 > 8192 || p->q2 > 8192))
        return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: lookup tables need 2 <= q1, q2 <= 8192 nodes");
    if (!(kappa > 0)) return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: kappa must be > 0");
    if (n_taps < 1) return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: n_taps must be >= 1");
    if (p->flags & ~(PAT_FLAG_ALLOW_CLIP | PAT_FLAG_CONV_TC | PAT_FLAG_PIECEWISE_PLANES))
        return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: unknown flags 0x%x", p->flags);
    if ((p->flags & PAT_FLAG_PIECEWISE_PLANES) && (p->np_planes < 1 || p->np_planes > 4096))
        return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: np_planes must be in [1, 4096]");
    for (int k = 0; k < K; ++k) {
        const pat_transducer &t = tx[k];
        int kind = (int)t.kind;
        if ((double)kind != t.kind || (kind != PAT_PLANE && kind != PAT_CYLINDER))
            return fail(PAT_ERR_INVALID_ARG, "transducer %d: unknown kind %g", k, t.kind);
        double n1 = t.e1[0] * t.e1[0] + t.e1[1] * t.e1[1] + t.e1[2] * t.e1[2];
        double n2 = t.e2[0] * t.e2[0] + t.e2[1] * t.e2[1] + t.e2[2] * t.e2[2];
        double d12 = t.e1[0] * t.e2[0] + t.e1[1] * t.e2[1] + t.e1[2] * t.e2[2];
        if (fabs(n1 - 1) > 1e-9 || fabs(n2 - 1) > 1e-9 || fabs(d12) > 1e-9)
            return fail(PAT_ERR_INVALID_ARG, "transducer %d: e1, e2 not orthonormal", k);
        if (kind == PAT_PLANE && !(t.L1 > 0 && t.L2 > 0))
            return fail(PAT_ERR_INVALID_ARG, "transducer %d: L1, L2 must be > 0", k);
        if (kind == PAT_CYLINDER && !(t.R > 0 && t.Lz > 0 && t.theta_max > 0 && t.theta_max < M_PI / 2))
            return fail(PAT_ERR_INVALID_ARG, "transducer %d: need R > 0, Lz > 0, 0 < theta_max < pi/2", k);
    }
    return PAT_OK;
}

// Piecewise-Planes (Sec. 4.3): the aperture [-theta_max, theta_max] cut into
// np equal sectors, sector j replaced by the plane tangent to the cylinder
// along the generator at its central angle theta_j, half-width R dtheta / 2
// across the generator and half-height Lz along the axis.  Planar elements
// pass through.  rows[j] = the element each plane belongs to.
static void expand_planes(const pat_transducer *tx, int K, int np, std::vector<pat_transducer> &out,
                          std::vector<int> &rows)
{
    for (int k = 0; k < K; ++k) {
        const pat_transducer &t = tx[k];
        if ((int)t.kind != PAT_CYLINDER) {
            out.push_back(t);
            rows.push_back(k);
            continue;
        }
        const double n[3] = {t.e1[1] * t.e2[2] - t.e1[2] * t.e2[1], t.e1[2] * t.e2[0] - t.e1[0] * t.e2[2],
                             t.e1[0] * t.e2[1] - t.e1[1] * t.e2[0]};
        const double dth = 2.0 * t.theta_max / np;
        for (int j = 0; j < np; ++j) {
            const double th = -t.theta_max + (j + 0.5) * dth, c = cos(th), sn = sin(th);
            pat_transducer f;
            memset(&f, 0, sizeof(f));
            f.kind = PAT_PLANE;
            for (int d = 0; d < 3; ++d) {
                const double radial = c * t.e2[d] + sn * n[d];
                f.c0[d] = t.c0[d] + t.R * radial;
                f.e1[d] = -sn * t.e2[d] + c * n[d]; // along the arc
                f.e2[d] = t.e1[d];                  // along the axis
            }
            f.L1 = 0.5 * t.R * dth;
            f.L2 = t.Lz;
            out.push_back(f);
            rows.push_back(k);
        }
    }
}

extern "C" pat_status pat_plan_create(pat_plan **out, const pat_grid *grid, const pat_transducer *tx, int32_t K,
                                      const pat_params *params, double kappa, const double *taps_host,
                                      int32_t n_taps, int32_t n_lo, void *stream)
{
    g_err.clear();
    if (!out) return fail(PAT_ERR_INVALID_ARG, "pat_plan_create: null out");
    *out = nullptr;
    pat_status st = validate(grid, tx, K, params, kappa, taps_host, n_taps);
    if (st != PAT_OK) return st;
    std::vector<pat_transducer> facets;
    std::vector<int> rows_h;
    if (params->flags & PAT_FLAG_PIECEWISE_PLANES) {
        expand_planes(tx, K, params->np_planes, facets, rows_h);
    } else {
        facets.assign(tx, tx + K);
        for (int k = 0; k < K; ++k) rows_h.push_back(k);
    }
    const int Kf = (int)facets.size();
    const pat_transducer *fx = facets.data();
    cudaStream_t s = (cudaStream_t)stream;
    pat_plan *p = new pat_plan();
    memset(p, 0, sizeof(*p));
    CK(cudaGetDevice(&p->device));
    p->K = K;
    p->Kf = Kf;
    p->grid = *grid;
    p->params = *params;
    p->kappa = kappa;
    p->N = (long long)grid->n[0] * grid->n[1] * grid->n[2];
    p->kind_all = (int)fx[0].kind;
    for (int k = 1; k < Kf; ++k)
        if ((int)fx[k].kind != p->kind_all) p->kind_all = kKindAny;
    GridDev &g = p->g;
    g.nx = grid->n[0];
    g.ny = grid->n[1];
    g.nz = grid->n[2];
    g.nbx = (g.nx + kBrickX - 1) / kBrickX;
    g.nby = (g.ny + kBrickY - 1) / kBrickY;
    g.nbz = (g.nz + kBrickZ - 1) / kBrickZ;
    g.nbricks = (long long)g.nbx * g.nby * g.nbz;
    g.nsx = (g.nbx + kSuper - 1) / kSuper;
    g.nsy = (g.nby + kSuper - 1) / kSuper;
    g.nsz = (g.nbz + kSuper - 1) / kSuper;
    g.nvb = (long long)g.nsx * g.nsy * g.nsz * kSuperBricks;
    TimeDev &tm = p->tm;
    tm.c = params->c;
    tm.t0 = params->t0;
    tm.ufs = (double)params->U * params->fs;
    tm.r0d = params->c * params->t0;
    tm.deltad = params->c / tm.ufs;
    tm.deltaf = (float)tm.deltad;
    tm.ufsf = (float)tm.ufs;
    tm.invcf = (float)(1.0 / params->c);
    auto split = [](double v) {
        float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    };
    tm.fr0 = split(tm.r0d);
    tm.fdelta = split(tm.deltad);
    tm.finvdelta = split(tm.ufs / params->c);
    tm.L = params->L;
    tm.U = params->U;
    tm.UL = params->L * params->U;
    tm.dl = params->dl;
    tm.method = params->method;
    tm.q1 = params->method == PAT_METHOD_POINT ? params->q1 : 1;
    tm.q2 = params->method == PAT_METHOD_POINT ? params->q2 : 1;

    int dev = p->device, optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    p->T = n_taps;
    p->n_lo = n_lo;
    p->nW = n_taps + params->U - 1;
    p->smem_optin = optin;
    p->tc = (params->flags & PAT_FLAG_CONV_TC) != 0;
    if (p->tc) {
        p->tcg = tc_geometry(n_taps, params->U, params->L, n_lo);
        // power-of-two scale of the operand tables: the largest tap times
        // 2^tscale in [1, 2) (every combined tap W is a mean of U taps)
        double tmax = 0.0;
        for (int i = 0; i < n_taps; ++i) tmax = std::max(tmax, std::fabs(taps_host[i]));
        if (tmax > 0.0 && std::isfinite(tmax)) p->tcg.tscale = std::min(100, std::max(-100, -std::ilogb(tmax)));
        const size_t need_tc = std::max(std::max(p->tcg.fwd_smem, p->tcg.adj_smem), p->tcg.fwd2_smem);
        if (need_tc > (size_t)optin) {
            delete p;
            return fail(PAT_ERR_UNSUPPORTED, "tensor-core convolution needs %zu bytes of shared memory per block, "
                        "device has %d", need_tc, optin);
        }
    }
    size_t need_epi = sizeof(float) * (size_t)(tm.UL + p->nW) + 64;
    size_t need_adj = sizeof(float) * (size_t)(tm.L + p->nW + tm.UL) + 64;
    if (need_epi > (size_t)optin || need_adj > (size_t)optin) {
        const int ul = tm.UL; // tm lives in *p
        delete p;
        return fail(PAT_ERR_UNSUPPORTED, "U L = %d needs %zu bytes of shared memory per block, device has %d", ul,
                    need_adj, optin);
    }

    // device constants
    double *raw = nullptr, *dorig = nullptr;
    void *lut_scratch = nullptr; // FP64 node values of the lookup tables, freed once the cells are built
    auto cleanup = [&]() {
        cudaFree(raw);
        cudaFree(dorig);
        cudaFree(lut_scratch);
    };
    if (cudaMalloc(&raw, sizeof(double) * 16 * (size_t)Kf) != cudaSuccess ||
        cudaMalloc(&p->tx, sizeof(TxDev) * (size_t)Kf) != cudaSuccess ||
        cudaMalloc(&p->rows, sizeof(int) * (size_t)Kf) != cudaSuccess ||
        cudaMalloc(&p->taps, sizeof(double) * (size_t)n_taps) != cudaSuccess ||
        cudaMalloc(&p->W, sizeof(float) * (size_t)p->nW) != cudaSuccess ||
        cudaMalloc(&p->scal, sizeof(double) * 8) != cudaSuccess) {
        cleanup();
        pat_plan_destroy(p);
        return fail(PAT_ERR_CUDA, "pat_plan_create: cudaMalloc failed");
    }
    static_assert(sizeof(pat_transducer) == 16 * sizeof(double), "descriptor layout");
    pat_status rc = PAT_OK;
    do {
        if (cudaMemcpyAsync(raw, fx, sizeof(double) * 16 * (size_t)Kf, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(p->rows, rows_h.data(), sizeof(int) * (size_t)Kf, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(p->taps, taps_host, sizeof(double) * (size_t)n_taps, cudaMemcpyHostToDevice, s) !=
                cudaSuccess) {
            rc = fail(PAT_ERR_CUDA, "pat_plan_create: copy failed");
            break;
        }
        if (launch_frames(raw, Kf, grid->origin, grid->pitch, tm.q1, tm.q2, p->tx, s) != cudaSuccess ||
            launch_combine_taps(p->taps, n_taps, params->U, p->W, s) != cudaSuccess) {
            rc = fail(PAT_ERR_CUDA, "pat_plan_create: setup kernels failed");
            break;
        }
        if (params->method == PAT_METHOD_LUT) {
            const int ns = params->q1, nm = params->q2;
            if (cudaMalloc(&p->lut_buf, lut_bytes(ns, nm)) != cudaSuccess ||
                cudaMalloc(&lut_scratch, sizeof(double2) * (size_t)ns * nm) != cudaSuccess) {
                rc = fail(PAT_ERR_CUDA, "pat_plan_create: cudaMalloc of the lookup tables failed");
                break;
            }
            if (launch_lut_tables(ns, nm, p->lut_buf, (double2 *)lut_scratch, tm.lut, s) != cudaSuccess) {
                rc = fail(PAT_ERR_CUDA, "pat_plan_create: lookup-table kernels failed");
                break;
            }
        }
        if (p->tc) {
            if (cudaMalloc(&p->tc_fwd_tab, p->tcg.fwd_table_bytes) != cudaSuccess ||
                cudaMalloc(&p->tc_adj_tab, p->tcg.adj_table_bytes) != cudaSuccess ||
                cudaMalloc(&p->tc_fwd2_tab, p->tcg.fwd2_table_bytes) != cudaSuccess ||
                cudaMalloc(&p->tc_err, sizeof(int)) != cudaSuccess) {
                rc = fail(PAT_ERR_CUDA, "pat_plan_create: cudaMalloc failed");
                break;
            }
            if (cudaMemsetAsync(p->tc_err, 0, sizeof(int), s) != cudaSuccess ||
                launch_tc_tables(p->taps, n_taps, params->U, p->tcg, p->tc_fwd_tab, p->tc_adj_tab, p->tc_fwd2_tab, s) !=
                    cudaSuccess) {
                rc = fail(PAT_ERR_CUDA, "pat_plan_create: tensor-core tables failed");
                break;
            }
        }
        // work split of the forward geometric kernel: one super-tile (512
        // bricks) per CTA, halved until there are 32 CTAs per SM (some ten
        // waves, so the last one is a small part of the run); the scan below
        // sizes the window for this chunking, and the autotuner may only
        // split it further
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        {
            long long bpc = kSuperBricks;
            while (bpc > kWarpsPerBlock && (long long)Kf * ((g.nvb + bpc - 1) / bpc) < 32LL * std::max(sms, 1))
                bpc /= 2;
            p->fwd_bpc = p->fwd_bpc0 = (int)bpc;
        }
        // scan every pair once
        void *sbuf = nullptr;
        size_t sb = sizeof(long long) * 6 * (size_t)Kf + 64;
        if (cudaMalloc(&sbuf, sb) != cudaSuccess) {
            rc = fail(PAT_ERR_CUDA, "pat_plan_create: cudaMalloc failed");
            break;
        }
        ScanOut so;
        so.lo = (long long *)sbuf;
        so.hi = so.lo + Kf;
        so.groups = (unsigned long long *)(so.hi + Kf);
        so.bins = so.groups + Kf;
        so.clipped = so.bins + Kf;
        so.quads = so.clipped + Kf;
        so.rmin_bits = so.quads + Kf;
        so.maxspan = so.rmin_bits + 1;
        so.misses = so.rmin_bits + 2;
        std::vector<long long> hb(6 * (size_t)Kf + 3);
        cudaError_t e = launch_scan(p->tx, Kf, tm, g, p->fwd_bpc0, so, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), sbuf, sizeof(long long) * (6 * (size_t)Kf + 3),
                                                  cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(sbuf);
        if (e != cudaSuccess) {
            rc = fail(PAT_ERR_CUDA, "pat_plan_create: scan failed: %s", cudaGetErrorString(e));
            break;
        }
        pat_plan_info &in = p->info;
        in.N = p->N;
        in.K = K;
        in.L = tm.L;
        in.U = tm.U;
        in.UL = tm.UL;
        in.dl = tm.dl;
        in.method = tm.method;
        in.n_taps = n_taps;
        in.n_lo = n_lo;
        in.bin_lo = 0x7fffffffffffffffLL;
        in.bin_hi = -0x7fffffffffffffffLL;
        // the largest forward window over the CTAs (fwd_window), plus two
        // bins in case the forward kernel's FP32 bounds round a tie the other
        // way than the scan's
        const long long span = hb[6 * (size_t)Kf + 1] + 2;
        p->fwd_span = (int)span;
        if (hb[6 * (size_t)Kf + 2] != 0) {
            rc = fail(PAT_ERR_UNSUPPORTED, "pat_plan_create: the FP32 window bound misses the bins of %lld pairs",
                      hb[6 * (size_t)Kf + 2]);
            break;
        }
        if (2 * sizeof(float) * (size_t)span > (size_t)p->smem_optin) {
            rc = fail(PAT_ERR_UNSUPPORTED, "a forward chunk's bins span %lld fine bins: %zu bytes of shared memory, "
                      "device has %d", span, 2 * sizeof(float) * (size_t)span, p->smem_optin);
            break;
        }
        // per element (plane facet); conv_clipped counts elements
        for (int k = 0; k < Kf; ++k) {
            long long lo = hb[k], hi = hb[Kf + k];
            in.bin_lo = std::min<long long>(in.bin_lo, lo);
            in.bin_hi = std::max<long long>(in.bin_hi, hi);
            in.area_evals += hb[2 * (size_t)Kf + k];
            in.pair_bins += hb[3 * (size_t)Kf + k];
            in.clipped_pairs += hb[4 * (size_t)Kf + k];
            in.quad_evals += hb[5 * (size_t)Kf + k];
            if (lo + n_lo < 0 || hi + n_lo + n_taps - 1 >= tm.UL) in.conv_clipped++;
        }
        unsigned long long rb = (unsigned long long)hb[6 * (size_t)Kf];
        memcpy(&in.dist_min, &rb, sizeof(double));
        // adjoint gather: bricks (warps) per CTA; smaller CTAs leave less idle
        // at their end (measured best: 2 for planes, c3; 4 for cylinders, c2)
        p->adj_wpb = p->kind_all == PAT_PLANE ? 2 : 4;
        in.fwd_blocks = (g.nvb + p->fwd_bpc - 1) / p->fwd_bpc * Kf;
        in.adj_blocks = (g.nbricks + p->adj_wpb - 1) / p->adj_wpb;
        if (!(in.dist_min >= kappa)) {
            rc = fail(PAT_ERR_GEOMETRY, "dist_min = %.6g m < kappa = %.6g m (Assumption 1(iii))", in.dist_min, kappa);
            break;
        }
        if (!(tm.deltad <= in.dist_min)) {
            rc = fail(PAT_ERR_GEOMETRY, "c/(U Fs) = %.6g m > dist_min = %.6g m (Prop. 3)", tm.deltad, in.dist_min);
            break;
        }
        if (in.clipped_pairs > 0 && !(params->flags & PAT_FLAG_ALLOW_CLIP)) {
            rc = fail(PAT_ERR_WINDOW, "%lld pairs have bins outside [0, %d): bins [%lld, %lld]", in.clipped_pairs,
                      tm.UL, in.bin_lo, in.bin_hi);
            break;
        }
    } while (0);
    cleanup();
    if (rc != PAT_OK) {
        std::string keep = g_err;
        pat_plan_destroy(p);
        g_err = keep;
        return rc;
    }
    *out = p;
    return PAT_OK;
}

extern "C" pat_status pat_plan_destroy(pat_plan *p)
{
    if (!p) return PAT_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    cudaFree(p->tx);
    cudaFree(p->taps);
    cudaFree(p->W);
    cudaFree(p->rows);
    cudaFree(p->scal);
    cudaFree(p->tc_fwd_tab);
    cudaFree(p->tc_adj_tab);
    cudaFree(p->tc_fwd2_tab);
    cudaFree(p->tc_err);
    cudaFree(p->lut_buf);
    cudaSetDevice(cur);
    delete p;
    return PAT_OK;
}

extern "C" pat_status pat_plan_get_info(const pat_plan *p, pat_plan_info *info)
{
    if (!p || !info) return fail(PAT_ERR_INVALID_ARG, "pat_plan_get_info: null pointer");
    *info = p->info;
    info->tc_error = 0;
    if (p->tc) {
        int e = 0, cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(p->device);
        cudaError_t ce = cudaMemcpy(&e, p->tc_err, sizeof(int), cudaMemcpyDeviceToHost);
        cudaSetDevice(cur);
        if (ce != cudaSuccess) return fail(PAT_ERR_CUDA, "pat_plan_get_info: %s", cudaGetErrorString(ce));
        info->tc_error = e;
    }
    return PAT_OK;
}

// forward: difference array D [K][UL + 1] doubles, then (tensor-core
// convolution) f as BF16 hi and lo planes [K][ld] each, ld = UL rounded up
// to a multiple of 8; adjoint: prefix sums P [K][UL + 1] float2, then
// (tensor-core convolution) v [K][UL] floats in the same place
static size_t ws_D(const pat_plan *p) { return align256(sizeof(double) * (size_t)(p->tm.UL + 1) * p->K); }
static size_t ws_P(const pat_plan *p) { return align256(sizeof(float2) * (size_t)(p->tm.UL + 1) * p->K); }
static size_t ws_planes(const pat_plan *p) { return align256(2 * sizeof(uint16_t) * (size_t)p->tcg.ld * p->K); }
static size_t ws_f(const pat_plan *p) { return p->tc ? ws_planes(p) : 0; }
static size_t ws_fwd(const pat_plan *p) { return ws_D(p) + ws_f(p); }
static size_t ws_adj(const pat_plan *p) { return ws_P(p) + ws_f(p); }
static size_t ws_fwd_dc(const pat_plan *p) { return 2 * ws_D(p); }
// autotuning: operator workspace, then z [N]
static size_t ws_tune(const pat_plan *p) { return std::max(ws_fwd(p), ws_adj(p)) + align256(sizeof(float) * p->N); }
static size_t ws_recon(const pat_plan *p)
{
    return std::max(ws_fwd(p), ws_adj(p)) + align256(sizeof(float) * (size_t)p->K * p->tm.L) +
           4 * align256(sizeof(float) * (size_t)p->N);
}

extern "C" size_t pat_workspace_bytes(const pat_plan *p, int32_t op)
{
    if (!p) return 0;
    if (op == PAT_OP_FORWARD) return ws_fwd(p);
    if (op == PAT_OP_ADJOINT) return ws_adj(p);
    if (op == PAT_OP_RECON) return ws_recon(p);
    if (op == PAT_OP_FORWARD_DC) return ws_fwd_dc(p);
    if (op == PAT_OP_AUTOTUNE) return ws_tune(p);
    if (op == PAT_OP_CONV_SPLIT) return p->tc ? ws_planes(p) : 0;
    return 0;
}

static pat_status check_ws(const pat_plan *p, void *ws, size_t bytes, size_t need, const char *who)
{
    if (!ws || bytes < need)
        return fail(PAT_ERR_WORKSPACE, "%s: workspace %zu bytes at %p, need %zu", who, bytes, ws, need);
    if (((uintptr_t)ws & 255) != 0) return fail(PAT_ERR_WORKSPACE, "%s: workspace must be 256-byte aligned", who);
    (void)p;
    return PAT_OK;
}

// s = A x (s may be null: geometric stage only, into f).  With the
// tensor-core convolution the epilogue writes f into the workspace and the
// tcgen05 kernel filters and downsamples it.
static pat_status enqueue_forward(pat_plan *p, const float *x, float *s, float *f, void *ws, cudaStream_t st)
{
    double *D = (double *)ws;
    CK(launch_fwd_geom(p->tx, p->Kf, p->K, p->rows, p->kind_all, p->tm, p->g, x, D, p->fwd_bpc, p->fwd_span,
                       st));
    int mode = p->tm.method == PAT_METHOD_POINT ? 1 : 0;
    if (p->tc && s) {
        // f leaves the epilogue as BF16 hi and lo planes, which the tensor-core
        // kernel's copy engine brings straight into the operand layout
        uint16_t *hi = (uint16_t *)((char *)ws + ws_D(p)), *lo = hi + (size_t)p->tcg.ld * p->K;
        CK(launch_fwd_epilogue(D, p->tm.UL + 1, p->W, p->nW, p->n_lo, p->tm, mode, p->K, nullptr, nullptr, st, hi, lo,
                               p->tcg.ld));
        CK(launch_conv_tc_fwd2(hi, lo, p->tc_fwd2_tab, p->tcg, p->K, p->tm.L, p->tm.U, s, p->tc_err, st));
        return PAT_OK;
    }
    CK(launch_fwd_epilogue(D, p->tm.UL + 1, p->W, p->nW, p->n_lo, p->tm, mode, p->K, s, f, st));
    return PAT_OK;
}

// z = A^T s (from_v = 0) or the geometric transpose of v (from_v = 1).
static pat_status enqueue_adjoint(pat_plan *p, const float *in, int from_v, float *z, void *ws, cudaStream_t st)
{
    int mode = p->tm.method == PAT_METHOD_POINT ? 1 : 0;
    double vscale = 1.0;
    if (p->tc && !from_v) {
        // v stays scaled by the tables' 2^tscale (of the signal's size, far
        // from FP32's smallest normal) and is unscaled in FP64 as it is read
        float *vw = (float *)((char *)ws + ws_P(p));
        CK(launch_conv_tc_adj(in, p->tc_adj_tab, p->tcg, p->K, p->tm.L, p->tm.U, vw, p->tc_err, st, false));
        in = vw;
        from_v = 1;
        vscale = ldexp(1.0, -p->tcg.tscale);
    }
    CK(launch_adj_conv(in, from_v, p->W, p->nW, p->n_lo, p->tm, mode, p->K, ws, st, vscale));
    CK(launch_adj_geom(p->tx, p->Kf, p->rows, p->kind_all, p->tm, p->g, ws, z, st, p->adj_wpb));
    return PAT_OK;
}

extern "C" pat_status pat_forward(pat_plan *p, const float *x, float *s, void *ws, size_t ws_bytes, void *stream)
{
    g_err.clear();
    if (!p || !x || !s) return fail(PAT_ERR_INVALID_ARG, "pat_forward: null pointer");
    pat_status st = check_ws(p, ws, ws_bytes, ws_fwd(p), "pat_forward");
    if (st != PAT_OK) return st;
    return enqueue_forward(p, x, s, nullptr, ws, (cudaStream_t)stream);
}

extern "C" pat_status pat_forward_geometric(pat_plan *p, const float *x, float *f, void *ws, size_t ws_bytes,
                                            void *stream)
{
    g_err.clear();
    if (!p || !x || !f) return fail(PAT_ERR_INVALID_ARG, "pat_forward_geometric: null pointer");
    pat_status st = check_ws(p, ws, ws_bytes, ws_fwd(p), "pat_forward_geometric");
    if (st != PAT_OK) return st;
    return enqueue_forward(p, x, nullptr, f, ws, (cudaStream_t)stream);
}

extern "C" pat_status pat_conv_forward(pat_plan *p, const float *f, float *s, void *stream)
{
    g_err.clear();
    if (!p || !f || !s) return fail(PAT_ERR_INVALID_ARG, "pat_conv_forward: null pointer");
    if (p->tc) {
        CK(launch_conv_tc_fwd(f, p->tc_fwd_tab, p->tcg, p->K, p->tm.L, p->tm.U, s, p->tc_err, (cudaStream_t)stream));
        return PAT_OK;
    }
    CK(launch_fwd_epilogue(f, p->tm.UL, p->W, p->nW, p->n_lo, p->tm, 2, p->K, s, nullptr, (cudaStream_t)stream));
    return PAT_OK;
}

extern "C" pat_status pat_conv_split(pat_plan *p, const float *f, uint16_t *planes, void *stream)
{
    g_err.clear();
    if (!p || !f || !planes) return fail(PAT_ERR_INVALID_ARG, "pat_conv_split: null pointer");
    if (!p->tc) return fail(PAT_ERR_UNSUPPORTED, "pat_conv_split: the plan has no tensor-core convolution");
    if (((uintptr_t)planes & 15) != 0) return fail(PAT_ERR_INVALID_ARG, "pat_conv_split: planes must be 16-byte aligned");
    CK(launch_split_bf16(f, p->K, p->tm.UL, p->tcg.ld, planes, planes + (size_t)p->tcg.ld * p->K,
                         (cudaStream_t)stream));
    return PAT_OK;
}

extern "C" pat_status pat_conv_forward_split(pat_plan *p, const uint16_t *planes, float *s, void *stream)
{
    g_err.clear();
    if (!p || !planes || !s) return fail(PAT_ERR_INVALID_ARG, "pat_conv_forward_split: null pointer");
    if (!p->tc) return fail(PAT_ERR_UNSUPPORTED, "pat_conv_forward_split: the plan has no tensor-core convolution");
    if (((uintptr_t)planes & 15) != 0)
        return fail(PAT_ERR_INVALID_ARG, "pat_conv_forward_split: planes must be 16-byte aligned");
    CK(launch_conv_tc_fwd2(planes, planes + (size_t)p->tcg.ld * p->K, p->tc_fwd2_tab, p->tcg, p->K, p->tm.L, p->tm.U, s,
                           p->tc_err, (cudaStream_t)stream));
    return PAT_OK;
}

extern "C" pat_status pat_conv_forward_split_withheld(pat_plan *p, const uint16_t *planes, float *s, void *stream)
{
    g_err.clear();
    if (!p || !planes || !s) return fail(PAT_ERR_INVALID_ARG, "pat_conv_forward_split_withheld: null pointer");
    if (!p->tc) return fail(PAT_ERR_UNSUPPORTED, "pat_conv_forward_split_withheld: the plan has no tensor-core convolution");
    if (((uintptr_t)planes & 15) != 0)
        return fail(PAT_ERR_INVALID_ARG, "pat_conv_forward_split_withheld: planes must be 16-byte aligned");
    const int ntiles = ((p->tm.L + kTcM - 1) / kTcM) * ((p->K + kTcN2 - 1) / kTcN2);
    if (ntiles < 3)
        return fail(PAT_ERR_INVALID_ARG, "pat_conv_forward_split_withheld: needs at least 3 output tiles, the plan has %d",
                    ntiles);
    CK(launch_conv_tc_fwd2(planes, planes + (size_t)p->tcg.ld * p->K, p->tc_fwd2_tab, p->tcg, p->K, p->tm.L, p->tm.U, s,
                           p->tc_err, (cudaStream_t)stream, true));
    return PAT_OK;
}

extern "C" pat_status pat_plan_clear_tc_error(pat_plan *p, void *stream)
{
    g_err.clear();
    if (!p) return fail(PAT_ERR_INVALID_ARG, "pat_plan_clear_tc_error: null pointer");
    if (p->tc) CK(cudaMemsetAsync(p->tc_err, 0, sizeof(int), (cudaStream_t)stream));
    return PAT_OK;
}

extern "C" pat_status pat_conv_adjoint(pat_plan *p, const float *s, float *v, void *stream)
{
    g_err.clear();
    if (!p || !s || !v) return fail(PAT_ERR_INVALID_ARG, "pat_conv_adjoint: null pointer");
    if (p->tc) {
        CK(launch_conv_tc_adj(s, p->tc_adj_tab, p->tcg, p->K, p->tm.L, p->tm.U, v, p->tc_err, (cudaStream_t)stream));
        return PAT_OK;
    }
    CK(launch_adj_conv(s, 0, p->W, p->nW, p->n_lo, p->tm, 2, p->K, v, (cudaStream_t)stream));
    return PAT_OK;
}

extern "C" pat_status pat_adjoint(pat_plan *p, const float *s, float *z, void *ws, size_t ws_bytes, void *stream)
{
    g_err.clear();
    if (!p || !s || !z) return fail(PAT_ERR_INVALID_ARG, "pat_adjoint: null pointer");
    pat_status st = check_ws(p, ws, ws_bytes, ws_adj(p), "pat_adjoint");
    if (st != PAT_OK) return st;
    return enqueue_adjoint(p, s, 0, z, ws, (cudaStream_t)stream);
}

extern "C" pat_status pat_adjoint_geometric(pat_plan *p, const float *v, float *z, void *ws, size_t ws_bytes,
                                            void *stream)
{
    g_err.clear();
    if (!p || !v || !z) return fail(PAT_ERR_INVALID_ARG, "pat_adjoint_geometric: null pointer");
    pat_status st = check_ws(p, ws, ws_bytes, ws_adj(p), "pat_adjoint_geometric");
    if (st != PAT_OK) return st;
    return enqueue_adjoint(p, v, 1, z, ws, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// speed-of-sound derivative of s = A x
// ---------------------------------------------------------------------------
extern "C" pat_status pat_forward_dc(pat_plan *p, const float *x, const double *dtaps, float *ds, void *ws,
                                     size_t ws_bytes, void *stream)
{
    g_err.clear();
    if (!p || !x || !dtaps || !ds) return fail(PAT_ERR_INVALID_ARG, "pat_forward_dc: null pointer");
    if (p->tm.method != PAT_METHOD_SURFACE)
        return fail(PAT_ERR_UNSUPPORTED, "pat_forward_dc: only the surface method (closed-form areas)");
    const size_t need4 = 4 * sizeof(float) * (size_t)p->fwd_span;
    const size_t need_epi = sizeof(float) * (size_t)(2 * p->tm.UL + 2 * p->nW);
    if (need4 > (size_t)p->smem_optin || need_epi > (size_t)p->smem_optin)
        return fail(PAT_ERR_UNSUPPORTED, "pat_forward_dc: needs %zu bytes of shared memory per block, device has %d",
                    std::max(need4, need_epi), p->smem_optin);
    pat_status st = check_ws(p, ws, ws_bytes, ws_fwd_dc(p), "pat_forward_dc");
    if (st != PAT_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    double *Dg = (double *)ws, *Dd = (double *)((char *)ws + ws_D(p));
    CK(launch_fwd_geom_dc(p->tx, p->Kf, p->K, p->rows, p->kind_all, p->tm, p->g, x, Dg, Dd, p->fwd_bpc, p->fwd_span,
                          cs));
    CK(launch_fwd_dc_epilogue(Dg, Dd, p->W, dtaps, p->T, p->nW, p->n_lo, p->tm, p->K, ds, cs));
    return PAT_OK;
}

// ---------------------------------------------------------------------------
// projected FISTA (Eq. nnls_tik)
// ---------------------------------------------------------------------------
// Workspace of one problem: operator workspace, residual r [K][L], then y,
// x_old, g, v [N] (v: power iteration).
struct ReconBufs {
    void *opws;
    float *r, *y, *xo, *g, *v;
};

static ReconBufs recon_bufs(const pat_plan *p, void *ws)
{
    char *w = (char *)ws;
    ReconBufs b;
    b.opws = w;
    w += std::max(ws_fwd(p), ws_adj(p));
    b.r = (float *)w;
    w += align256(sizeof(float) * (size_t)p->K * p->tm.L);
    b.y = (float *)w;
    w += align256(sizeof(float) * (size_t)p->N);
    b.xo = (float *)w;
    w += align256(sizeof(float) * (size_t)p->N);
    b.g = (float *)w;
    w += align256(sizeof(float) * (size_t)p->N);
    b.v = (float *)w;
    return b;
}

// 1 / (1.05 (|A^T A| + lambda)) by 20 power iterations (synchronises cs)
static pat_status recon_step(pat_plan *p, const ReconBufs &b, const float *x, float lambda_R, float *step,
                             cudaStream_t cs)
{
    const long long N = p->N;
    CK(cudaMemcpyAsync(b.v, x, sizeof(float) * N, cudaMemcpyDeviceToDevice, cs));
    CK(launch_dot(b.v, b.v, N, p->scal, cs));
    double nv = 0;
    CK(cudaMemcpyAsync(&nv, p->scal, sizeof(double), cudaMemcpyDeviceToHost, cs));
    CK(cudaStreamSynchronize(cs));
    if (!(nv > 0)) {
        std::vector<float> ones((size_t)N, 1.f);
        CK(cudaMemcpyAsync(b.v, ones.data(), sizeof(float) * N, cudaMemcpyHostToDevice, cs));
        CK(cudaStreamSynchronize(cs));
    }
    CK(launch_dot(b.v, b.v, N, p->scal, cs));
    CK(launch_scale(b.v, b.v, N, p->scal, cs));
    double lam_max = 0;
    for (int it = 0; it < 20; ++it) {
        pat_status e = enqueue_forward(p, b.v, b.r, nullptr, b.opws, cs);
        if (e != PAT_OK) return e;
        e = enqueue_adjoint(p, b.r, 0, b.g, b.opws, cs);
        if (e != PAT_OK) return e;
        CK(launch_dot(b.g, b.v, N, p->scal, cs)); // Rayleigh quotient, |v| = 1
        CK(launch_dot(b.g, b.g, N, p->scal + 1, cs));
        double h[2];
        CK(cudaMemcpyAsync(h, p->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, cs));
        CK(cudaStreamSynchronize(cs));
        lam_max = h[0];
        if (!(h[1] > 0)) break;
        CK(launch_scale(b.g, b.v, N, p->scal + 1, cs));
    }
    const double Lc = lam_max + lambda_R;
    if (!(Lc > 0)) return fail(PAT_ERR_INVALID_ARG, "pat_recon: operator norm estimate is zero");
    *step = (float)(1.0 / (1.05 * Lc));
    return PAT_OK;
}

// y = x_old = x0, t = 1 (device scalars scal[4], scal[5])
static pat_status recon_init(pat_plan *p, const ReconBufs &b, const float *x, cudaStream_t cs)
{
    static const double t0[2] = {1.0, 0.0};
    CK(cudaMemcpyAsync(b.y, x, sizeof(float) * p->N, cudaMemcpyDeviceToDevice, cs));
    CK(cudaMemcpyAsync(b.xo, x, sizeof(float) * p->N, cudaMemcpyDeviceToDevice, cs));
    CK(cudaMemcpyAsync(p->scal + 4, t0, sizeof(t0), cudaMemcpyHostToDevice, cs));
    return PAT_OK;
}

// One FISTA iteration: r = A y - s, g = A^T r, momentum, projected update.
// The same launches every time (all scalars on the device).
static pat_status recon_iteration(pat_plan *p, const ReconBufs &b, const float *s, float step, float lambda_R,
                                  cudaStream_t cs)
{
    pat_status e = enqueue_forward(p, b.y, b.r, nullptr, b.opws, cs);
    if (e != PAT_OK) return e;
    CK(launch_sub(b.r, s, b.r, (long long)p->K * p->tm.L, cs));
    e = enqueue_adjoint(p, b.r, 0, b.g, b.opws, cs);
    if (e != PAT_OK) return e;
    CK(launch_fista(b.y, b.g, b.xo, p->N, step, lambda_R, p->scal + 4, cs));
    return PAT_OK;
}

// Can work on cs be captured into a graph here?  Not on the legacy stream and
// not while the caller is capturing cs already (the iterations then go into
// the caller's graph as plain launches).
static bool capturable(cudaStream_t cs)
{
    if (cs == nullptr || cs == cudaStreamLegacy || cs == cudaStreamPerThread) return false;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(cs, &st) != cudaSuccess) return false;
    return st == cudaStreamCaptureStatusNone;
}

// Captures build(cs) once into a graph and launches it n times on cs.
template <class Build> static pat_status replay(cudaStream_t cs, int n, Build build)
{
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    pat_status e = build(cs);
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (e != PAT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return e;
    }
    CK(ce);
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ce);
    for (int i = 0; i < n && ce == cudaSuccess; ++i) ce = cudaGraphLaunch(exec, cs);
    cudaGraphExecDestroy(exec); // freed once the launches in flight complete
    CK(ce);
    return PAT_OK;
}

extern "C" pat_status pat_recon(pat_plan *p, const float *s, float *x, int32_t iters, float lambda_R, float step,
                                void *ws, size_t ws_bytes, void *stream)
{
    g_err.clear();
    if (!p || !s || !x) return fail(PAT_ERR_INVALID_ARG, "pat_recon: null pointer");
    if (iters < 0 || !(lambda_R >= 0)) return fail(PAT_ERR_INVALID_ARG, "pat_recon: need iters >= 0, lambda_R >= 0");
    pat_status st = check_ws(p, ws, ws_bytes, ws_recon(p), "pat_recon");
    if (st != PAT_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    const ReconBufs b = recon_bufs(p, ws);
    if (!(step > 0)) {
        st = recon_step(p, b, x, lambda_R, &step, cs);
        if (st != PAT_OK) return st;
    }
    st = recon_init(p, b, x, cs);
    if (st != PAT_OK) return st;
    if (iters >= 2 && capturable(cs)) {
        st = replay(cs, iters, [&](cudaStream_t c) { return recon_iteration(p, b, s, step, lambda_R, c); });
    } else {
        for (int it = 0; it < iters && st == PAT_OK; ++it) st = recon_iteration(p, b, s, step, lambda_R, cs);
    }
    if (st != PAT_OK) return st;
    CK(cudaMemcpyAsync(x, b.xo, sizeof(float) * p->N, cudaMemcpyDeviceToDevice, cs));
    return PAT_OK;
}

extern "C" pat_status pat_recon_batch(pat_plan *const *plans, int32_t nprob, const float *const *s, float *const *x,
                                      int32_t iters, const float *lambda_R, const float *step, void *const *ws,
                                      const size_t *ws_bytes, void *stream)
{
    g_err.clear();
    if (!plans || !s || !x || !lambda_R || !ws || !ws_bytes || nprob < 1 || iters < 0)
        return fail(PAT_ERR_INVALID_ARG, "pat_recon_batch: null pointer, nprob < 1 or iters < 0");
    for (int i = 0; i < nprob; ++i) {
        if (!plans[i] || !s[i] || !x[i]) return fail(PAT_ERR_INVALID_ARG, "pat_recon_batch: problem %d: null pointer", i);
        if (!(lambda_R[i] >= 0)) return fail(PAT_ERR_INVALID_ARG, "pat_recon_batch: problem %d: lambda_R < 0", i);
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return fail(PAT_ERR_INVALID_ARG, "pat_recon_batch: plan of problem %d repeats", i);
        pat_status st = check_ws(plans[i], ws[i], ws_bytes[i], ws_recon(plans[i]), "pat_recon_batch");
        if (st != PAT_OK) return st;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    std::vector<ReconBufs> b((size_t)nprob);
    std::vector<float> stp((size_t)nprob);
    for (int i = 0; i < nprob; ++i) {
        b[i] = recon_bufs(plans[i], ws[i]);
        stp[i] = step ? step[i] : 0.f;
        if (!(stp[i] > 0)) {
            pat_status st = recon_step(plans[i], b[i], x[i], lambda_R[i], &stp[i], cs);
            if (st != PAT_OK) return st;
        }
        pat_status st = recon_init(plans[i], b[i], x[i], cs);
        if (st != PAT_OK) return st;
    }
    pat_status st = PAT_OK;
    if (iters >= 1 && nprob > 1 && capturable(cs)) {
        // one graph per iteration of all problems: a fork to one stream per
        // problem and a join, so independent problems overlap on the GPU
        std::vector<cudaStream_t> sub((size_t)nprob, nullptr);
        std::vector<cudaEvent_t> ev((size_t)nprob + 1, nullptr);
        cudaError_t ce = cudaSuccess;
        for (int i = 0; i < nprob && ce == cudaSuccess; ++i) ce = cudaStreamCreateWithFlags(&sub[i], cudaStreamNonBlocking);
        for (int i = 0; i <= nprob && ce == cudaSuccess; ++i) ce = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        if (ce == cudaSuccess) {
            st = replay(cs, iters, [&](cudaStream_t c) -> pat_status {
                CK(cudaEventRecord(ev[nprob], c));
                for (int i = 0; i < nprob; ++i) {
                    CK(cudaStreamWaitEvent(sub[i], ev[nprob], 0));
                    pat_status e = recon_iteration(plans[i], b[i], s[i], stp[i], lambda_R[i], sub[i]);
                    if (e != PAT_OK) return e;
                    CK(cudaEventRecord(ev[i], sub[i]));
                    CK(cudaStreamWaitEvent(c, ev[i], 0));
                }
                return PAT_OK;
            });
        } else {
            st = fail(PAT_ERR_CUDA, "pat_recon_batch: stream or event creation failed: %s", cudaGetErrorString(ce));
        }
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
        for (auto q : sub)
            if (q) cudaStreamDestroy(q);
    } else {
        for (int it = 0; it < iters && st == PAT_OK; ++it)
            for (int i = 0; i < nprob && st == PAT_OK; ++i)
                st = recon_iteration(plans[i], b[i], s[i], stp[i], lambda_R[i], cs);
    }
    if (st != PAT_OK) return st;
    for (int i = 0; i < nprob; ++i)
        CK(cudaMemcpyAsync(x[i], b[i].xo, sizeof(float) * plans[i]->N, cudaMemcpyDeviceToDevice, cs));
    return PAT_OK;
}

// ---------------------------------------------------------------------------
// autotuning of the launch shapes
// ---------------------------------------------------------------------------
extern "C" pat_status pat_plan_autotune(pat_plan *p, const float *x, void *ws, size_t ws_bytes, void *stream)
{
    g_err.clear();
    if (!p || !x) return fail(PAT_ERR_INVALID_ARG, "pat_plan_autotune: null pointer");
    pat_status st = check_ws(p, ws, ws_bytes, ws_tune(p), "pat_plan_autotune");
    if (st != PAT_OK) return st;
    if (!capturable((cudaStream_t)stream) && stream != nullptr)
        return fail(PAT_ERR_INVALID_ARG, "pat_plan_autotune: the stream is being captured");
    cudaStream_t cs = (cudaStream_t)stream;
    double *D = (double *)ws;
    float *z = (float *)((char *)ws + std::max(ws_fwd(p), ws_adj(p)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto timed = [&](auto launch) -> float {
        float best = 3.0e38f;
        for (int rep = 0; rep < 3; ++rep) { // the first run warms up
            if (cudaEventRecord(e0, cs) != cudaSuccess || launch() != cudaSuccess ||
                cudaEventRecord(e1, cs) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                return -1.f;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, ms);
        }
        return best;
    };
    // forward: bricks per CTA, the planned chunking and its halves and
    // quarters (each nested in a planned chunk, so within the planned window)
    const int bpc0 = p->fwd_bpc0;
    int best_b = bpc0;
    float best_t = 3.0e38f;
    for (int f : {1, 2, 4}) {
        const int b = bpc0 / f;
        if (b < kWarpsPerBlock) break;
        const float t = timed([&] {
            return launch_fwd_geom(p->tx, p->Kf, p->K, p->rows, p->kind_all, p->tm, p->g, x, D, b, p->fwd_span, cs);
        });
        if (t < 0.f) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return fail(PAT_ERR_CUDA, "pat_plan_autotune: forward launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        }
        if (t < best_t) {
            best_t = t;
            best_b = b;
        }
    }
    // adjoint gather: bricks per CTA (the workspace holds finite values from
    // the forward runs; the timing does not depend on them)
    int best_w = p->adj_wpb;
    float best_a = 3.0e38f;
    CK(cudaMemsetAsync(ws, 0, ws_P(p), cs));
    for (int wpb : {2, 4, 8}) {
        const float t =
            timed([&] { return launch_adj_geom(p->tx, p->Kf, p->rows, p->kind_all, p->tm, p->g, ws, z, cs, wpb); });
        if (t < 0.f) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return fail(PAT_ERR_CUDA, "pat_plan_autotune: adjoint launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        }
        if (t < best_a) {
            best_a = t;
            best_w = wpb;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->fwd_bpc = best_b;
    p->adj_wpb = best_w;
    p->info.fwd_blocks = (p->g.nvb + best_b - 1) / best_b * p->Kf;
    p->info.adj_blocks = (p->g.nbricks + best_w - 1) / best_w;
    return PAT_OK;
}

// ---------------------------------------------------------------------------
// Forward operator with fixed scratch, for callers that cannot allocate.
// ---------------------------------------------------------------------------
// In host code g_static_scratch names a host-side stand-in, not device memory:
// only the address returned by cudaGetSymbolAddress may reach a kernel.
static __device__ __align__(256) unsigned char g_static_scratch[PAT_STATIC_SCRATCH_BYTES];

static std::mutex g_static_mu;
static void *g_static_ptr[256]; // per device, filled on the first call there

extern "C" pat_status pat_forward_static(pat_plan *p, const float *x, float *s, void *stream)
{
    g_err.clear();
    if (!p || !x || !s) return fail(PAT_ERR_INVALID_ARG, "pat_forward_static: null pointer");
    const size_t need = ws_fwd(p);
    if (need > (size_t)PAT_STATIC_SCRATCH_BYTES)
        return fail(PAT_ERR_WORKSPACE,
                    "pat_forward_static: this plan needs %zu bytes of scratch (%s), the fixed array holds %u; "
                    "use pat_forward with a caller workspace",
                    need, p->tc ? "K (U L + 1) 8 + K ld 4 bytes, ld = U L rounded up to a multiple of 8"
                                : "K (U L + 1) 8 bytes",
                    (unsigned)PAT_STATIC_SCRATCH_BYTES);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev != p->device) return fail(PAT_ERR_INVALID_ARG, "pat_forward_static: plan belongs to device %d", p->device);
    if (dev < 0 || dev >= 256) return fail(PAT_ERR_UNSUPPORTED, "pat_forward_static: device index %d", dev);
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[dev]) {
            void *q = nullptr;
            CK(cudaGetSymbolAddress(&q, g_static_scratch));
            g_static_ptr[dev] = q;
        }
        ptr = g_static_ptr[dev];
    }
    return enqueue_forward(p, x, s, nullptr, ptr, (cudaStream_t)stream);
}
