// pat_kernels.cu -- CUDA kernels of the PAT operator for sm_103a.
//
//   frames_kernel        per-element frames (Eq. plane_param, Eq. cylinder_param)
//   scan_kernel          one pass over all pairs at plan time: bin window,
//                        separation (Eq. min_dist), work per application
//   fwd_geom_kernel      geometric assembly of A (Alg. 3 + Alg. 4 / Alg. 2):
//                        CTA = (voxel chunk, transducer), difference-array
//                        histogram of f_k in shared memory
//   fwd_epilogue_kernel  prefix sum, 1/(c tau) weights (Eq. ui_area), then the
//                        convolution with h-bar and the downsampling by U
//                        (Eq. discrete_conv) fused, FP64 accumulation
//   adj_conv_kernel      upsampling transpose + correlation with h-bar^-
//                        (App. G), weights, and prefix sums for the gather
//   adj_geom_kernel      gather of Alg. 7 / Alg. 6: CTA = 8 bricks of
//                        4x4x2 voxels, loop over all transducers, no write
//                        conflicts (App. G)
//   taps_kernel          discrete system kernel h-bar (Eq. def_bh), FP64
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>

#include "pat_geom.cuh"
#include "pat_kernels.cuh"

namespace pat {

// the arc-integral mode of a surface method
__host__ __device__ constexpr int area_mode(int method)
{
    return method == PAT_METHOD_TRAPEZOID ? kAreaTrap : method == PAT_METHOD_LUT ? kAreaLut : kAreaExact;
}

// ---------------------------------------------------------------------------
// frames
// ---------------------------------------------------------------------------
__device__ float2 split_ff(double v)
{
    float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

__global__ void frames_kernel(const double *__restrict__ raw, int K, double ox, double oy, double oz, double pitch,
                              int q1, int q2, TxDev *__restrict__ out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double *r = raw + 16 * (size_t)k;
    const double c0[3] = {r[1], r[2], r[3]}, e1[3] = {r[4], r[5], r[6]}, e2[3] = {r[7], r[8], r[9]};
    const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    TxDev t;
    t.kind = (int)r[0];
    const double *rows[3];
    if (t.kind == PAT_PLANE) { // rows e1, e2, e1 x e2
        rows[0] = e1;
        rows[1] = e2;
        rows[2] = n;
    } else { // rows e2, e1 x e2, e1
        rows[0] = e2;
        rows[1] = n;
        rows[2] = e1;
    }
    const double d[3] = {ox - c0[0], oy - c0[1], oz - c0[2]};
    for (int j = 0; j < 3; ++j) {
        const double *w = rows[j];
        t.a0d[j] = w[0] * d[0] + w[1] * d[1] + w[2] * d[2];
        t.axd[j] = w[0] * pitch;
        t.ayd[j] = w[1] * pitch;
        t.azd[j] = w[2] * pitch;
        t.a0[j] = (float)t.a0d[j];
        t.ax[j] = (float)t.axd[j];
        t.ay[j] = (float)t.ayd[j];
        t.az[j] = (float)t.azd[j];
    }
    t.L1d = r[10];
    t.L2d = r[11];
    t.Rd = r[12];
    t.Lzd = r[14];
    t.cthd = cos(r[13]);
    t.sthd = sin(r[13]);
    t.thmaxd = r[13];
    t.L1 = (float)r[10];
    t.L2 = (float)r[11];
    t.R = (float)r[12];
    t.thmax = (float)r[13];
    t.Lz = (float)r[14];
    for (int j = 0; j < 3; ++j) {
        t.fa0[j] = split_ff(t.a0d[j]);
        t.fax[j] = split_ff(t.axd[j]);
        t.fay[j] = split_ff(t.ayd[j]);
        t.faz[j] = split_ff(t.azd[j]);
    }
    t.fR = split_ff(r[12]);
    t.fRc = split_ff(r[12] * t.cthd);
    t.fRs = split_ff(r[12] * t.sthd);
    t.fL1 = split_ff(r[10]);
    t.fL2 = split_ff(r[11]);
    t.fLz = split_ff(r[14]);
    if (t.kind == PAT_PLANE) t.dq = (float)((2.0 * r[10] / q1) * (2.0 * r[11] / q2));
    else t.dq = (float)(r[12] * (2.0 * r[13] / q1) * (2.0 * r[14] / q2));
    t.pad = 0.f;
    out[k] = t;
}

// ---------------------------------------------------------------------------
// plan-time scan of all pairs
// ---------------------------------------------------------------------------
__global__ void scan_init_kernel(ScanOut s, int K)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) {
        s.lo[k] = 0x7fffffffffffffffLL;
        s.hi[k] = -0x7fffffffffffffffLL;
        s.groups[k] = 0;
        s.bins[k] = 0;
        s.clipped[k] = 0;
        s.quads[k] = 0;
    }
    if (k == 0) {
        s.rmin_bits[0] = 0x7ff0000000000000ULL; // +inf
        s.maxspan[0] = 0;
        s.misses[0] = 0;
    }
}

// CTA = (aligned run of bricks_per_cta bricks of the super-tile-major order,
// transducer),
// the chunking of the forward kernel, so that the largest window any forward
// CTA needs (s.maxspan) is known before the first launch.
__global__ void scan_kernel(const TxDev *__restrict__ tx, TimeDev tm, GridDev g, int bricks_per_cta, ScanOut s)
{
    __shared__ int s_lohi[2];
    const int k = blockIdx.y;
    const TxDev &t = tx[k];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_lohi[0] = 0x7fffffff;
        s_lohi[1] = -0x7fffffff;
    }
    __syncthreads();
    long long lo = 0x7fffffffffffffffLL, hi = -0x7fffffffffffffffLL;
    int wlo = 0x7fffffff, whi = -0x7fffffff; // pair_bins_fast extremes, as fwd_window
    unsigned long long groups = 0, bins = 0, clipped = 0, quads = 0, misses = 0;
    double rmin = INFINITY;
    const long long b0 = (long long)blockIdx.x * bricks_per_cta, b1 = b0 + bricks_per_cta;
    const SuperTile stl = super_tile(g, b0);
    for (long long br = b0 + warp; br < b1; br += kWarpsPerBlock) {
        int ix, iy, iz;
        if (!tile_voxel(g, stl, br, lane, ix, iy, iz)) continue;
        int fb0, fb1;
        pair_bins_fast(t, tm, ix, iy, iz, fb0, fb1);
        wlo = min(wlo, fb0);
        whi = max(whi, fb1);
        PairRange pr;
        pair_range(t, tm, ix, iy, iz, pr);
        if (pr.bmax < pr.bmin) continue;
        // the window bound pass 1 of the forward kernel takes must hold every edge
        if (pr.bmin - 1 < fb0 - kWinBelow || pr.bmax + 2 > fb1 + kWinAbove) misses++;
        lo = min(lo, (long long)pr.bmin);
        hi = max(hi, (long long)pr.bmax);
        unsigned long long nb = (unsigned long long)(pr.bmax - pr.bmin + 1);
        bins += nb;
        unsigned long long ng = (tm.method == PAT_METHOD_POINT) ? (unsigned long long)tm.q1 * tm.q2 : (nb + tm.dl - 1) / tm.dl;
        groups += ng;
        if (tm.method != PAT_METHOD_POINT)
            quads += ng * (unsigned long long)count_quadrants(t, pr.a1, pr.a2, pr.a3);
        if (pr.bmin < 0 || pr.bmax >= tm.UL) clipped++;
        rmin = fmin(rmin, (double)pr.rmin);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        groups += __shfl_xor_sync(0xffffffffu, groups, o);
        bins += __shfl_xor_sync(0xffffffffu, bins, o);
        clipped += __shfl_xor_sync(0xffffffffu, clipped, o);
        quads += __shfl_xor_sync(0xffffffffu, quads, o);
        misses += __shfl_xor_sync(0xffffffffu, misses, o);
        rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    }
    wlo = __reduce_min_sync(0xffffffffu, wlo);
    whi = __reduce_max_sync(0xffffffffu, whi);
    if (lane == 0) {
        atomicMin((long long *)&s.lo[k], lo);
        atomicMax((long long *)&s.hi[k], hi);
        atomicAdd(&s.groups[k], groups);
        atomicAdd(&s.bins[k], bins);
        atomicAdd(&s.clipped[k], clipped);
        atomicAdd(&s.quads[k], quads);
        if (rmin < INFINITY) atomicMin(&s.rmin_bits[0], (unsigned long long)__double_as_longlong(rmin));
        if (misses) atomicAdd(s.misses, misses);
        atomicMin(&s_lohi[0], wlo);
        atomicMax(&s_lohi[1], whi);
    }
    __syncthreads();
    // this CTA's forward window, as fwd_window computes it
    if (threadIdx.x == 0 && s_lohi[0] <= s_lohi[1] + 2) {
        const int base = max(s_lohi[0] - kWinBelow, 0), top = min(s_lohi[1] + kWinAbove, tm.UL);
        if (top >= base) atomicMax((unsigned long long *)s.maxspan, (unsigned long long)(top - base + 1));
    }
}

// ---------------------------------------------------------------------------
// forward geometric assembly
// ---------------------------------------------------------------------------
// The forward window of fwd_geom_kernel is an FP64 array in shared memory
// (span doubles): every group adds the exact difference of two consecutive
// FP32 shares with one FP64 atomic, so the long prefix sum of the epilogue
// does not pile up FP32 rounding.  The derivative kernel keeps two windows
// and accumulates each as an FP32 pair, below.
//
// Compensated accumulation in shared memory: hi[i] takes the FP32 atomic sum,
// lo[i] the exact rounding error of every addition (recomputed from the value
// the atomic returns: FP32 atomic addition rounds to nearest even), plus any
// low part of the addend.  hi + lo then holds the sum to about 2^-44 relative
// to the partial sums, so the long prefix sum over the difference array does
// not pile up FP32 rounding.
__device__ __forceinline__ void acc2(float *hi, float *lo, int i, float v, float vlo)
{
    const float old = atomicAdd(&hi[i], v);
    const float s = old + v;
    const float bb = s - old;
    const float err = (old - (s - bb)) + (v - bb);
    const float l = err + vlo;
    if (l != 0.f) atomicAdd(&lo[i], l);
}

// Fine-bin window of one transducer in shared memory: edges base..top.
struct BinWindow {
    float *hi, *lo;
    int base, top;
    __device__ __forceinline__ int idx(int e) const { return min(max(e, base), top) - base; }
};

struct FwdSurfaceSink {
    BinWindow w;
    float x, prev;
    __device__ __forceinline__ void start(int) {}
    __device__ __forceinline__ void pre(int, int) {}
    __device__ __forceinline__ void group(int e0, int, float val, float)
    {
        const float v = x * val;
        if (v != prev) atomicAdd((double *)w.hi + w.idx(e0), (double)v - (double)prev);
        prev = v;
    }
    __device__ __forceinline__ void finish(int end)
    {
        if (prev != 0.f) atomicAdd((double *)w.hi + w.idx(end), -(double)prev);
    }
};

// The cylinder forward's window in fixed point: each per-bin share x val,
// scaled by the CTA's power of two, is rounded once to an int64, and the
// group adds the exact integer difference to the one before with an int64
// shared atomic (native, where the FP64 shared addition above is a
// compare-and-swap loop on the FP64 pipe).  x arrives multiplied by the CTA's
// two powers of two (its normalization and the share scale), so a share costs
// one multiply.  The telescoping sums stay exact; the quantum is 2^-46 of a
// bound of the CTA's shares.  Measured: the c2
// forward 4.5 % faster, c5's first positions and Exp-1's trapezoidal rule 2 %
// slower; on planes, whose group loop is short, the conversion costs more than
// the loop it removes (c3 5 % slower), so planar kernels keep the FP64 window.
struct FwdFixedSink {
    BinWindow w;
    float xs; // x times both powers of two (exact)
    long long prev;
    __device__ __forceinline__ void start(int) {}
    __device__ __forceinline__ void pre(int, int) {}
    __device__ __forceinline__ void group(int e0, int, float val, float)
    {
        const long long v = __float2ll_rn(xs * val);
        if (v != prev) atomicAdd((unsigned long long *)w.hi + w.idx(e0), (unsigned long long)(v - prev));
        prev = v;
    }
    __device__ __forceinline__ void finish(int end)
    {
        if (prev != 0) atomicAdd((unsigned long long *)w.hi + w.idx(end), (unsigned long long)(-prev));
    }
};

// Forward sink of the speed-of-sound derivative: the per-bin shares and their
// c-derivatives, each into its own compensated difference array.
struct FwdDerivSink {
    BinWindow w, wd;
    float x, prev, dprev;
    __device__ __forceinline__ void start(int) {}
    __device__ __forceinline__ void pre(int, int) {}
    __device__ __forceinline__ void group(int e0, int, float val, float dval)
    {
        const float v = x * val, dv = x * dval;
        const float2 a = ff_two_sum(v, -prev), b = ff_two_sum(dv, -dprev);
        if (a.x != 0.f) acc2(w.hi, w.lo, w.idx(e0), a.x, a.y);
        if (b.x != 0.f) acc2(wd.hi, wd.lo, wd.idx(e0), b.x, b.y);
        prev = v;
        dprev = dv;
    }
    __device__ __forceinline__ void finish(int end)
    {
        if (prev != 0.f) acc2(w.hi, w.lo, w.idx(end), -prev, 0.f);
        if (dprev != 0.f) acc2(wd.hi, wd.lo, wd.idx(end), -dprev, 0.f);
    }
};

// Consecutive points of a pair that fall in the same bin (neighbouring points
// of the element) are summed in a register first: one shared-memory FP64
// atomic per run of equal bins instead of one per point.
struct FwdPointSink {
    BinWindow w;
    int UL;
    float x;
    int cb;    // bin of the current run (-1: none)
    float acc; // its summed weights
    __device__ __forceinline__ void flush()
    {
        if (cb >= w.base && cb <= w.top && cb < UL) atomicAdd((double *)w.hi + (cb - w.base), (double)(x * acc));
    }
    __device__ __forceinline__ void point(int b, float wt)
    {
        if (b != cb) {
            flush();
            cb = b;
            acc = 0.f;
        }
        acc += wt;
    }
};

// The fine-bin window [base, top] of this CTA (bricks [b0, b1) of super-tile
// stl): the bins of its pairs (Eq. rmin_rmax) from pair_bins_fast, widened by
// kWinBelow and kWinAbove, clipped to [0, U L] and to the `span` bins the
// launch provides (the plan-time scan sizes it for this chunking, so the clip
// never bites).  A chunk of bricks close together sees a short range of
// distances, so the window stays small however far the element's bins spread
// over the grid.  False when no pair has a bin in [0, U L].  With x, also the
// largest |x| over the run's voxels into s_lohi[2] (as bits: |x| >= 0 orders
// as its bit pattern; infinite if any value is not finite), read in the same
// pass.
template <int KIND>
__device__ bool fwd_window(const TxDev &t, const TimeDev &tm, const GridDev &g, const SuperTile &stl, long long b0,
                           long long b1, int span, int &base, int &top, int *s_lohi, const float *x = nullptr)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_lohi[0] = 0x7fffffff;
        s_lohi[1] = -0x7fffffff;
        if (x) s_lohi[2] = 0;
    }
    __syncthreads();
    int lo = 0x7fffffff, hi = -0x7fffffff;
    float xm = 0.f;
    for (long long br = b0 + warp; br < b1; br += kWarpsPerBlock) { // warp-uniform trip count
        int ix, iy, iz;
        if (tile_voxel(g, stl, br, lane, ix, iy, iz)) {
            if (x) { // a non-finite value (NaN included) makes the maximum infinite
                const float a = fabsf(x[((long long)iz * g.ny + iy) * g.nx + ix]);
                xm = a <= 3.40282347e38f ? fmaxf(xm, a) : __int_as_float(0x7f800000);
            }
            int b_lo, b_hi;
            pair_bins_fast<KIND>(t, tm, ix, iy, iz, b_lo, b_hi);
            lo = min(lo, b_lo);
            hi = max(hi, b_hi);
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    const unsigned xu = x ? __reduce_max_sync(0xffffffffu, __float_as_uint(xm)) : 0u;
    if (lane == 0) {
        atomicMin(&s_lohi[0], lo);
        atomicMax(&s_lohi[1], hi);
        if (x) atomicMax((unsigned *)&s_lohi[2], xu);
    }
    __syncthreads();
    lo = s_lohi[0];
    hi = s_lohi[1];
    if (lo > hi + 2) return false; // no voxel of the grid in the run
    base = max(lo - kWinBelow, 0);
    top = min(min(hi + kWinAbove, tm.UL), base + span - 1);
    return top >= base;
}

// bricks_per_cta: bricks of the super-tile-major order per CTA (blockIdx.x
// takes the run [blockIdx.x bricks_per_cta, ...), in one super-tile); span:
// bins of the largest window.  Dg: [K][UL + 1] doubles, zeroed by the launcher; each CTA adds its
// window into row k.
// rows[k]: the signal row that element (or plane facet) k adds into; with
// exclusive != 0 every row has one element, and a CTA that covers its whole
// element stores its window instead of adding it.
template <int METHOD, int KIND>
__global__ void __launch_bounds__(kThreads, geom_min_ctas(KIND, true)) fwd_geom_kernel(const TxDev *__restrict__ tx, TimeDev tm, GridDev g,
                                                            const float *__restrict__ x, double *__restrict__ Dg,
                                                            int bricks_per_cta, int span,
                                                            const int *__restrict__ rows, int exclusive)
{
    extern __shared__ float sD[];
    __shared__ float glx[kGLTable], glw[kGLTable];
    __shared__ int s_lohi[3];
    const int k = blockIdx.y;
    const int n = tm.UL + 1;
    gl_fill(glx, glw, threadIdx.x);
    const TxDev &t = tx[k];
    const long long b0 = (long long)blockIdx.x * bricks_per_cta, b1 = b0 + bricks_per_cta;
    const SuperTile stl = super_tile(g, b0);
    BinWindow win; // the window at sD: FP64 (FwdSurfaceSink, FwdPointSink) or int64 (FwdFixedSink)
    win.hi = sD;
    win.lo = nullptr;
    constexpr bool kFixed = METHOD != PAT_METHOD_POINT && KIND == PAT_CYLINDER;
    if (!fwd_window<KIND>(t, tm, g, stl, b0, b1, span, win.base, win.top, s_lohi, kFixed ? x : nullptr)) return;
    const int m = win.top - win.base + 1;
    for (int b = threadIdx.x; b < 2 * m; b += blockDim.x) sD[b] = 0.f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // cylinder surface kernels: the fixed-point window (FwdFixedSink).  x is
    // normalized by 2^-qx (max |x| over the CTA's voxels, from the window pass,
    // below 2^qx; with subnormals flushed 2^-qx is an FP32 number) and the
    // shares by 2^(46 - qa), 2^qa above a bound of the element's area (12.8 R
    // Lz, about 12 times the swept area of the aperture), so that every scaled
    // share stays below 2^46 and no partial sum of the at most 2^14 differences
    // a bin receives from the CTA's pairs comes near 2^62; the flush undoes
    // both in FP64.
    float xscale = 1.f, scale = 1.f;
    double iscale = 1.0;
    bool bad = false; // a non-finite x: the window's rows get NaN, as FP64 arithmetic would give
    if (kFixed) {
        const float xmax = __uint_as_float((unsigned)s_lohi[2]);
        bad = !(xmax <= 3.40282347e38f);
        int qx = 0, qa = 0;
        if (!bad && xmax > 0.f) frexpf(xmax, &qx);
        frexpf(12.8f * t.R * t.Lz, &qa);
        // both powers of two stay normal FP32 numbers: |x| near FLT_MAX moves
        // the rest of its exponent into the share scale, which only shrinks
        const int ex = -min(qx, 125), es = min(46 - qa - (qx + ex), 126);
        xscale = ldexpf(1.f, ex);
        scale = ldexpf(1.f, es);
        iscale = bad ? __longlong_as_double(0x7ff8000000000000LL) : ldexp(1.0, -ex - es); // exact
    }
    __syncthreads();
    for (long long br = b0 + warp; br < b1; br += kWarpsPerBlock) { // warp-uniform trip count
        int ix, iy, iz;
        if (tile_voxel(g, stl, br, lane, ix, iy, iz)) {
            float xv = x[((long long)iz * g.ny + iy) * g.nx + ix];
            if (METHOD == PAT_METHOD_POINT) {
                FwdPointSink s{win, tm.UL, xv, -1, 0.f};
                point_pair<KIND>(t, tm, ix, iy, iz, s);
                s.flush();
            } else if (kFixed) {
                FwdFixedSink s{win, xv * xscale * scale, 0};
                surface_pair<KIND, false, area_mode(METHOD)>(t, tm, ix, iy, iz, s, glx, glw);
            } else {
                FwdSurfaceSink s{win, xv, 0.f};
                surface_pair<KIND, false, area_mode(METHOD)>(t, tm, ix, iy, iz, s, glx, glw);
            }
        }
        __syncwarp();
    }
    __syncthreads();
    double *row = Dg + (size_t)rows[k] * n + win.base;
    const double *wd = (const double *)sD;
    const long long *wl = (const long long *)sD;
    if (gridDim.x == 1 && exclusive) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) row[i] = kFixed ? (double)wl[i] * iscale : wd[i];
    } else {
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const double v = kFixed ? (double)wl[i] * iscale : wd[i];
            if (v != 0.0) atomicAdd(&row[i], v);
        }
    }
}

// Speed-of-sound derivative of the geometric assembly: the difference arrays
// of f (Dg) and of its c-derivative at fixed bins (Dd), same layout and
// window as fwd_geom_kernel (four window arrays in shared memory).
template <int KIND>
__global__ void __launch_bounds__(kThreads) fwd_geom_dc_kernel(const TxDev *__restrict__ tx, TimeDev tm, GridDev g,
                                                               const float *__restrict__ x, double *__restrict__ Dg,
                                                               double *__restrict__ Dd, int bricks_per_cta, int span,
                                                               const int *__restrict__ rows, int exclusive)
{
    extern __shared__ float sD[];
    __shared__ float glx[kGLTable], glw[kGLTable];
    __shared__ int s_lohi[2];
    const int k = blockIdx.y;
    const int n = tm.UL + 1;
    gl_fill(glx, glw, threadIdx.x);
    const TxDev &t = tx[k];
    const long long b0 = (long long)blockIdx.x * bricks_per_cta, b1 = b0 + bricks_per_cta;
    const SuperTile stl = super_tile(g, b0);
    BinWindow win, wind;
    win.hi = sD;
    win.lo = sD + span;
    wind.hi = sD + 2 * span;
    wind.lo = sD + 3 * span;
    if (!fwd_window<KIND>(t, tm, g, stl, b0, b1, span, win.base, win.top, s_lohi)) return;
    wind.base = win.base;
    wind.top = win.top;
    const int m = win.top - win.base + 1;
    for (int b = threadIdx.x; b < m; b += blockDim.x) win.hi[b] = win.lo[b] = wind.hi[b] = wind.lo[b] = 0.f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (long long br = b0 + warp; br < b1; br += kWarpsPerBlock) {
        int ix, iy, iz;
        if (tile_voxel(g, stl, br, lane, ix, iy, iz)) {
            FwdDerivSink s{win, wind, x[((long long)iz * g.ny + iy) * g.nx + ix], 0.f, 0.f};
            surface_pair<KIND, true>(t, tm, ix, iy, iz, s, glx, glw);
        }
        __syncwarp();
    }
    __syncthreads();
    double *row = Dg + (size_t)rows[k] * n + win.base, *rowd = Dd + (size_t)rows[k] * n + win.base;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double v = (double)win.hi[i] + (double)win.lo[i];
        const double vd = (double)wind.hi[i] + (double)wind.lo[i];
        if (gridDim.x == 1 && exclusive) {
            row[i] = v;
            rowd[i] = vd;
        } else {
            if (v != 0.0) atomicAdd(&row[i], v);
            if (vd != 0.0) atomicAdd(&rowd[i], vd);
        }
    }
}

// ---------------------------------------------------------------------------
// block-wide exclusive scan of one double per thread (kThreads threads)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_exclusive_scan(double v, double *tmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        double y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        double w = lane < kWarpsPerBlock ? tmp[lane] : 0.0;
        for (int o = 1; o < 32; o <<= 1) {
            double y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kWarpsPerBlock) tmp[lane] = w; // inclusive warp totals
    }
    __syncthreads();
    double base = warp > 0 ? tmp[warp - 1] : 0.0;
    double r = base + inc - v;
    __syncthreads();
    return r;
}

// 1/(c tau_{b+1/2}) times U Fs, in FP64
__device__ __forceinline__ double bin_weight(const TimeDev &tm, int b)
{
    return tm.ufs / (tm.r0d + ((double)b + 0.5) * tm.deltad);
}

// Convolution with h-bar and downsampling by U (Eq. discrete_conv):
// s[l] = sum_j W[j] f[U l - n_lo + U - 1 - j], W = box_U * h-bar / U.
__device__ __forceinline__ void conv_down(const float *f, const float *W, int nW, int n_lo, const TimeDev &tm,
                                          float *s_out)
{
    for (int l = threadIdx.x; l < tm.L; l += blockDim.x) {
        long long base = (long long)tm.U * l - n_lo + tm.U - 1;
        int j0 = (int)max(0LL, base - (tm.UL - 1));
        int j1 = (int)min((long long)nW - 1, base);
        double acc = 0.0;
        for (int j = j0; j <= j1; ++j) acc = fma((double)W[j], (double)f[base - j], acc);
        s_out[l] = (float)acc;
    }
}

// mode 0: D (difference array of the surface method, doubles) -> f; mode 1:
// H (point histogram, doubles) -> f; mode 2: f given (floats).
__global__ void __launch_bounds__(kThreads) fwd_epilogue_kernel(const void *__restrict__ in, int in_stride,
                                                                 const float *__restrict__ Wg, int nW, int n_lo,
                                                                 TimeDev tm, int mode, float *__restrict__ s,
                                                                 float *__restrict__ f_out, uint16_t *__restrict__ f_hi,
                                                                 uint16_t *__restrict__ f_lo, int ld)
{
    extern __shared__ float sm[];
    __shared__ double tmp[kWarpsPerBlock];
    float *f = sm;            // UL
    float *W = sm + tm.UL;    // nW
    const int k = blockIdx.x;
    const double *drow = (const double *)in + (size_t)k * in_stride;
    const float *row = (const float *)in + (size_t)k * in_stride;
    for (int j = threadIdx.x; j < nW; j += blockDim.x) W[j] = Wg[j];
    const int UL = tm.UL;
    if (mode == 0) {
        const int chunk = (UL + blockDim.x - 1) / blockDim.x;
        const int c0 = min(UL, (int)threadIdx.x * chunk), c1 = min(UL, c0 + chunk);
        double part = 0.0;
        for (int b = c0; b < c1; ++b) part += drow[b];
        double run = block_exclusive_scan(part, tmp);
        for (int b = c0; b < c1; ++b) {
            run += drow[b];
            f[b] = (float)(run * bin_weight(tm, b));
        }
    } else if (mode == 1) {
        for (int b = threadIdx.x; b < UL; b += blockDim.x) f[b] = (float)(drow[b] * tm.ufs);
    } else {
        for (int b = threadIdx.x; b < UL; b += blockDim.x) f[b] = row[b];
    }
    __syncthreads();
    if (f_out) {
        float *fo = f_out + (size_t)k * UL;
        for (int b = threadIdx.x; b < UL; b += blockDim.x) fo[b] = f[b];
    }
    if (f_hi) { // f split into BF16 planes for the tensor-core convolution: hi = bf16(f), lo = bf16(f - hi)
        uint16_t *ho = f_hi + (size_t)k * ld, *lo = f_lo + (size_t)k * ld;
        for (int b = threadIdx.x; b < UL; b += blockDim.x) {
            const __nv_bfloat16 h = __float2bfloat16_rn(f[b]);
            ho[b] = __bfloat16_as_ushort(h);
            lo[b] = __bfloat16_as_ushort(__float2bfloat16_rn(f[b] - __bfloat162float(h)));
        }
    }
    if (s) conv_down(f, W, nW, n_lo, tm, s + (size_t)k * tm.L);
}

// ds/dc = downsample_U(h-bar * f' + (dh-bar/dc) * f) with f' the c-derivative
// of f: f'[b] = prefix(Dd)[b] w_b - f[b] / c (the weight U Fs / (c tau) also
// depends on c).  Dg, Dd: difference arrays [K][UL + 1]; dtaps: dh-bar/dc,
// T doubles, combined with the U-box like W.
__global__ void __launch_bounds__(kThreads) fwd_dc_epilogue_kernel(const double *__restrict__ Dg,
                                                                   const double *__restrict__ Dd,
                                                                   const float *__restrict__ Wg,
                                                                   const double *__restrict__ dtaps, int T, int nW,
                                                                   int n_lo, TimeDev tm, float *__restrict__ ds)
{
    extern __shared__ float sm[];
    __shared__ double tmp[kWarpsPerBlock];
    float *f = sm, *fd = sm + tm.UL, *W = sm + 2 * tm.UL, *Wc = W + nW;
    const int k = blockIdx.x, UL = tm.UL, U = tm.U;
    for (int j = threadIdx.x; j < nW; j += blockDim.x) {
        W[j] = Wg[j];
        double acc = 0.0;
        for (int u = 0; u < U; ++u) {
            const int t = j - (U - 1) + u;
            if (t >= 0 && t < T) acc += dtaps[t];
        }
        Wc[j] = (float)(acc / U);
    }
    const double *drow = Dg + (size_t)k * (UL + 1), *ddrow = Dd + (size_t)k * (UL + 1);
    const int chunk = (UL + blockDim.x - 1) / blockDim.x;
    const int c0 = min(UL, (int)threadIdx.x * chunk), c1 = min(UL, c0 + chunk);
    double part = 0.0, partd = 0.0;
    for (int b = c0; b < c1; ++b) {
        part += drow[b];
        partd += ddrow[b];
    }
    double run = block_exclusive_scan(part, tmp);
    double rund = block_exclusive_scan(partd, tmp);
    for (int b = c0; b < c1; ++b) {
        run += drow[b];
        rund += ddrow[b];
        const double wb = bin_weight(tm, b);
        f[b] = (float)(run * wb);
        fd[b] = (float)(rund * wb - run * wb / tm.c);
    }
    __syncthreads();
    float *out = ds + (size_t)k * tm.L;
    for (int l = threadIdx.x; l < tm.L; l += blockDim.x) {
        const long long bs = (long long)U * l - n_lo + U - 1;
        const int j0 = (int)max(0LL, bs - (UL - 1));
        const int j1 = (int)min((long long)nW - 1, bs);
        double acc = 0.0;
        for (int j = j0; j <= j1; ++j) {
            acc = fma((double)W[j], (double)fd[bs - j], acc);
            acc = fma((double)Wc[j], (double)f[bs - j], acc);
        }
        out[l] = (float)acc;
    }
}

// ---------------------------------------------------------------------------
// adjoint: v = h-bar^- * upsample^T(s); mode 0: P[b] = sum_{b'<b} wgt v (float2
// hi/lo), mode 1: w = U Fs v (point method), mode 2: v itself.  from_v: v
// given, times vscale (in FP64; a power of two undoes the tensor-core
// adjoint's table scale exactly).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) adj_conv_kernel(const float *__restrict__ s, int from_v,
                                                            const float *__restrict__ Wg, int nW, int n_lo,
                                                            TimeDev tm, int mode, void *__restrict__ out,
                                                            double vscale)
{
    extern __shared__ float sm[];
    __shared__ double tmp[kWarpsPerBlock];
    float *ss = sm;          // L
    float *W = sm + tm.L;    // nW
    float *w = W + nW;       // UL (mode 0)
    const int k = blockIdx.x;
    const int UL = tm.UL, U = tm.U, L = tm.L;
    for (int j = threadIdx.x; j < nW; j += blockDim.x) W[j] = Wg[j];
    if (!from_v)
        for (int l = threadIdx.x; l < L; l += blockDim.x) ss[l] = s[(size_t)k * L + l];
    __syncthreads();
    const long long c0 = U - 1 - n_lo;
    const int chunk = (UL + blockDim.x - 1) / blockDim.x;
    const int b0 = min(UL, (int)threadIdx.x * chunk), b1 = min(UL, b0 + chunk);
    double part = 0.0;
    for (int b = b0; b < b1; ++b) {
        // v[b] = sum_l s[l] W[U l + c0 - b], 0 <= U l + c0 - b < nW
        long long lo = b - c0;
        int l0 = (int)max(0LL, lo >= 0 ? (lo + U - 1) / U : -((-lo) / U));
        long long hi = b - c0 + nW - 1;
        int l1 = (int)min((long long)L - 1, hi >= 0 ? hi / U : -1LL);
        double acc = 0.0;
        if (from_v) acc = (double)s[(size_t)k * UL + b] * vscale; // v given (stage entry point, or the
                                                                   // tensor-core adjoint's scaled v)
        else
            for (int l = l0; l <= l1; ++l) acc = fma((double)ss[l], (double)W[U * l + c0 - b], acc);
        if (mode == 0) {
            double wv = acc * bin_weight(tm, b);
            w[b] = (float)wv;
            part += (double)w[b];
        } else if (mode == 1) {
            ((float *)out)[(size_t)k * (UL + 1) + b] = (float)(acc * tm.ufs);
        } else {
            ((float *)out)[(size_t)k * UL + b] = (float)acc;
        }
    }
    if (mode != 0) return;
    double run = block_exclusive_scan(part, tmp);
    float2 *P = (float2 *)out + (size_t)k * (UL + 1);
    for (int b = b0; b < b1; ++b) {
        float hi = (float)run;
        P[b] = make_float2(hi, (float)(run - (double)hi));
        run += (double)w[b];
    }
    if (b1 == UL && b0 < b1) {
        float hi = (float)run;
        P[UL] = make_float2(hi, (float)(run - (double)hi));
    }
    if (UL == 0 && threadIdx.x == 0) P[0] = make_float2(0.f, 0.f);
}

// ---------------------------------------------------------------------------
// adjoint gather
// ---------------------------------------------------------------------------
struct AdjSurfaceSink {
    const float2 *__restrict__ P;
    int UL;
    float acc;
    float2 pe;  // P at the current group start, loaded by start()
    float2 pn;  // P at its end, loaded by pre()
    __device__ __forceinline__ int clampi(int e) const { return min(max(e, 0), UL); }
    __device__ __forceinline__ void start(int e) { pe = __ldg(&P[clampi(e)]); }
    __device__ __forceinline__ void pre(int, int e1) { pn = __ldg(&P[clampi(e1)]); }
    __device__ __forceinline__ void group(int, int, float val, float)
    {
        acc = fmaf(val, (pn.x - pe.x) + (pn.y - pe.y), acc);
        pe = pn;
    }
    __device__ __forceinline__ void finish(int) {}
};

struct AdjPointSink {
    const float *__restrict__ w;
    int UL;
    float acc;
    __device__ __forceinline__ void point(int b, float wt)
    {
        if (b >= 0 && b < UL) acc = fmaf(wt, __ldg(&w[b]), acc);
    }
};

template <int METHOD, int KIND>
__global__ void __launch_bounds__(kThreads, geom_min_ctas(KIND, false)) adj_geom_kernel(const TxDev *__restrict__ tx, int K, TimeDev tm,
                                                            GridDev g, const void *__restrict__ Pv,
                                                            float *__restrict__ z, const int *__restrict__ rows)
{
    __shared__ float glx[kGLTable], glw[kGLTable];
    gl_fill(glx, glw, threadIdx.x);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long br = (long long)blockIdx.x * (blockDim.x >> 5) + warp; // one brick per warp
    if (br >= g.nbricks) return;
    int ix, iy, iz;
    const bool ok = brick_voxel(g, br, lane, ix, iy, iz); // ragged bricks: idle lanes stay for the syncs
    const int stride = tm.UL + 1;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
        if (ok) {
            const TxDev &t = tx[k];
            if (METHOD == PAT_METHOD_POINT) {
                AdjPointSink s{(const float *)Pv + (size_t)rows[k] * stride, tm.UL, 0.f};
                point_pair<KIND>(t, tm, ix, iy, iz, s);
                acc += (double)s.acc;
            } else {
                AdjSurfaceSink s{(const float2 *)Pv + (size_t)rows[k] * stride, tm.UL, 0.f, make_float2(0.f, 0.f),
                                 make_float2(0.f, 0.f)};
                surface_pair<KIND, false, area_mode(METHOD)>(t, tm, ix, iy, iz, s, glx, glw);
                acc += (double)s.acc;
            }
        }
        __syncwarp(); // reconverge before the next pair (FP64 setup at full width)
    }
    if (!ok) return;
    z[((long long)iz * g.ny + iy) * g.nx + ix] = (float)acc;
}

// ---------------------------------------------------------------------------
// discrete system kernel (Eq. def_bh) on the device, FP64
// h-bar[n] = (1/D) int_{-D}^{D} (D - |s|) h(n D + s) ds,  h(t) = int e(t') g(t - t') dt'
// Composite 16-point Gauss-Legendre, nodes by Newton iteration on P_16.
// ---------------------------------------------------------------------------
constexpr int kGL = 16;

struct SysDev {
    int rbf, eir;
    double kappa, c;
    double e[4];
};

__device__ double rbf_dev(int kind, double kappa, double r)
{
    r = fabs(r);
    if (r >= kappa) return 0.0;
    double q = r / kappa;
    if (kind == PAT_RBF_BUMP) return (1.0 - q * q) * (1.0 - q * q);
    if (kind == PAT_RBF_CONE) return 1.0 - q;
    return (1.0 - q) * (1.0 - q);
}

// d(r phi(r))/dr, the radial factor of dg/dc: g(t) = -1/2 c t phi(|c t|) gives
// dg/dc = -1/2 t [phi(rho) + rho phi'(rho)], rho = |c t|.
__device__ double rbf_dc_dev(int kind, double kappa, double r)
{
    r = fabs(r);
    if (r >= kappa) return 0.0;
    double q = r / kappa;
    if (kind == PAT_RBF_BUMP) return (1.0 - q * q) * (1.0 - 5.0 * q * q);
    if (kind == PAT_RBF_CONE) return 1.0 - 2.0 * q;
    return (1.0 - q) * (1.0 - 3.0 * q);
}

__device__ double eir_dev(const SysDev &sy, double t)
{
    if (t < 0.0 || t > sy.e[3]) return 0.0;
    if (sy.eir == PAT_EIR_GAUSS_SINE) {
        double d = t - sy.e[2];
        return exp(-d * d / (2.0 * sy.e[1] * sy.e[1])) * sin(2.0 * 3.141592653589793 * sy.e[0] * d);
    }
    return sy.e[0];
}

// h(t) = (e * g)(t); with dc, (e * dg/dc)(t) instead.
__device__ double h_dev(const SysDev &sy, const double *gx, const double *gw, double t, bool dc = false)
{
    // pieces of [max(0, t - k/c), min(Te, t + k/c)] split at t (kink of g at 0)
    const double kc = sy.kappa / sy.c;
    double a = fmax(0.0, t - kc), b = fmin(sy.e[3], t + kc);
    if (!(b > a)) return 0.0;
    double cuts[3] = {a, b, b};
    int nc = 2;
    if (t > a && t < b) {
        cuts[1] = t;
        cuts[2] = b;
        nc = 3;
    }
    double acc = 0.0;
    const int panels = 4;
    for (int p = 0; p + 1 < nc; ++p) {
        double lo = cuts[p], hi = cuts[p + 1], wdt = (hi - lo) / panels;
        for (int q = 0; q < panels; ++q) {
            double m = lo + (q + 0.5) * wdt;
            for (int i = 0; i < kGL; ++i) {
                double tp = m + 0.5 * wdt * gx[i];
                double ct = sy.c * (t - tp);
                const double g = dc ? -0.5 * (t - tp) * rbf_dc_dev(sy.rbf, sy.kappa, ct)
                                    : -0.5 * ct * rbf_dev(sy.rbf, sy.kappa, ct);
                acc += 0.5 * wdt * gw[i] * eir_dev(sy, tp) * g;
            }
        }
    }
    return acc;
}

__global__ void taps_kernel(SysDev sy, double ufs, int n_lo, int T, double *__restrict__ taps, bool dc)
{
    __shared__ double gx[kGL], gw[kGL];
    if (threadIdx.x < kGL) {
        int i = threadIdx.x;
        double x = cos(3.141592653589793 * (i + 0.75) / (kGL + 0.5)), dp = 1.0;
        for (int it = 0; it < 60; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= kGL; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = kGL * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        gx[i] = x;
        gw[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    __syncthreads();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const double D = 1.0 / ufs, kc = sy.kappa / sy.c, Te = sy.e[3];
    const double nD = (double)(n_lo + t) * D;
    // breakpoints of the triangle weight (0) and of h (kinks of e and g, shifted)
    double bp[9];
    int nb = 0;
    bp[nb++] = -D;
    bp[nb++] = 0.0;
    bp[nb++] = D;
    const double kinks[6] = {-kc, 0.0, kc, Te - kc, Te, Te + kc};
    for (int i = 0; i < 6; ++i) {
        double s = kinks[i] - nD;
        if (s > -D && s < D && s != 0.0) bp[nb++] = s;
    }
    for (int i = 1; i < nb; ++i) // insertion sort
        for (int j = i; j > 0 && bp[j - 1] > bp[j]; --j) {
            double tt = bp[j];
            bp[j] = bp[j - 1];
            bp[j - 1] = tt;
        }
    double acc = 0.0;
    const int panels = 3;
    for (int p = 0; p + 1 < nb; ++p) {
        double lo = bp[p], hi = bp[p + 1];
        if (!(hi > lo)) continue;
        double wdt = (hi - lo) / panels;
        for (int q = 0; q < panels; ++q) {
            double m = lo + (q + 0.5) * wdt;
            for (int i = 0; i < kGL; ++i) {
                double sv = m + 0.5 * wdt * gx[i];
                acc += 0.5 * wdt * gw[i] * (D - fabs(sv)) * h_dev(sy, gx, gw, nD + sv, dc);
            }
        }
    }
    taps[t] = acc / D;
}

// W[j] = (1/U) sum_{u<U} h-bar[n_lo + j - (U-1) + u]: the U-box and h-bar combined
__global__ void combine_taps_kernel(const double *__restrict__ taps, int T, int U, float *__restrict__ W)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int nW = T + U - 1;
    if (j >= nW) return;
    double acc = 0.0;
    for (int u = 0; u < U; ++u) {
        int t = j - (U - 1) + u;
        if (t >= 0 && t < T) acc += taps[t];
    }
    W[j] = (float)(acc / U);
}

// ---------------------------------------------------------------------------
// vector kernels for the FISTA loop of pat_recon
// ---------------------------------------------------------------------------
__global__ void sub_kernel(const float *__restrict__ a, const float *__restrict__ b, float *__restrict__ o, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        o[i] = a[i] - b[i];
}

// x_new = max(0, y - step (g + lam y)); y = x_new + mom (x_new - x_old); x_old = x_new.
// The momentum comes from the device scalars of fista_momentum_kernel, so
// that one iteration is the same launch sequence every time (graph replay).
__global__ void fista_kernel(float *__restrict__ y, const float *__restrict__ g, float *__restrict__ xo, long long n,
                             float step, float lam, const double *__restrict__ tstate)
{
    const float mom = (float)tstate[1];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float yi = y[i];
        float xn = fmaxf(0.f, yi - step * (g[i] + lam * yi));
        float xold = xo[i];
        xo[i] = xn;
        y[i] = xn + mom * (xn - xold);
    }
}

// FISTA step-size sequence on the device: t' = (1 + sqrt(1 + 4 t^2)) / 2,
// momentum (t - 1) / t'.  tstate[0] = t, tstate[1] = momentum of this step.
__global__ void fista_momentum_kernel(double *__restrict__ tstate)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double t = tstate[0], tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        tstate[1] = (t - 1.0) / tn;
        tstate[0] = tn;
    }
}

__global__ void dot_kernel(const float *__restrict__ a, const float *__restrict__ b, long long n,
                           double *__restrict__ out)
{
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

__global__ void scale_kernel(const float *__restrict__ a, float *__restrict__ o, long long n,
                             const double *__restrict__ nrm2)
{
    float sc = (float)(1.0 / sqrt(fmax(nrm2[0], 1e-300)));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        o[i] = a[i] * sc;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
// Dynamic shared memory above 48 KB needs an opt-in per function; set it only
// when a launch needs more than the default.
static void set_smem_attr(const void *fn, size_t bytes)
{
    if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
cudaError_t launch_frames(const double *raw, int K, const double *origin, double pitch, int q1, int q2, TxDev *out,
                          cudaStream_t st)
{
    frames_kernel<<<(K + 127) / 128, 128, 0, st>>>(raw, K, origin[0], origin[1], origin[2], pitch, q1, q2, out);
    return cudaGetLastError();
}

// The forward-chunk kernels take the element from blockIdx.y; more elements
// than a grid's y extent go in slabs of launches.
constexpr int kMaxGridY = 65535;

// a forward chunk: a power of two of bricks, at least one per warp, inside one super-tile
static bool fwd_bpc_ok(int bpc)
{
    return bpc >= kWarpsPerBlock && bpc <= kSuperBricks && (bpc & (bpc - 1)) == 0;
}

cudaError_t launch_scan(const TxDev *tx, int K, const TimeDev &tm, const GridDev &g, int bpc, ScanOut s,
                        cudaStream_t st)
{
    if (!fwd_bpc_ok(bpc)) return cudaErrorInvalidValue;
    scan_init_kernel<<<(K + 255) / 256, 256, 0, st>>>(s, K);
    for (int k0 = 0; k0 < K; k0 += kMaxGridY) { // elements along grid y, in slabs
        ScanOut sk = s;
        sk.lo += k0;
        sk.hi += k0;
        sk.groups += k0;
        sk.bins += k0;
        sk.clipped += k0;
        sk.quads += k0;
        const dim3 grid((unsigned)(g.nvb / bpc), (unsigned)std::min(kMaxGridY, K - k0));
        scan_kernel<<<grid, kThreads, 0, st>>>(tx + k0, tm, g, bpc, sk);
    }
    return cudaGetLastError();
}

// One instantiation per (method, element kind); kind kKindAny reads it from
// each descriptor.
struct FacetArgs {
    const int *rows;
    int exclusive;
};

template <int METHOD, int KIND>
static cudaError_t fwd_geom_go(dim3 grid, size_t smem, cudaStream_t st, const TxDev *tx, const TimeDev &tm,
                               const GridDev &g, const float *x, double *Dg, int bpc, int span, FacetArgs fa)
{
    set_smem_attr((const void *)fwd_geom_kernel<METHOD, KIND>, smem);
    fwd_geom_kernel<METHOD, KIND><<<grid, kThreads, smem, st>>>(tx, tm, g, x, Dg, bpc, span, fa.rows, fa.exclusive);
    return cudaGetLastError();
}

static cudaError_t fwd_geom_dispatch(dim3 grid, size_t smem, cudaStream_t st, const TxDev *tx, int kind,
                                     const TimeDev &tm, const GridDev &g, const float *x, double *Dg, int b, int span,
                                     FacetArgs fa)
{
    if (tm.method == PAT_METHOD_POINT) {
        if (kind == PAT_PLANE) return fwd_geom_go<PAT_METHOD_POINT, PAT_PLANE>(grid, smem, st, tx, tm, g, x, Dg, b, span, fa);
        if (kind == PAT_CYLINDER)
            return fwd_geom_go<PAT_METHOD_POINT, PAT_CYLINDER>(grid, smem, st, tx, tm, g, x, Dg, b, span, fa);
        return fwd_geom_go<PAT_METHOD_POINT, kKindAny>(grid, smem, st, tx, tm, g, x, Dg, b, span, fa);
    }
    if (tm.method == PAT_METHOD_TRAPEZOID) {
        if (kind == PAT_PLANE)
            return fwd_geom_go<PAT_METHOD_TRAPEZOID, PAT_PLANE>(grid, smem, st, tx, tm, g, x, Dg, b, span, fa);
        if (kind == PAT_CYLINDER)
            return fwd_geom_go<PAT_METHOD_TRAPEZOID, PAT_CYLINDER>(grid, smem, st, tx, tm, g, x, Dg, b, span, fa);
        return fwd_geom_go<PAT_METHOD_TRAPEZOID, kKindAny>(grid, smem, st, tx, tm, g, x, Dg, b, span, fa);
    }
    if (tm.method == PAT_METHOD_LUT && kind != PAT_PLANE) { // planes keep their closed form
        if (kind == PAT_CYLINDER)
            return fwd_geom_go<PAT_METHOD_LUT, PAT_CYLINDER>(grid, smem, st, tx, tm, g, x, Dg, b, span, fa);
        return fwd_geom_go<PAT_METHOD_LUT, kKindAny>(grid, smem, st, tx, tm, g, x, Dg, b, span, fa);
    }
    if (kind == PAT_PLANE) return fwd_geom_go<PAT_METHOD_SURFACE, PAT_PLANE>(grid, smem, st, tx, tm, g, x, Dg, b, span, fa);
    if (kind == PAT_CYLINDER)
        return fwd_geom_go<PAT_METHOD_SURFACE, PAT_CYLINDER>(grid, smem, st, tx, tm, g, x, Dg, b, span, fa);
    return fwd_geom_go<PAT_METHOD_SURFACE, kKindAny>(grid, smem, st, tx, tm, g, x, Dg, b, span, fa);
}

cudaError_t launch_fwd_geom(const TxDev *tx, int Kf, int K, const int *rows, int kind, const TimeDev &tm,
                            const GridDev &g, const float *x, double *Dg, int bpc, int span, cudaStream_t st)
{
    if (!fwd_bpc_ok(bpc)) return cudaErrorInvalidValue;
    size_t smem = 2 * sizeof(float) * (size_t)span;
    unsigned gx = (unsigned)(g.nvb / bpc);
    cudaError_t e = cudaMemsetAsync(Dg, 0, sizeof(double) * (size_t)(tm.UL + 1) * K, st);
    for (int k0 = 0; k0 < Kf && e == cudaSuccess; k0 += kMaxGridY) {
        const dim3 grid(gx, (unsigned)std::min(kMaxGridY, Kf - k0));
        e = fwd_geom_dispatch(grid, smem, st, tx + k0, kind, tm, g, x, Dg, bpc, span,
                              FacetArgs{rows + k0, Kf == K ? 1 : 0});
    }
    return e;
}

cudaError_t launch_fwd_geom_dc(const TxDev *tx, int Kf, int K, const int *rows, int kind, const TimeDev &tm,
                               const GridDev &g, const float *x, double *Dg, double *Dd, int bpc, int span,
                               cudaStream_t st)
{
    if (!fwd_bpc_ok(bpc)) return cudaErrorInvalidValue;
    size_t smem = 4 * sizeof(float) * (size_t)span;
    unsigned gx = (unsigned)(g.nvb / bpc);
    const size_t bytes = sizeof(double) * (size_t)(tm.UL + 1) * K;
    cudaError_t e = cudaMemsetAsync(Dg, 0, bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(Dd, 0, bytes, st);
    if (e != cudaSuccess) return e;
    const int excl = Kf == K ? 1 : 0;
    const void *fn = kind == PAT_PLANE      ? (const void *)fwd_geom_dc_kernel<PAT_PLANE>
                     : kind == PAT_CYLINDER ? (const void *)fwd_geom_dc_kernel<PAT_CYLINDER>
                                            : (const void *)fwd_geom_dc_kernel<kKindAny>;
    set_smem_attr(fn, smem);
    for (int k0 = 0; k0 < Kf; k0 += kMaxGridY) {
        const dim3 grid(gx, (unsigned)std::min(kMaxGridY, Kf - k0));
        const TxDev *t = tx + k0;
        const int *r = rows + k0;
        if (kind == PAT_PLANE)
            fwd_geom_dc_kernel<PAT_PLANE><<<grid, kThreads, smem, st>>>(t, tm, g, x, Dg, Dd, bpc, span, r, excl);
        else if (kind == PAT_CYLINDER)
            fwd_geom_dc_kernel<PAT_CYLINDER><<<grid, kThreads, smem, st>>>(t, tm, g, x, Dg, Dd, bpc, span, r, excl);
        else
            fwd_geom_dc_kernel<kKindAny><<<grid, kThreads, smem, st>>>(t, tm, g, x, Dg, Dd, bpc, span, r, excl);
    }
    return cudaGetLastError();
}

cudaError_t launch_fwd_dc_epilogue(const double *Dg, const double *Dd, const float *W, const double *dtaps, int T,
                                   int nW, int n_lo, const TimeDev &tm, int K, float *ds, cudaStream_t st)
{
    size_t smem = sizeof(float) * (size_t)(2 * tm.UL + 2 * nW);
    set_smem_attr((const void *)fwd_dc_epilogue_kernel, smem);
    fwd_dc_epilogue_kernel<<<K, kThreads, smem, st>>>(Dg, Dd, W, dtaps, T, nW, n_lo, tm, ds);
    return cudaGetLastError();
}

cudaError_t launch_fwd_epilogue(const void *in, int in_stride, const float *W, int nW, int n_lo, const TimeDev &tm,
                                int mode, int K, float *s, float *f_out, cudaStream_t st, uint16_t *f_hi,
                                uint16_t *f_lo, int ld)
{
    size_t smem = sizeof(float) * (size_t)(tm.UL + nW);
    set_smem_attr((const void *)fwd_epilogue_kernel, smem);
    fwd_epilogue_kernel<<<K, kThreads, smem, st>>>(in, in_stride, W, nW, n_lo, tm, mode, s, f_out, f_hi, f_lo, ld);
    return cudaGetLastError();
}

cudaError_t launch_adj_conv(const float *s, int from_v, const float *W, int nW, int n_lo, const TimeDev &tm, int mode,
                            int K, void *out, cudaStream_t st, double vscale)
{
    size_t smem = sizeof(float) * (size_t)(tm.L + nW + (mode == 0 ? tm.UL : 0));
    set_smem_attr((const void *)adj_conv_kernel, smem);
    adj_conv_kernel<<<K, kThreads, smem, st>>>(s, from_v, W, nW, n_lo, tm, mode, out, vscale);
    return cudaGetLastError();
}

cudaError_t launch_adj_geom(const TxDev *tx, int K, const int *rows, int kind, const TimeDev &tm, const GridDev &g,
                            const void *P, float *z, cudaStream_t st, int wpb)
{
    wpb = wpb == 4 || wpb == 2 ? wpb : kWarpsPerBlock; // warps (bricks) per CTA
    const unsigned grid = (unsigned)((g.nbricks + wpb - 1) / wpb), thr = 32u * wpb;
    if (tm.method == PAT_METHOD_POINT) {
        if (kind == PAT_PLANE) adj_geom_kernel<PAT_METHOD_POINT, PAT_PLANE><<<grid, thr, 0, st>>>(tx, K, tm, g, P, z, rows);
        else if (kind == PAT_CYLINDER)
            adj_geom_kernel<PAT_METHOD_POINT, PAT_CYLINDER><<<grid, thr, 0, st>>>(tx, K, tm, g, P, z, rows);
        else adj_geom_kernel<PAT_METHOD_POINT, kKindAny><<<grid, thr, 0, st>>>(tx, K, tm, g, P, z, rows);
    } else if (tm.method == PAT_METHOD_TRAPEZOID) {
        if (kind == PAT_PLANE) adj_geom_kernel<PAT_METHOD_TRAPEZOID, PAT_PLANE><<<grid, thr, 0, st>>>(tx, K, tm, g, P, z, rows);
        else if (kind == PAT_CYLINDER)
            adj_geom_kernel<PAT_METHOD_TRAPEZOID, PAT_CYLINDER><<<grid, thr, 0, st>>>(tx, K, tm, g, P, z, rows);
        else adj_geom_kernel<PAT_METHOD_TRAPEZOID, kKindAny><<<grid, thr, 0, st>>>(tx, K, tm, g, P, z, rows);
    } else if (tm.method == PAT_METHOD_LUT && kind != PAT_PLANE) { // planes keep their closed form
        if (kind == PAT_CYLINDER)
            adj_geom_kernel<PAT_METHOD_LUT, PAT_CYLINDER><<<grid, thr, 0, st>>>(tx, K, tm, g, P, z, rows);
        else adj_geom_kernel<PAT_METHOD_LUT, kKindAny><<<grid, thr, 0, st>>>(tx, K, tm, g, P, z, rows);
    } else {
        if (kind == PAT_PLANE) adj_geom_kernel<PAT_METHOD_SURFACE, PAT_PLANE><<<grid, thr, 0, st>>>(tx, K, tm, g, P, z, rows);
        else if (kind == PAT_CYLINDER)
            adj_geom_kernel<PAT_METHOD_SURFACE, PAT_CYLINDER><<<grid, thr, 0, st>>>(tx, K, tm, g, P, z, rows);
        else adj_geom_kernel<PAT_METHOD_SURFACE, kKindAny><<<grid, thr, 0, st>>>(tx, K, tm, g, P, z, rows);
    }
    return cudaGetLastError();
}

cudaError_t launch_taps(int rbf, int eir, double kappa, double c, const double *e, double ufs, int n_lo, int T,
                        double *taps, cudaStream_t st, bool dc)
{
    SysDev sy;
    sy.rbf = rbf;
    sy.eir = eir;
    sy.kappa = kappa;
    sy.c = c;
    for (int i = 0; i < 4; ++i) sy.e[i] = e[i];
    taps_kernel<<<(T + 63) / 64, 64, 0, st>>>(sy, ufs, n_lo, T, taps, dc);
    return cudaGetLastError();
}

cudaError_t launch_combine_taps(const double *taps, int T, int U, float *W, cudaStream_t st)
{
    int nW = T + U - 1;
    combine_taps_kernel<<<(nW + 255) / 256, 256, 0, st>>>(taps, T, U, W);
    return cudaGetLastError();
}

cudaError_t launch_sub(const float *a, const float *b, float *o, long long n, cudaStream_t st)
{
    sub_kernel<<<1216, 256, 0, st>>>(a, b, o, n);
    return cudaGetLastError();
}

cudaError_t launch_fista(float *y, const float *g, float *xo, long long n, float step, float lam, double *tstate,
                         cudaStream_t st)
{
    fista_momentum_kernel<<<1, 32, 0, st>>>(tstate);
    fista_kernel<<<1216, 256, 0, st>>>(y, g, xo, n, step, lam, tstate);
    return cudaGetLastError();
}

cudaError_t launch_dot(const float *a, const float *b, long long n, double *out, cudaStream_t st)
{
    cudaMemsetAsync(out, 0, sizeof(double), st);
    dot_kernel<<<1216, 256, 0, st>>>(a, b, n, out);
    return cudaGetLastError();
}

cudaError_t launch_scale(const float *a, float *o, long long n, const double *nrm2, cudaStream_t st)
{
    scale_kernel<<<1216, 256, 0, st>>>(a, o, n, nrm2);
    return cudaGetLastError();
}

} // namespace pat
