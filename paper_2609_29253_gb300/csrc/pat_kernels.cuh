// pat_kernels.cuh -- host-side launchers of the PAT kernels (pat_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "pat_internal.cuh"

namespace pat {

// Per-transducer results of the plan-time scan over all pairs.
struct ScanOut {
    long long *lo, *hi;                      // extreme fine bins
    unsigned long long *groups, *bins, *clipped, *quads;
    unsigned long long *rmin_bits;           // min distance (bits of a positive double)
    unsigned long long *maxspan;             // largest forward window (edges) over the CTAs
    unsigned long long *misses;              // pairs whose edges the window bound of pass 1 would miss (0)
};

cudaError_t launch_frames(const double *raw, int K, const double *origin, double pitch, int q1, int q2, TxDev *out,
                          cudaStream_t st);
// bpc: bricks per CTA of the forward kernels the scan sizes the window for
// (a power of two from kWarpsPerBlock to kSuperBricks, else cudaErrorInvalidValue)
cudaError_t launch_scan(const TxDev *tx, int K, const TimeDev &tm, const GridDev &g, int bpc, ScanOut s,
                        cudaStream_t st);
// Dg: [K][UL + 1] doubles.  CTA (i, k) takes bricks [i bpc, (i + 1) bpc) of the
// super-tile-major order against element k; span: the largest fine-bin window
// of a CTA (from the scan with a chunking that bpc divides).
// kind: PAT_PLANE or PAT_CYLINDER when every descriptor has it, else kKindAny.
// Kf elements (or plane facets) add into K signal rows, element k into
// rows[k] (Kf == K: one element per row).
cudaError_t launch_fwd_geom(const TxDev *tx, int Kf, int K, const int *rows, int kind, const TimeDev &tm,
                            const GridDev &g, const float *x, double *Dg, int bpc, int span, cudaStream_t st);
// in: doubles for mode 0 / 1 (difference array, histogram), floats for mode 2 (f);
// f_hi, f_lo (optional): f as BF16 hi and lo planes of row length ld
cudaError_t launch_fwd_epilogue(const void *in, int in_stride, const float *W, int nW, int n_lo, const TimeDev &tm,
                                int mode, int K, float *s, float *f_out, cudaStream_t st, uint16_t *f_hi = nullptr,
                                uint16_t *f_lo = nullptr, int ld = 0);
// from_v: in is v [K][U L], multiplied by vscale in FP64 as it is read
cudaError_t launch_adj_conv(const float *in, int from_v, const float *W, int nW, int n_lo, const TimeDev &tm, int mode,
                            int K, void *out, cudaStream_t st, double vscale = 1.0);
// wpb: warps (4x4x2 voxel bricks) per CTA, 2, 4 or 8
cudaError_t launch_adj_geom(const TxDev *tx, int K, const int *rows, int kind, const TimeDev &tm, const GridDev &g,
                            const void *P, float *z, cudaStream_t st, int wpb = kWarpsPerBlock);
// dc: dh-bar/dc instead of h-bar
cudaError_t launch_taps(int rbf, int eir, double kappa, double c, const double *e, double ufs, int n_lo, int T,
                        double *taps, cudaStream_t st, bool dc = false);
// speed-of-sound derivative: difference arrays of f and of df/dc (fixed bins)
cudaError_t launch_fwd_geom_dc(const TxDev *tx, int Kf, int K, const int *rows, int kind, const TimeDev &tm,
                               const GridDev &g, const float *x, double *Dg, double *Dd, int bpc, int span,
                               cudaStream_t st);
cudaError_t launch_fwd_dc_epilogue(const double *Dg, const double *Dd, const float *W, const double *dtaps, int T,
                                   int nW, int n_lo, const TimeDev &tm, int K, float *ds, cudaStream_t st);
cudaError_t launch_combine_taps(const double *taps, int T, int U, float *W, cudaStream_t st);
cudaError_t launch_sub(const float *a, const float *b, float *o, long long n, cudaStream_t st);
// advances the device momentum state tstate = {t, momentum}, then the update
cudaError_t launch_fista(float *y, const float *g, float *xo, long long n, float step, float lam, double *tstate,
                         cudaStream_t st);
cudaError_t launch_dot(const float *a, const float *b, long long n, double *out, cudaStream_t st);
cudaError_t launch_scale(const float *a, float *o, long long n, const double *nrm2, cudaStream_t st);
// PAT_METHOD_LUT (pat_lut.cu): device bytes of the tables of an ns x nm grid, and their
// construction into buf (lut_bytes(ns, nm) bytes) through scratch (ns nm double2), filling L
size_t lut_bytes(int ns, int nm);
cudaError_t launch_lut_tables(int ns, int nm, void *buf, double2 *scratch, LutDev &L, cudaStream_t st);

} // namespace pat
