// pat_conv_tc.cuh -- host side of the tensor-core (tcgen05) temporal
// convolution and its transpose (pat_conv_tc.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pat {

constexpr int kTcM = 128;      // output samples per tile (MMA M)
constexpr int kTcN = 64;       // transducers per tile (MMA N)
constexpr int kTcKStage = 64;  // contraction length per pipeline stage
constexpr int kTcThreads = 128;     // adjoint kernel
constexpr int kTcThreadsFwd = 544;  // forward kernel: sixteen converter warps and the issuing warp
constexpr int kTcN2 = 256;          // transducers per tile of the split-plane forward
constexpr int kTcThreadsFwd2 = 192; // split-plane forward: copy warp, MMA warp, four epilogue warps

// Tile geometry of one plan (taps, U, n_lo fixed).
struct TcGeometry {
    int c;         // U - 1 - n_lo
    int m0off;     // forward window start: m0 = U l0 + m0off
    int nst_fwd;   // forward stages per tile
    int d0;        // adjoint window start: l = m0 + d0 + lambda
    int nst_adj;   // adjoint stages per tile and phase
    size_t fwd_table_bytes, adj_table_bytes;
    size_t fwd_smem, adj_smem; // dynamic shared memory per CTA
    int sms;                   // SMs of the device (the forward kernel splits its stages to fill them)
    // split-plane forward (f as BF16 hi and lo planes of [K][ld])
    int shift;                 // m0off mod 8: leading zero columns of its table
    int m0a;                   // its window start: m0 = U l0 + m0a, a multiple of 8
    int nst_fwd2;              // its stages per tile
    int ld;                    // plane row length: U L rounded up to a multiple of 8
    size_t fwd2_table_bytes, fwd2_smem;
    // The operand tables hold W 2^tscale, with max |W| 2^tscale in [1/U, 2):
    // the system kernel in SI units is of order 1e-20, and the products of
    // the hi / lo split (about 2^-8 of W times the signal) would otherwise
    // fall below FP32's smallest normal in the tensor cores.  The kernels
    // multiply their outputs by oscale (2^-tscale, exact); 0 until the plan
    // sets it from its taps.
    int tscale;
};

TcGeometry tc_geometry(int T, int U, int L, int n_lo);
// Toeplitz operand tables (BF16 hi / lo, shared-memory layout) from the FP64
// taps, times 2^g.tscale.
cudaError_t launch_tc_tables(const double *taps, int T, int U, const TcGeometry &g, uint8_t *Tf, uint8_t *Ta,
                             uint8_t *Tf2, cudaStream_t st);
// s[K][L] from f[K][U L]; v[K][U L] from s[K][L].  err: device int, set
// non-zero if a CTA gave up waiting on the TMA engine or the tensor cores.
cudaError_t launch_conv_tc_fwd(const float *f, const uint8_t *Tf, const TcGeometry &g, int K, int L, int U, float *s,
                               int *err, cudaStream_t st);
// unscale = false leaves v times 2^g.tscale (a consumer that undoes it in FP64).
cudaError_t launch_conv_tc_adj(const float *s, const uint8_t *Ta, const TcGeometry &g, int K, int L, int U, float *v,
                               int *err, cudaStream_t st, bool unscale = true);
// f [K][U L] floats -> BF16 hi and lo planes [K][g.ld] (hi = bf16(f), lo = bf16(f - hi)).
cudaError_t launch_split_bf16(const float *f, int K, int UL, int ld, uint16_t *hi, uint16_t *lo, cudaStream_t st);
// s [K][L] from the hi and lo planes (16-byte aligned, rows of g.ld, only the
// first U L columns of a row read): the persistent tensor-map / tcgen05 kernel.
// withhold: a test of its give-up path on one CTA (at least 3 tiles; s is
// then undefined and *err becomes non-zero after about two seconds).
cudaError_t launch_conv_tc_fwd2(const uint16_t *hi, const uint16_t *lo, const uint8_t *Tf2, const TcGeometry &g, int K,
                                int L, int U, float *s, int *err, cudaStream_t st, bool withhold = false);

} // namespace pat
