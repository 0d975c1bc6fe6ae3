// pat_conv_tc.cu -- the temporal convolution of A and its transpose as
// Toeplitz contractions on the tcgen05 tensor cores (sm_103a).
//
// Forward (Eq. discrete_conv, filter then downsample by U):
//   s[k][l] = sum_j W[j] f[k][U l + c - j],   c = U - 1 - n_lo,
// with W = box_U * h-bar / U (nW = T + U - 1 taps) and f = 0 outside
// [0, U L).  For an output tile l = l0 + i, i < 128, the inputs lie in the
// window m = m0 + mu, m0 = U l0 + c - (nW - 1), mu < 127 U + nW, and
//   s[k][l0 + i] = sum_mu Tf[i][mu] f[k][m0 + mu],  Tf[i][mu] = W[U i + nW - 1 - mu],
// where Tf does not depend on l0: one constant Toeplitz matrix for every tile.
//
// Adjoint (App. G, transpose of the above):
//   v[k][b] = sum_l s[k][l] W[U l + c - b].
// Split b = U m + p (polyphase, p < U) and l = m + d:
//   v[k][U (m0 + i) + p] = sum_lambda Ta_p[i][lambda] s[k][m0 + d0 + lambda],
//   Ta_p[i][lambda] = W[U (d0 + lambda - i) + c - p],
// with d0 the smallest d that any phase reaches; again one constant matrix per
// phase for every tile m0.
//
// Each CTA computes one D = T (128 x Kw) x B^T (Kw x 64) tile: M = 128 output
// samples, N = 64 transducers, in K stages of 64.  Operands are BF16 split in
// two (x = hi + lo, hi = bf16(x), lo = bf16(x - hi)) and the tile is
// accumulated as hi*hi + hi*lo + lo*hi in FP32 in tensor memory, which keeps
// about 16 significant bits per product (a single BF16 pass loses too much to
// the cancellation of the band-pass kernel: Sum h-bar = 0).
//
//   * T (hi and lo) is precomputed once per plan, per stage, in the exact
//     shared-memory operand layout, and brought in by one bulk copy (TMA,
//     cp.async.bulk) per stage, completing on an mbarrier;
//   * B (f or s rows, FP32 in HBM) is read with coalesced loads, split, and
//     stored in the operand layout by all threads;
//   * one thread issues tcgen05.mma (kind::f16, BF16 in, FP32 accumulate,
//     M = 128, N = 64, K = 16) and tcgen05.commit onto an mbarrier that frees
//     the stage's buffers; the forward kernel cycles a four-slot ring of
//     stage buffers, the adjoint kernel alternates two;
//   * the accumulator (128 lanes x 64 columns of TMEM) is read back with
//     tcgen05.ld, each warp its 32 lanes, and stored to s or v.
// Operand layout: K-major, 128-byte swizzle (op_off), 1024-byte aligned tiles
// (checked at kernel entry: a CTA whose shared memory is not so aligned records
// an error and returns before touching the tensor cores).  Every wait is
// bounded: after about two seconds the CTA records an error code, finishes
// what it issued and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "pat_conv_tc.cuh"

namespace pat {

namespace {

constexpr int kM = kTcM, kN = kTcN, kKS = kTcKStage;
constexpr int kAHalf = kM * kKS * 2;           // bytes of one T stage (hi or lo)
constexpr int kBHalf = kN * kKS * 2;           // bytes of one B stage (hi or lo)
constexpr long long kSpinCycles = 4000000000LL; // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05 for a K-major operand in the
// 128-byte swizzle layout (see op_off): start address, leading byte offset
// (not used when the K extent is one 128-byte row; 16 B), stride byte offset
// 1024 (between groups of 8 rows), descriptor version 1 (bits 46-47),
// swizzle mode 2 = 128 B (bits 61-63).  A K step of 16 values inside the row
// advances the start address by 32 B; the swizzle is applied to the final
// address bits, so the tile must sit on a 1024-byte boundary.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Waits for the phase of `bar` with the given parity to complete; false after
// about two seconds.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        __nanosleep(64);
        if (clock64() - t0 > kSpinCycles) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One bulk copy global -> shared through the TMA engine, completing on bar.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
                 "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16])
{
    uint32_t u[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
                   "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]),
                   "=r"(u[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) r[j] = __uint_as_float(u[j]);
}

// Byte offset of element (row, kk), kk < kKS = 64, in a K-major operand tile
// in the 128-byte swizzle layout: each row holds its 64 BF16 values in 128
// bytes, rows go in groups of 8 (1024-byte atoms), and the 16-byte chunk c of
// row r is stored at chunk c ^ (r mod 8), so that the 8 rows of an atom read
// at the same K fall on different shared-memory banks.
__device__ __forceinline__ uint32_t op_off(int row, int kk)
{
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((kk >> 3) ^ row) & 7) << 4) + (kk & 7) * 2);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// B stage: rows n < kN (transducers k0 + n of src, row length len, row
// stride ld), columns kk < kKS (source index start + kk); zero outside the
// row and beyond K.  One 16-byte core-matrix row (8 values) per item; threads
// tid = 0 .. nthr - 1 share the items.
__device__ __forceinline__ void build_b(const float *__restrict__ src, long long ld, int len, int K, int k0, int start,
                                        uint8_t *bhi, uint8_t *blo, int tid, int nthr)
{
    for (int item = tid; item < kN * (kKS / 8); item += nthr) {
        const int n = item / (kKS / 8), q = item % (kKS / 8);
        const int k = k0 + n;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int m = start + q * 8 + e;
            v[e] = (k < K && m >= 0 && m < len) ? __ldg(&src[(long long)k * ld + m]) : 0.f;
        }
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * e]), h1 = __float2bfloat16_rn(v[2 * e + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * e] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * e + 1] - __bfloat162float(h1));
            h[e] = pack2(h0, h1);
            l[e] = pack2(l0, l1);
        }
        const uint32_t off = op_off(n, q * 8);
        *reinterpret_cast<uint4 *>(bhi + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(blo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// build_b for exactly kN (kKS / 8) / nthr items per thread, all loads issued
// before any conversion (memory-level parallelism: the loads of one stage are
// in flight together instead of one item at a time).
template <int kItems>
__device__ __forceinline__ void build_b_batched(const float *__restrict__ src, long long ld, int len, int K, int k0,
                                                int start, uint8_t *bhi, uint8_t *blo, int tid, int nthr)
{
    float v[kItems][8];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int item = tid + it * nthr;
        const int n = item / (kKS / 8), q = item % (kKS / 8);
        const int k = k0 + n;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int m = start + q * 8 + e;
            v[it][e] = (k < K && m >= 0 && m < len) ? __ldg(&src[(long long)k * ld + m]) : 0.f;
        }
    }
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int item = tid + it * nthr;
        const int n = item / (kKS / 8), q = item % (kKS / 8);
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(v[it][2 * e]), h1 = __float2bfloat16_rn(v[it][2 * e + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(v[it][2 * e] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(v[it][2 * e + 1] - __bfloat162float(h1));
            h[e] = pack2(h0, h1);
            l[e] = pack2(l0, l1);
        }
        const uint32_t off = op_off(n, q * 8);
        *reinterpret_cast<uint4 *>(bhi + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(blo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// Shared memory of one CTA: two A buffers (T hi + lo per stage), B buffers,
// mbarriers and the TMEM address slot.
struct TcSmem {
    uint8_t *a[2];  // kAHalf hi then kAHalf lo
    uint8_t *b;     // nb buffers of 2 kBHalf (hi, lo)
    uint32_t full[2], empty[2];
    uint32_t *tslot;
    int *abort_flag;
};

__device__ __forceinline__ TcSmem carve(uint8_t *base, int nb)
{
    TcSmem s;
    s.a[0] = base;
    s.a[1] = base + 2 * kAHalf;
    s.b = base + 4 * kAHalf;
    uint8_t *tail = s.b + (size_t)nb * 2 * kBHalf;
    uint64_t *bars = reinterpret_cast<uint64_t *>(tail);
    s.full[0] = smem_u32(&bars[0]);
    s.full[1] = smem_u32(&bars[1]);
    s.empty[0] = smem_u32(&bars[2]);
    s.empty[1] = smem_u32(&bars[3]);
    s.tslot = reinterpret_cast<uint32_t *>(&bars[4]);
    s.abort_flag = reinterpret_cast<int *>(&bars[5]);
    return s;
}

// barrier set-up and TMEM allocation (warp 0), kN FP32 columns
__device__ __forceinline__ uint32_t tc_setup(const TcSmem &S)
{
    if (threadIdx.x == 0) {
        mbar_init(S.full[0], 1);
        mbar_init(S.full[1], 1);
        mbar_init(S.empty[0], 1);
        mbar_init(S.empty[1], 1);
        *S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(S.tslot)),
                     "r"((uint32_t)kN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    return *S.tslot;
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem)
{
    fence_before();
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kN)
                     : "memory");
}

// Issues the 3 split products of one stage: K = kKS in kKS / 16 MMAs each.
__device__ __forceinline__ void issue_stage(uint32_t tmem, const uint8_t *a, const uint8_t *bhi, const uint8_t *blo,
                                            bool first)
{
    const uint32_t ahi = smem_u32(a), alo = smem_u32(a + kAHalf), bh = smem_u32(bhi), bl = smem_u32(blo);
#pragma unroll
    for (int ks = 0; ks < kKS / 16; ++ks) {
        const uint32_t o = ks * 32; // 16 BF16 values along K
        mma_bf16(tmem, sdesc(ahi + o), sdesc(bh + o), (first && ks == 0) ? 0u : 1u);
        mma_bf16(tmem, sdesc(ahi + o), sdesc(bl + o), 1u);
        mma_bf16(tmem, sdesc(alo + o), sdesc(bh + o), 1u);
    }
}

// Records a failed wait: the CTA stops issuing, drains and returns.
__device__ __forceinline__ void note_timeout(const TcSmem &S, int *err, int code)
{
    *S.abort_flag = 1;
    atomicExch(err, code);
}

// Issue state of the one thread that drives the TMA engine and the tensor
// cores (thread 0).  Stage q uses buffer q & 1; its copy completes phase
// q >> 1 of full[q & 1] and its MMAs (through tcgen05.commit) phase q >> 1 of
// empty[q & 1].
struct Pipe {
    int issued = 0, landed = 0, committed = 0;

    // T stage q into buffer q & 1, once the MMAs of stage q - 2 (the last
    // readers of that buffer) are done.
    __device__ __forceinline__ bool load(const TcSmem &S, const uint8_t *tab, int q)
    {
        const int b = q & 1;
        if (q >= 2 && !mbar_wait(S.empty[b], ((q - 2) >> 1) & 1)) return false;
        mbar_expect_tx(S.full[b], 2 * kAHalf);
        bulk_g2s(smem_u32(S.a[b]), tab + (size_t)q * 2 * kAHalf, 2 * kAHalf, S.full[b]);
        issued = q + 1;
        return true;
    }
    __device__ __forceinline__ bool mma(const TcSmem &S, uint32_t tmem, int q, const uint8_t *bhi, bool first)
    {
        const int b = q & 1;
        if (!mbar_wait(S.full[b], (q >> 1) & 1)) return false;
        landed = q + 1;
        fence_after();
        issue_stage(tmem, S.a[b], bhi, bhi + kBHalf, first);
        mma_commit(S.empty[b]);
        committed = q + 1;
        return true;
    }
    // after a timeout: bounded waits for every copy and MMA still in flight
    __device__ __forceinline__ void drain(const TcSmem &S) const
    {
        for (int q = landed; q < issued; ++q) mbar_wait(S.full[q & 1], (q >> 1) & 1);
        if (committed > 0) mbar_wait(S.empty[(committed - 1) & 1], ((committed - 1) >> 1) & 1);
    }
};

} // namespace

// ---------------------------------------------------------------------------
// Forward: grid (ceil(L / 128), ceil(K / 64), nsplit); Tf: nst stages of
// 2 kAHalf.  CTA z of a tile takes the stages [z nst / nsplit, (z+1) nst /
// nsplit) and adds its partial tile into s (zeroed by the launcher) when
// nsplit > 1.
//
// Pipeline: a ring of kRing slots, each holding one stage's T (hi, lo) and B
// (hi, lo).  Warp kIssuerWarp, lane 0, brings T into the slots by bulk copy
// kLookA stages ahead of the tensor cores and issues each stage's MMAs once
// its T and B have landed; kRing groups of four warps split B into the slots,
// group g for the stages of slot g, so that kRing stages load at once.  Slot
// q % kRing is reused by stage q once the MMAs of stage q - kRing have
// completed (tcgen05.commit on empty[slot]); T lands on fullA[slot]
// (transaction count), B on fullB[slot] (one arrival per warp of the group);
// a last commit on `done` releases the epilogue.  Every barrier is waited on
// in phase order by each of its waiters, so a parity test never meets a
// barrier two phases behind.  Every wait gives up after about two seconds or
// as soon as another thread has given up.
// ---------------------------------------------------------------------------
namespace {

constexpr int kRing = 4, kLookA = 2;
constexpr int kSlot = 2 * kAHalf + 2 * kBHalf;
// converter groups of four warps, one per ring slot: group g splits stages
// g, g + kRing, ..., so that the global loads of several stages are in
// flight at once, and each slot's empty barrier is waited on by one group, in
// order (a waiter never runs two phases ahead of a barrier, where the parity
// test would pass on the older phase)
constexpr int kConvGroups = kRing, kGroupWarps = 4;
constexpr int kConvWarps = kConvGroups * kGroupWarps, kIssuerWarp = kConvWarps;
static_assert(kTcThreadsFwd == 32 * (kConvWarps + 1), "forward block size");

struct Ring {
    uint8_t *slot[kRing];
    uint32_t fullA[kRing], fullB[kRing], empty[kRing];
    uint32_t done; // one phase: every MMA of the CTA has completed
    uint32_t *tslot;
    int *abort_flag;
};

__device__ __forceinline__ Ring carve_ring(uint8_t *base)
{
    Ring r;
    for (int i = 0; i < kRing; ++i) r.slot[i] = base + (size_t)i * kSlot;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + (size_t)kRing * kSlot);
    for (int i = 0; i < kRing; ++i) {
        r.fullA[i] = smem_u32(&bars[i]);
        r.fullB[i] = smem_u32(&bars[kRing + i]);
        r.empty[i] = smem_u32(&bars[2 * kRing + i]);
    }
    r.done = smem_u32(&bars[3 * kRing]);
    r.tslot = reinterpret_cast<uint32_t *>(&bars[3 * kRing + 1]);
    r.abort_flag = reinterpret_cast<int *>(&bars[3 * kRing + 2]);
    return r;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// mbar_wait that also gives up once another thread of the CTA has
__device__ __forceinline__ bool ring_wait(const Ring &R, uint32_t bar, uint32_t parity)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (*(volatile int *)R.abort_flag) return false;
        __nanosleep(32);
        if (clock64() - t0 > kSpinCycles) return false;
    }
    return true;
}

__device__ __forceinline__ void ring_abort(const Ring &R, int *err, int code)
{
    *(volatile int *)R.abort_flag = 1;
    atomicExch(err, code);
}

} // namespace

__global__ void __launch_bounds__(kTcThreadsFwd, 1)
    conv_tc_fwd_kernel(const float *__restrict__ f, const uint8_t *__restrict__ Tf, int nst, int m0off, int K, int L,
                       int UL, int U, float *__restrict__ s, int *__restrict__ err, float oscale)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    if (smem_u32(smem_raw) & 1023u) { // swizzled operand tiles need 1024-byte alignment
        if (threadIdx.x == 0) atomicExch(err, 6);
        return;
    }
    const Ring R = carve_ring(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kRing; ++i) {
            mbar_init(R.fullA[i], 1);
            mbar_init(R.fullB[i], kGroupWarps);
            mbar_init(R.empty[i], 1);
        }
        mbar_init(R.done, 1);
        *R.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(R.tslot)),
                     "r"((uint32_t)kN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *R.tslot;
    const int l0 = blockIdx.x * kM, k0 = blockIdx.y * kN;
    const int st0 = (int)((long long)blockIdx.z * nst / gridDim.z), st1 = (int)((long long)(blockIdx.z + 1) * nst / gridDim.z);
    const int n = st1 - st0;
    const long long m0 = (long long)U * l0 + m0off + (long long)st0 * kKS;

    if (warp == kIssuerWarp) {
        if (lane == 0) {
            int issued = 0, committed = 0; // T copies started, stages whose MMAs were committed
            bool ok = true;
            auto load_a = [&](int q) -> bool {
                const int b = q % kRing;
                if (q >= kRing && !ring_wait(R, R.empty[b], ((q / kRing) - 1) & 1)) return false;
                mbar_expect_tx(R.fullA[b], 2 * kAHalf);
                bulk_g2s(smem_u32(R.slot[b]), Tf + (size_t)(st0 + q) * 2 * kAHalf, 2 * kAHalf, R.fullA[b]);
                issued = q + 1;
                return true;
            };
            for (int q = 0; q < kLookA && q < n && ok; ++q) ok = load_a(q);
            for (int q = 0; q < n && ok; ++q) {
                if (q + kLookA < n && !load_a(q + kLookA)) {
                    ok = false;
                    break;
                }
                const int b = q % kRing;
                if (!ring_wait(R, R.fullA[b], (q / kRing) & 1) || !ring_wait(R, R.fullB[b], (q / kRing) & 1)) {
                    ok = false;
                    break;
                }
                fence_after();
                issue_stage(tmem, R.slot[b], R.slot[b] + 2 * kAHalf, R.slot[b] + 2 * kAHalf + kBHalf, q == 0);
                mma_commit(R.empty[b]);
                committed = q + 1;
            }
            if (ok) mma_commit(R.done); // after the last stage: all of this thread's MMAs
            if (!ok) {
                ring_abort(R, err, 4);
                // bounded waits for the copies and MMAs still in flight
                for (int q = committed; q < issued; ++q) mbar_wait(R.fullA[q % kRing], (q / kRing) & 1);
                if (committed > 0) mbar_wait(R.empty[(committed - 1) % kRing], ((committed - 1) / kRing) & 1);
            }
        }
    } else {
        // converters: B of every stage into its slot.  Lane 0 of each warp
        // waits and the warp follows its verdict, so that every decision (and
        // the warp-collective tcgen05.ld below) is warp-uniform.
        const int grp = warp / kGroupWarps, tid = threadIdx.x - grp * 32 * kGroupWarps;
        for (int q = grp; q < n; q += kConvGroups) {
            const int b = q % kRing;
            int okw = 1;
            if (q >= kRing) {
                if (lane == 0) okw = ring_wait(R, R.empty[b], ((q / kRing) - 1) & 1) ? 1 : 0;
                okw = __shfl_sync(0xffffffffu, okw, 0);
            }
            if (!okw) {
                if (lane == 0) ring_abort(R, err, 2);
                break;
            }
            uint8_t *bh = R.slot[b] + 2 * kAHalf;
            static_assert(kN * (kKS / 8) % (32 * kGroupWarps) == 0, "items per converter thread");
            build_b_batched<kN * (kKS / 8) / (32 * kGroupWarps)>(f, UL, UL, K, k0, (int)(m0 + (long long)q * kKS), bh,
                                                                  bh + kBHalf, tid, 32 * kGroupWarps);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(R.fullB[b]);
        }
        // epilogue (warps 0-3, one per 32 TMEM lanes): wait for all MMAs
        int ok = 0;
        if (lane == 0 && warp < 4) {
            ok = *(volatile int *)R.abort_flag ? 0 : 1;
            if (ok && !ring_wait(R, R.done, 0)) {
                ring_abort(R, err, 5);
                ok = 0;
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        fence_after();
        if (ok) {
            const int l = l0 + warp * 32 + lane;
            const bool split = gridDim.z > 1;
#pragma unroll 1
            for (int c = 0; c < kN; c += 16) {
                float r[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
                if (l < L) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int k = k0 + c + j;
                        if (k < K) {
                            if (split) atomicAdd(&s[(long long)k * L + l], r[j] * oscale);
                            else s[(long long)k * L + l] = r[j] * oscale;
                        }
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kN)
                     : "memory");
}

// ---------------------------------------------------------------------------
// Adjoint: grid (ceil(L / 128), ceil(K / 64)); Ta: U phases x nst stages of
// 2 kAHalf.  B (the s window, nst stages) is built once and reused by every
// phase; T stages stream through two buffers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads) conv_tc_adj_kernel(const float *__restrict__ s, const uint8_t *__restrict__ Ta,
                                                                 int nst, int d0, int K, int L, int UL, int U,
                                                                 float *__restrict__ v, int *__restrict__ err,
                                                                 float oscale)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    if (smem_u32(smem_raw) & 1023u) { // swizzled operand tiles need 1024-byte alignment
        if (threadIdx.x == 0) atomicExch(err, 6);
        return;
    }
    const TcSmem S = carve(smem_raw, nst);
    const uint32_t tmem = tc_setup(S);
    const int m0 = blockIdx.x * kM, k0 = blockIdx.y * kN;
    Pipe pipe;
    if (threadIdx.x == 0 && !pipe.load(S, Ta, 0)) note_timeout(S, err, 1);
    for (int st = 0; st < nst; ++st) {
        uint8_t *bhi = S.b + (size_t)st * 2 * kBHalf;
        build_b(s, L, L, K, k0, m0 + d0 + st * kKS, bhi, bhi + kBHalf, threadIdx.x, blockDim.x);
    }
    fence_proxy_async();
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = m0 + warp * 32 + lane;
    const int total = U * nst; // (phase, stage) pairs in order
    bool ok = true;
    for (int g = 0; g < total; ++g) {
        const int p = g / nst, st = g % nst;
        if (threadIdx.x == 0 && !*S.abort_flag) {
            if (g + 1 < total && !pipe.load(S, Ta, g + 1)) note_timeout(S, err, 3);
            else if (!pipe.mma(S, tmem, g, S.b + (size_t)st * 2 * kBHalf, st == 0)) note_timeout(S, err, 4);
        }
        if (st != nst - 1) continue;
        // phase p is complete once its last commit lands: read it out
        __syncthreads();
        if (*S.abort_flag) {
            ok = false;
            break;
        }
        if (!mbar_wait(S.empty[g & 1], (g >> 1) & 1)) {
            atomicExch(err, 5);
            *S.abort_flag = 1;
        }
        __syncthreads();
        if (*S.abort_flag) {
            ok = false;
            break;
        }
        fence_after();
#pragma unroll 1
        for (int c = 0; c < kN; c += 16) {
            float r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
            if (m < L) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int k = k0 + c + j;
                    if (k < K) v[(long long)k * UL + (long long)U * m + p] = r[j] * oscale;
                }
            }
        }
        // every lane's reads of this phase finish before the next phase's
        // first MMA overwrites the accumulator
        fence_before();
        __syncthreads();
        fence_after();
    }
    if (!ok && threadIdx.x == 0) pipe.drain(S);
    tc_teardown(tmem);
}

// ---------------------------------------------------------------------------
// Forward from split planes: s from f given as two BF16 planes (hi, lo) of
// [K][ld] elements (ld a multiple of 8), persistent CTAs, one per SM.
//
// Tile: 128 output samples x 256 transducers (M 128, N 256: one MMA keeps
// the tensor cores at their full rate, where N = 64 ran them at about a
// third).  Stage: 64 fine bins of the window, T (hi, lo) from the table by
// one bulk copy and B (hi, lo) by two tensor-map copies (TMA) that land in
// the 128-byte swizzle layout of the operand descriptor, so no thread
// touches f: the kernel is a copy engine feeding the tensor cores.  The
// window of output tile l0 starts at U l0 + m0a with m0a = m0off - shift a
// multiple of 8 (the table's leading `shift` columns are zero), so every
// tensor-map x coordinate is a multiple of 8 BF16 elements (16 bytes); the
// coordinates outside [0, U L) and the rows beyond K read the copy engine's
// zero fill.  A CTA takes tiles blockIdx.x, + gridDim.x, ..., output tiles
// fastest, and odd output tiles take their stages in reverse order (the
// tensor cores add the same products in the other order): the window halos
// of neighbouring tiles are then read twice within a short time, the second
// time from L2 (in forward order the second read came about 70 % of a tile
// later and went back to DRAM: 1.37 GB read for 1.04 GB of planes).
//
// Warp roles: warp 0 (lane 0) issues the copies into a ring of two stage
// slots; warp 1 (lane 0) issues 3 x 4 MMAs per stage into one of two TMEM
// accumulators of 256 columns, alternating between tiles, and commits each
// stage onto the slot's `empty` barrier and each tile onto the accumulator's
// `tfull`; warps 2-5 read a finished accumulator (each warp the TMEM lanes
// of its rank within the warp group), store the tile into s and arrive on
// `tempty`, so that the MMAs of the next tile overlap the store.  Every wait
// is bounded (about 2 s, or as soon as another thread has given up); a
// thread that gives up records an error, waits (bounded) for what it issued
// and leaves.  withhold != 0 (a test of that path, one CTA): the epilogue
// does not release the first accumulator, so the MMA warp's wait for it at
// the third tile runs out.
// ---------------------------------------------------------------------------
namespace {

constexpr int kN2 = kTcN2, kRing2 = 2;
constexpr int kB2Half = kN2 * kKS * 2;            // bytes of one B plane stage
constexpr int kSlot2 = 2 * kAHalf + 2 * kB2Half; // T hi, T lo, B hi, B lo
constexpr uint32_t kIdesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN2 >> 3) << 17) |
                             ((uint32_t)(kM >> 4) << 24);
static_assert(kTcThreadsFwd2 == 192, "copy warp, MMA warp, four epilogue warps");

__device__ __forceinline__ void mma_bf16_n256(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
                 "l"(a), "l"(b), "r"(kIdesc2), "r"(accumulate)
                 : "memory");
}

// 2-D tensor-map copy of one box into shared memory, completing on bar.
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                 "[%4];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}

struct Fwd2 {
    uint8_t *slot[kRing2];
    uint32_t full[kRing2], empty[kRing2], tfull[2], tempty[2];
    uint32_t *tslot;
    int *abort_flag;
};

__device__ __forceinline__ Fwd2 carve_fwd2(uint8_t *base)
{
    Fwd2 r;
    for (int i = 0; i < kRing2; ++i) r.slot[i] = base + (size_t)i * kSlot2;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + (size_t)kRing2 * kSlot2);
    for (int i = 0; i < kRing2; ++i) {
        r.full[i] = smem_u32(&bars[i]);
        r.empty[i] = smem_u32(&bars[kRing2 + i]);
    }
    for (int i = 0; i < 2; ++i) {
        r.tfull[i] = smem_u32(&bars[2 * kRing2 + i]);
        r.tempty[i] = smem_u32(&bars[2 * kRing2 + 2 + i]);
    }
    r.tslot = reinterpret_cast<uint32_t *>(&bars[2 * kRing2 + 4]);
    r.abort_flag = reinterpret_cast<int *>(&bars[2 * kRing2 + 5]);
    return r;
}

__device__ __forceinline__ bool fwd2_wait(const Fwd2 &R, uint32_t bar, uint32_t parity)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (*(volatile int *)R.abort_flag) return false;
        __nanosleep(32);
        if (clock64() - t0 > kSpinCycles) return false;
    }
    return true;
}

__device__ __forceinline__ void fwd2_abort(const Fwd2 &R, int *err, int code)
{
    *(volatile int *)R.abort_flag = 1;
    atomicExch(err, code);
}

} // namespace

__global__ void __launch_bounds__(kTcThreadsFwd2, 1)
    conv_tc_fwd2_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                        const uint8_t *__restrict__ Tf, int nst, int m0a, int K, int L, int U,
                        float *__restrict__ s, int *__restrict__ err, int withhold, float oscale)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    if (smem_u32(smem_raw) & 1023u) { // swizzled operand tiles need 1024-byte alignment
        if (threadIdx.x == 0) atomicExch(err, 6);
        return;
    }
    const Fwd2 R = carve_fwd2(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kRing2; ++i) {
            mbar_init(R.full[i], 1);
            mbar_init(R.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(R.tfull[i], 1);
            mbar_init(R.tempty[i], 4);
        }
        *R.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) { // two accumulators of kN2 FP32 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(R.tslot)),
                     "r"((uint32_t)(2 * kN2))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *R.tslot;
    const int nlt = (L + kM - 1) / kM, nkt = (K + kN2 - 1) / kN2, ntiles = nlt * nkt;

    if (warp == 0) {
        if (lane == 0) {
            // copies: stage g of this CTA into slot g % 2 once the MMAs of stage g - 2 are done
            int g = 0;
            bool ok = (m0a & 7) == 0;
            if (!ok) fwd2_abort(R, err, 7);
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int l0 = (t % nlt) * kM, k0 = (t / nlt) * kN2;
                const int x0 = U * l0 + m0a;
                // neighbouring output tiles share the last / first (nW - 1) / 64
                // stages of their windows; odd tiles walk theirs backwards, so
                // both read a shared stretch at about the same time and the
                // second read finds it in L2
                const bool back = ((t % nlt) & 1) != 0;
                for (int it = 0; it < nst; ++it, ++g) {
                    const int st = back ? nst - 1 - it : it;
                    const int b = g & 1;
                    if (g >= kRing2 && !fwd2_wait(R, R.empty[b], ((g >> 1) - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    uint8_t *sl = R.slot[b];
                    mbar_expect_tx(R.full[b], (uint32_t)kSlot2);
                    bulk_g2s(smem_u32(sl), Tf + (size_t)st * 2 * kAHalf, 2 * kAHalf, R.full[b]);
                    tma_2d(smem_u32(sl + 2 * kAHalf), &map_hi, x0 + st * kKS, k0, R.full[b]);
                    tma_2d(smem_u32(sl + 2 * kAHalf + kB2Half), &map_lo, x0 + st * kKS, k0, R.full[b]);
                }
            }
            if (!ok) {
                fwd2_abort(R, err, 8);
                // bounded waits for the copies still in flight: at most the last
                // two stages, each its slot's latest phase
                for (int q = g > kRing2 ? g - kRing2 : 0; q < g; ++q) mbar_wait(R.full[q & 1], (q >> 1) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int g = 0, ti = 0, last_commit = -1;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++ti) {
                const int a = ti & 1;
                if (ti >= 2 && !fwd2_wait(R, R.tempty[a], ((ti >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                const uint32_t td = tmem + (uint32_t)(a * kN2);
                for (int st = 0; st < nst; ++st, ++g) {
                    const int b = g & 1;
                    if (!fwd2_wait(R, R.full[b], (g >> 1) & 1)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint8_t *sl = R.slot[b];
                    const uint32_t ahi = smem_u32(sl), alo = ahi + kAHalf, bh = ahi + 2 * kAHalf, bl = bh + kB2Half;
#pragma unroll
                    for (int ks = 0; ks < kKS / 16; ++ks) {
                        const uint32_t o = ks * 32;
                        mma_bf16_n256(td, sdesc(ahi + o), sdesc(bh + o), (st == 0 && ks == 0) ? 0u : 1u);
                        mma_bf16_n256(td, sdesc(ahi + o), sdesc(bl + o), 1u);
                        mma_bf16_n256(td, sdesc(alo + o), sdesc(bh + o), 1u);
                    }
                    mma_commit(R.empty[b]);
                    last_commit = g;
                }
                if (ok) mma_commit(R.tfull[a]);
            }
            if (!ok) {
                fwd2_abort(R, err, 9);
                if (last_commit >= 0) mbar_wait(R.empty[last_commit & 1], (last_commit >> 1) & 1);
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (output samples)
        const int q4 = warp & 3;
        int ti = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++ti) {
            const int a = ti & 1;
            int ok = 0;
            if (lane == 0) ok = fwd2_wait(R, R.tfull[a], (ti >> 1) & 1) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) fwd2_abort(R, err, 10);
                break;
            }
            fence_after();
            const int l0 = (t % nlt) * kM, k0 = (t / nlt) * kN2;
            const int l = l0 + q4 * 32 + lane;
#pragma unroll 1
            for (int c = 0; c < kN2; c += 16) {
                float r[16];
                tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(a * kN2 + c), r);
                if (l < L) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int k = k0 + c + j;
                        if (k < K) s[(long long)k * L + l] = r[j] * oscale;
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0 && !(withhold && ti == 0)) mbar_arrive(R.tempty[a]);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * kN2))
                     : "memory");
}

// f [K][UL] floats -> hi, lo planes [K][ld] (the split of build_b; the
// padding columns are zero).
__global__ void split_bf16_kernel(const float *__restrict__ f, int K, int UL, int ld, uint16_t *__restrict__ hi,
                                  uint16_t *__restrict__ lo)
{
    const long long n = (long long)K * ld;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / ld), m = (int)(e % ld);
        const float v = m < UL ? f[(long long)k * UL + m] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        hi[e] = __bfloat16_as_ushort(h);
        lo[e] = __bfloat16_as_ushort(l);
    }
}

// ---------------------------------------------------------------------------
// Operand tables (plan set-up, FP64 taps -> BF16 hi / lo in the operand layout)
// ---------------------------------------------------------------------------
// W[j] = (1/U) sum_{u<U} h-bar[j - (U-1) + u] in FP64
__device__ double w64(const double *__restrict__ taps, int T, int U, int j)
{
    if (j < 0 || j >= T + U - 1) return 0.0;
    double acc = 0.0;
    for (int u = 0; u < U; ++u) {
        const int t = j - (U - 1) + u;
        if (t >= 0 && t < T) acc += taps[t];
    }
    return acc / U;
}

__device__ __forceinline__ void put_split(uint8_t *stage, int row, int kk, double w)
{
    const __nv_bfloat16 hi = __float2bfloat16_rn((float)w);
    const __nv_bfloat16 lo = __float2bfloat16_rn((float)(w - (double)__bfloat162float(hi)));
    const uint32_t off = op_off(row, kk);
    *reinterpret_cast<__nv_bfloat16 *>(stage + off) = hi;
    *reinterpret_cast<__nv_bfloat16 *>(stage + kAHalf + off) = lo;
}

// Tf[st]: element (i, kk) = W[U i + nW - 1 - (st kKS + kk - shift)] (zero for
// the shift's leading columns: a window that starts shift bins early)
__global__ void tc_table_fwd_kernel(const double *__restrict__ taps, int T, int U, int nst, int shift, double sc,
                                    uint8_t *__restrict__ Tf)
{
    const long long n = (long long)nst * kM * kKS;
    const int nW = T + U - 1;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int st = (int)(e / (kM * kKS)), r = (int)(e % (kM * kKS)), i = r / kKS, kk = r % kKS;
        const int mu = st * kKS + kk - shift;
        put_split(Tf + (size_t)st * 2 * kAHalf, i, kk, w64(taps, T, U, U * i + nW - 1 - mu) * sc);
    }
}

// Ta[p][st]: element (i, kk) = W[U (d0 + lambda - i) + c - p], lambda = st kKS + kk
__global__ void tc_table_adj_kernel(const double *__restrict__ taps, int T, int U, int nst, int d0, int c, double sc,
                                    uint8_t *__restrict__ Ta)
{
    const long long n = (long long)U * nst * kM * kKS;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long g = e / (kM * kKS);
        const int r = (int)(e % (kM * kKS)), i = r / kKS, kk = r % kKS;
        const int p = (int)(g / nst), st = (int)(g % nst);
        const int lam = st * kKS + kk;
        put_split(Ta + (size_t)g * 2 * kAHalf, i, kk, w64(taps, T, U, U * (d0 + lam - i) + c - p) * sc);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
TcGeometry tc_geometry(int T, int U, int L, int n_lo)
{
    TcGeometry g;
    const int nW = T + U - 1, c = U - 1 - n_lo;
    g.m0off = c - (nW - 1);
    const int kw = (kM - 1) * U + nW; // forward window length
    g.nst_fwd = (kw + kKS - 1) / kKS;
    // adjoint: d over all phases with 0 <= U d + c - p < nW
    int dmin = 1 << 30, dmax = -(1 << 30);
    for (int p = 0; p < U; ++p)
        for (int j = 0; j < nW; ++j)
            if ((j - c + p) % U == 0) { // U d = j - c + p
                const int d = (j - c + p) / U;
                dmin = d < dmin ? d : dmin;
                dmax = d > dmax ? d : dmax;
            }
    g.d0 = dmin;
    const int ka = dmax - dmin + kM;
    g.nst_adj = (ka + kKS - 1) / kKS;
    g.c = c;
    g.fwd_table_bytes = (size_t)g.nst_fwd * 2 * kAHalf;
    g.adj_table_bytes = (size_t)U * g.nst_adj * 2 * kAHalf;
    g.fwd_smem = (size_t)kRing * kSlot + 3 * kRing * 8 + 24;
    int dev = 0;
    g.sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&g.sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        g.sms = 1;
    g.adj_smem = 4 * kAHalf + (size_t)g.nst_adj * 2 * kBHalf + 64;
    // split-plane forward: window start shifted down to a multiple of 8 fine bins
    g.shift = ((g.m0off % 8) + 8) % 8;
    g.m0a = g.m0off - g.shift;
    g.nst_fwd2 = (kw + g.shift + kKS - 1) / kKS;
    g.fwd2_table_bytes = (size_t)g.nst_fwd2 * 2 * kAHalf;
    g.fwd2_smem = (size_t)kRing2 * kSlot2 + 8 * (2 * kRing2 + 6) + 1024;
    g.ld = (U * L + 7) / 8 * 8;
    g.tscale = 0;
    return g;
}

cudaError_t launch_tc_tables(const double *taps, int T, int U, const TcGeometry &g, uint8_t *Tf, uint8_t *Ta,
                             uint8_t *Tf2, cudaStream_t st)
{
    const double sc = ldexp(1.0, g.tscale); // exact
    tc_table_fwd_kernel<<<304, 256, 0, st>>>(taps, T, U, g.nst_fwd, 0, sc, Tf);
    tc_table_adj_kernel<<<608, 256, 0, st>>>(taps, T, U, g.nst_adj, g.d0, g.c, sc, Ta);
    tc_table_fwd_kernel<<<304, 256, 0, st>>>(taps, T, U, g.nst_fwd2, g.shift, sc, Tf2);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled from the driver, looked up once (the library links
// the runtime statically and not the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        looked = true;
    }
    return fn;
}

// Tensor map of one BF16 plane [K][ld]: boxes of 64 fine bins (128 bytes, the
// swizzle span) x 256 rows, 128-byte swizzle, zero fill outside.
static cudaError_t plane_map(CUtensorMap *m, const uint16_t *plane, int K, int UL, int ld)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    if (((uintptr_t)plane & 15) != 0 || (ld % 8) != 0 || UL > ld) return cudaErrorInvalidValue;
    // extent U L: the row padding [U L, ld) reads as zero fill, like every column outside
    const cuuint64_t dims[2] = {(cuuint64_t)UL, (cuuint64_t)K};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kKS, (cuuint32_t)kN2};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)plane, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_split_bf16(const float *f, int K, int UL, int ld, uint16_t *hi, uint16_t *lo, cudaStream_t st)
{
    split_bf16_kernel<<<1216, 256, 0, st>>>(f, K, UL, ld, hi, lo);
    return cudaGetLastError();
}

cudaError_t launch_conv_tc_fwd2(const uint16_t *hi, const uint16_t *lo, const uint8_t *Tf2, const TcGeometry &g, int K,
                                int L, int U, float *s, int *err, cudaStream_t st, bool withhold)
{
    CUtensorMap mh, ml;
    cudaError_t e = plane_map(&mh, hi, K, U * L, g.ld);
    if (e == cudaSuccess) e = plane_map(&ml, lo, K, U * L, g.ld);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute((const void *)conv_tc_fwd2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)g.fwd2_smem);
    if (e != cudaSuccess) return e;
    const int ntiles = ((L + kM - 1) / kM) * ((K + kN2 - 1) / kN2);
    if (withhold && ntiles < 3) return cudaErrorInvalidValue; // the withheld release is waited for at the third tile
    const unsigned grid = withhold ? 1u : (unsigned)std::max(1, std::min(ntiles, g.sms));
    conv_tc_fwd2_kernel<<<grid, kTcThreadsFwd2, g.fwd2_smem, st>>>(mh, ml, Tf2, g.nst_fwd2, g.m0a, K, L, U, s, err,
                                                                     withhold ? 1 : 0, ldexpf(1.f, -g.tscale));
    return cudaGetLastError();
}

cudaError_t launch_conv_tc_fwd(const float *f, const uint8_t *Tf, const TcGeometry &g, int K, int L, int U, float *s,
                               int *err, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute((const void *)conv_tc_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)g.fwd_smem);
    if (e != cudaSuccess) return e;
    const unsigned gx = (unsigned)((L + kM - 1) / kM), gy = (unsigned)((K + kN - 1) / kN);
    // split the stages when the tiles alone leave SMs idle (one CTA per SM)
    int nsplit = std::max(1, std::min(std::min(4, g.nst_fwd), g.sms / (int)(gx * gy)));
    if (nsplit > 1) {
        e = cudaMemsetAsync(s, 0, sizeof(float) * (size_t)K * L, st);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(gx, gy, (unsigned)nsplit);
    conv_tc_fwd_kernel<<<grid, kTcThreadsFwd, g.fwd_smem, st>>>(f, Tf, g.nst_fwd, g.m0off, K, L, U * L, U, s, err,
                                                                ldexpf(1.f, -g.tscale));
    return cudaGetLastError();
}

cudaError_t launch_conv_tc_adj(const float *s, const uint8_t *Ta, const TcGeometry &g, int K, int L, int U, float *v,
                               int *err, cudaStream_t st, bool unscale)
{
    cudaError_t e = cudaFuncSetAttribute((const void *)conv_tc_adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)g.adj_smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((L + kM - 1) / kM), (unsigned)((K + kN - 1) / kN));
    conv_tc_adj_kernel<<<grid, kTcThreads, g.adj_smem, st>>>(s, Ta, g.nst_adj, g.d0, K, L, U * L, U, v, err,
                                                             unscale ? ldexpf(1.f, -g.tscale) : 1.f);
    return cudaGetLastError();
}

} // namespace pat
