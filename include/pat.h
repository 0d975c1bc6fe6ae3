/*
 * pat.h -- C ABI of the GB300 (sm_103a) library for the matrix-free
 * photoacoustic operator A and its adjoint A^T (surface method with closed
 * form areas, and point-detector method), after Do, Escande, Chaux, Gateau and
 * Lee, "Scalable photoacoustic tomography implementations accounting for the
 * spatial impulse response of transducers".
 *
 * Conventions shared by every entry point
 *   - SI units.  Voxel i = (iz * ny + iy) * nx + ix sits at
 *     origin + pitch * (ix, iy, iz) (Sec. 2.4, flattened index).
 *   - Fine time bins b in [0, U L) are [tau_b, tau_{b+1}) with
 *     tau_b = t0 + b / (U Fs); the paper's l is b + 1 (Sec. 3.1).
 *   - Device buffers are borrowed: the caller allocates them (any allocator,
 *     e.g. PyTorch), keeps them alive until the work queued on `stream` has
 *     finished, and must not alias an output with an input.  The library
 *     allocates device memory only inside pat_plan_create (plan constants)
 *     and frees it in pat_plan_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Compute entry points only enqueue work; they do not
 *     synchronise.  An asynchronous kernel fault surfaces as PAT_ERR_CUDA on a
 *     later call.
 *   - Every entry point returns a pat_status and never throws;
 *     pat_last_error() returns a thread-local message for the last failure.
 *   - Calls on different plans may run concurrently; calls on one plan from
 *     several host threads must be serialised by the caller.
 */
#ifndef PAT_H
#define PAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pat_status {
    PAT_OK = 0,
    PAT_ERR_INVALID_ARG = 1, /* null pointer, bad size or unknown enum */
    PAT_ERR_GEOMETRY = 2,    /* separation violated: dist_min < kappa (Ass. 1(iii)) or c/(U Fs) > dist_min (Prop. 3) */
    PAT_ERR_WINDOW = 3,      /* some pair's bins leave [0, U L) and PAT_FLAG_ALLOW_CLIP is not set */
    PAT_ERR_WORKSPACE = 4,   /* workspace pointer null or smaller than pat_workspace_bytes() */
    PAT_ERR_CUDA = 5,        /* a CUDA call or kernel launch failed */
    PAT_ERR_UNSUPPORTED = 6  /* valid request this build does not implement (e.g. shared memory too small) */
} pat_status;

enum { PAT_PLANE = 0, PAT_CYLINDER = 1 };
/* PAT_METHOD_TRAPEZOID: the surface method with the paper's trapezoidal
 * approximation of the cylinder's arc integral (Eq. trapezoid_Il: the level
 * curve between its two ends replaced by its chord); planes keep their
 * closed form.  An approximation of PAT_METHOD_SURFACE, cheaper per area.
 * PAT_METHOD_LUT: the surface method with the cylinder's arc integral in the
 * elliptic closed form of Eq. (cyl_Il), E read from the paper's lookup tables
 * (Sec. 4.2.2): E~(s, m) = E(arcsin s, m) and F~(s, m) = F(arcsin s, m) on the
 * power-law grid of Eq. (LUT_sampling) with eps = 1e-16, q1 nodes in s and q2
 * in m, bilinear interpolation, the reciprocal-modulus transformation of
 * Eq. (reciprocal_modulus) for nu > 1.  The tables (one 40-byte record per
 * grid cell, about 40 q1 q2 bytes of device memory, plus the float-float node
 * arrays) are built at plan creation from FP64 node values; the arc integral
 * is evaluated in float-float arithmetic (about 48 significant bits) on the
 * FP32 units.  Planes keep their closed form. */
enum { PAT_METHOD_SURFACE = 0, PAT_METHOD_POINT = 1, PAT_METHOD_TRAPEZOID = 2, PAT_METHOD_LUT = 3 };
enum { PAT_RBF_BUMP = 0, PAT_RBF_CONE = 1, PAT_RBF_WENDLAND = 2 };
enum { PAT_EIR_GAUSS_SINE = 0, PAT_EIR_BOX = 1 };
/* Plan flags (pat_params.flags, OR-ed):
 *   PAT_FLAG_ALLOW_CLIP  drop fine bins outside [0, U L) instead of failing
 *                        plan creation;
 *   PAT_FLAG_CONV_TC     run the temporal convolution (Eq. discrete_conv) and
 *                        its transpose (App. G) as Toeplitz contractions on the
 *                        tcgen05 tensor cores: BF16 operands split in two
 *                        (hi + lo), hi*hi + hi*lo + lo*hi accumulated in FP32.
 *                        Areas and accumulation of f stay FP32 / FP64; the
 *                        convolution then carries about 16 significant bits
 *                        per product instead of FP64 accumulation.  The
 *                        operand tables hold the taps times a power of two
 *                        (the largest in [1, 2)), undone exactly on the
 *                        outputs, so that no product nears FP32's smallest
 *                        normal for taps of SI size (about 1e-20);
 *   PAT_FLAG_PIECEWISE_PLANES  the paper's Piecewise-Planes approximation
 *                        (Sec. 4.3): every cylindrical element is replaced by
 *                        np_planes planes tangent at the centres of equal
 *                        angular sectors (half-width R dtheta / 2, half-height
 *                        Lz), whose geometric signals add into the element's
 *                        row (Eq. plane_decomp_u); planar elements are kept.
 *                        pat_plan_info counts pairs and windows per plane. */
enum { PAT_FLAG_ALLOW_CLIP = 1, PAT_FLAG_CONV_TC = 2, PAT_FLAG_PIECEWISE_PLANES = 4 };
enum { PAT_OP_FORWARD = 1, PAT_OP_ADJOINT = 2, PAT_OP_RECON = 3, PAT_OP_FORWARD_DC = 4, PAT_OP_AUTOTUNE = 5,
       PAT_OP_CONV_SPLIT = 6 };

/* Uniform voxel grid (Sec. 2.4): centres origin + pitch * (ix, iy, iz). */
typedef struct pat_grid {
    int32_t n[3]; /* nx, ny, nz, each >= 1 */
    int32_t reserved;
    double origin[3];
    double pitch; /* > 0 */
} pat_grid;

/* One transducer position, 16 doubles (the row layout of the Python side).
 *   plane    (Eq. plane_param):    c0 + x1 e1 + x2 e2, |x1| <= L1, |x2| <= L2;
 *   cylinder (Eq. cylinder_param): c0 + R cos(t) e2 + R sin(t) (e1 x e2) + z e1,
 *            |t| <= theta_max < pi/2, |z| <= Lz, c0 on the focal line,
 *            e1 the cylinder axis.
 * e1 and e2 must be orthonormal.  kind is PAT_PLANE or PAT_CYLINDER stored as
 * a double. */
typedef struct pat_transducer {
    double kind;
    double c0[3], e1[3], e2[3];
    double L1, L2;
    double R, theta_max, Lz;
    double reserved;
} pat_transducer;

/* Time axis and discretisation.  Recording samples l in [0, L) cover
 * [t0 + l/Fs, t0 + (l+1)/Fs) (Eq. def_operatorS); U is the upsampling factor,
 * dl the area step of Remark 1 (1 <= dl <= U; dl = 1 is Alg. 3 exactly).
 * Groups of dl fine bins start at each pair's first bin l_min of
 * Eq. (rmin_rmax); the last group stops at l_max and its area is split over
 * its actual length.  method: PAT_METHOD_SURFACE (Alg. 3 + Alg. 4),
 * PAT_METHOD_POINT (Alg. 2 with a q1 x q2 midpoint quadrature of each
 * element, Prop. 2), PAT_METHOD_TRAPEZOID, or PAT_METHOD_LUT (q1 x q2 table
 * nodes in s and m, each 2 .. 8192; the paper takes 1000 x 1000).  flags: PAT_FLAG_ALLOW_CLIP drops fine bins outside
 * [0, U L) instead of failing plan creation. */
typedef struct pat_params {
    double c;  /* speed of sound, > 0 */
    double fs; /* sampling frequency, > 0 */
    double t0; /* recording origin, >= 0 */
    int32_t L, U, dl, method, q1, q2, flags;
    int32_t np_planes; /* PAT_FLAG_PIECEWISE_PLANES: planes per cylindrical element, 1..4096 (else ignored) */
} pat_params;

/* Radial function and electrical impulse response that define the system
 * kernel h = e * g with g(t) = -1/2 c t phi(|c t|) (Prop. 1).
 *   rbf_kind: PAT_RBF_BUMP (1 - r^2/k^2)^2, PAT_RBF_CONE 1 - r/k,
 *             PAT_RBF_WENDLAND (1 - r/k)^2, all on r < kappa;
 *   eir_kind: PAT_EIR_GAUSS_SINE exp(-(t-tc)^2/(2 s^2)) sin(2 pi fc (t-tc)) on
 *             [0, Te], eir = {fc, s, tc, Te};  PAT_EIR_BOX eir[0] on [0, Te],
 *             eir = {amplitude, -, -, Te}. */
typedef struct pat_system {
    int32_t rbf_kind, eir_kind;
    double kappa;
    double eir[4];
} pat_system;

typedef struct pat_plan pat_plan;

typedef struct pat_plan_info {
    int64_t N, K, L, U, UL, dl, method;
    int64_t n_taps, n_lo;
    int64_t bin_lo, bin_hi;   /* extreme fine bins over all pairs (Eq. rmin_rmax) */
    int64_t area_evals;       /* per application: sum over pairs of ceil(bins / dl) (surface), N K q1 q2 (point) */
    int64_t pair_bins;        /* sum over pairs of l_max - l_min + 1 */
    int64_t quad_evals;       /* surface method: sum over pairs of groups x non-degenerate quadrants */
    int64_t clipped_pairs;    /* pairs with bins outside [0, U L) */
    int64_t conv_clipped;     /* transducers whose filtered response leaves [0, U L) (dropped by definition) */
    double dist_min;          /* min over pairs of the distance to the element (Eq. min_dist) */
    int64_t fwd_blocks, adj_blocks; /* CTAs of one forward / adjoint geometric launch */
    int64_t tc_error;         /* PAT_FLAG_CONV_TC plans: non-zero if a tensor-core CTA gave up waiting on the
                                 TMA engine or the tensor cores (its output tile is then left unwritten);
                                 reading it synchronises with the plan's device */
} pat_plan_info;

/* Discrete system kernel (Eq. def_bh):
 *   h-bar[n] = U Fs int_0^D int_0^D h(t - t' + n D) dt dt',  D = 1/(U Fs),
 * for n = n_lo .. n_lo + n_taps - 1, computed on the device in FP64 by
 * composite Gauss-Legendre quadrature split at every kink of e and g.
 * taps_dev: device array of n_taps doubles (caller-owned, overwritten).
 * Errors: PAT_ERR_INVALID_ARG for null pointers, n_taps < 1, U < 1, bad kinds
 * or non-positive c, fs, kappa, Te. */
pat_status pat_system_kernel(const pat_system *sys, double c, double fs, int32_t U, int32_t n_lo, int32_t n_taps,
                             double *taps_dev, void *stream);

/* Derivative of the discrete system kernel with respect to the speed of
 * sound, d h-bar[n] / dc for the same n as pat_system_kernel (Eq. def_bh with
 * g(t) = -1/2 c t phi(|c t|) replaced by dg/dc = -1/2 t [phi + r phi'](|c t|);
 * the triangle window D = 1/(U Fs) does not depend on c).  Same arguments,
 * quadrature and errors as pat_system_kernel. */
pat_status pat_system_kernel_dc(const pat_system *sys, double c, double fs, int32_t U, int32_t n_lo, int32_t n_taps,
                                double *dtaps_dev, void *stream);

/* Creates a plan: copies the grid, the K transducer descriptors (host array
 * tx[K]) and the taps (host array taps_host[n_taps], h-bar[n_lo + t]) to the
 * device, derives the per-element frames, and scans every voxel-transducer
 * pair once on the device to find the bin window, the separation dist_min and
 * the work per application.  kappa is the support radius of the radial
 * function (Ass. 1).  Synchronises `stream`.  Host arrays are not retained.
 * Errors: PAT_ERR_INVALID_ARG (null, K < 1, sizes, kinds, dl not in [1, U],
 * q1/q2 < 1 for the point method, frame not orthonormal, theta_max not in
 * (0, pi/2)); PAT_ERR_GEOMETRY (separation, Ass. 1(iii) and Prop. 3);
 * PAT_ERR_WINDOW (bins outside [0, U L) without PAT_FLAG_ALLOW_CLIP);
 * PAT_ERR_UNSUPPORTED (a forward chunk's bins too many for the shared-memory
 * window, a pair whose bins the forward kernel's FP32 window bound would miss,
 * or a tap window too wide for the tensor-core convolution's shared memory);
 * PAT_ERR_CUDA.  *out is NULL on failure. */
pat_status pat_plan_create(pat_plan **out, const pat_grid *grid, const pat_transducer *tx, int32_t K,
                           const pat_params *params, double kappa, const double *taps_host, int32_t n_taps,
                           int32_t n_lo, void *stream);

/* Frees the plan's device memory (after synchronising the device). NULL is a no-op. */
pat_status pat_plan_destroy(pat_plan *plan);

/* Plan facts (see pat_plan_info). */
pat_status pat_plan_get_info(const pat_plan *plan, pat_plan_info *info);

/* Workspace bytes needed by op (PAT_OP_FORWARD, PAT_OP_ADJOINT, PAT_OP_RECON,
 * PAT_OP_FORWARD_DC, PAT_OP_AUTOTUNE; PAT_OP_CONV_SPLIT: the planes of
 * pat_conv_split); 0 for a null plan or unknown op. */
size_t pat_workspace_bytes(const pat_plan *plan, int32_t op);

/* s = A x (Alg. 1): x device float[N], s device float[K][L] (overwritten).
 * Geometric assembly (Alg. 3 / Alg. 2) then convolution with h-bar and
 * downsampling by U (Eq. discrete_conv).  ws: device workspace of at least
 * pat_workspace_bytes(plan, PAT_OP_FORWARD) bytes, 256-byte aligned. */
pat_status pat_forward(pat_plan *plan, const float *x, float *s, void *ws, size_t ws_bytes, void *stream);

/* z = A^T s (Alg. 5): s device float[K][L], z device float[N] (overwritten).
 * Upsampling transpose, correlation with h-bar^-, then the gather of
 * Alg. 7 / Alg. 6 (App. G).  ws as for pat_forward with PAT_OP_ADJOINT. */
pat_status pat_adjoint(pat_plan *plan, const float *s, float *z, void *ws, size_t ws_bytes, void *stream);

/* Stages, for testing and for callers that keep f: */
/* f = [K][U L] geometric signals (Eq. ui_area with Remark 1 / Eq. def_f_point), overwritten. */
pat_status pat_forward_geometric(pat_plan *plan, const float *x, float *f, void *ws, size_t ws_bytes, void *stream);
/* s[K][L] = downsample_U(h-bar * f) (Eq. discrete_conv) from f[K][U L]. */
pat_status pat_conv_forward(pat_plan *plan, const float *f, float *s, void *stream);
/* v[K][U L] = h-bar^- * upsample_U^T(s) (App. G) from s[K][L]. */
pat_status pat_conv_adjoint(pat_plan *plan, const float *s, float *v, void *stream);
/* Tensor-core plans (PAT_FLAG_CONV_TC) only, else PAT_ERR_UNSUPPORTED: the
 * convolution of Eq. (discrete_conv) from f in the split form pat_forward
 * uses inside.  pat_conv_split writes f[K][U L] (device floats) as two BF16
 * planes, hi = bf16(f) then lo = bf16(f - hi), each [K][ld] with ld = U L
 * rounded up to a multiple of 8, into planes (device uint16, 16-byte
 * aligned, pat_workspace_bytes(plan, PAT_OP_CONV_SPLIT) bytes; the padding
 * columns are zero).  pat_conv_forward_split computes s[K][L] (device
 * floats, overwritten) from such planes with the persistent tensor-map /
 * tcgen05 kernel (only the first U L columns of each row are read).  Both
 * are asynchronous on stream; a wait that gave up on the device shows in
 * pat_plan_info.tc_error. */
pat_status pat_conv_split(pat_plan *plan, const float *f, uint16_t *planes, void *stream);
pat_status pat_conv_forward_split(pat_plan *plan, const uint16_t *planes, float *s, void *stream);
/* Test of the tensor-core kernels' give-up path, with no fault and no endless
 * wait: pat_conv_forward_split's kernel on one CTA, its epilogue withholding
 * the release of the first TMEM accumulator, so that the bounded wait for it
 * (about two seconds) runs out at the third output tile.  The kernel then
 * stops every warp, waits (bounded) for the copies and MMAs it issued,
 * frees its TMEM and leaves; pat_plan_info.tc_error becomes non-zero and s
 * is undefined.  Needs a plan with at least 3 output tiles
 * (ceil(L / 128) ceil(K / 256) >= 3; else PAT_ERR_INVALID_ARG).
 * pat_plan_clear_tc_error resets tc_error to 0 (asynchronous on stream). */
pat_status pat_conv_forward_split_withheld(pat_plan *plan, const uint16_t *planes, float *s, void *stream);
pat_status pat_plan_clear_tc_error(pat_plan *plan, void *stream);
/* z[N] = transpose of the geometric assembly applied to v[K][U L] (Alg. 7 / Alg. 6). */
pat_status pat_adjoint_geometric(pat_plan *plan, const float *v, float *z, void *ws, size_t ws_bytes, void *stream);

/* ds = d(A x)/dc, the derivative of the forward operator with respect to the
 * speed of sound c at the plan's c, for a fixed x (surface method).  c enters
 * through the bin radii r = c tau (the swept areas: d|M|/dc = tau_e A'(r_e)
 * at the two radii of a bin or group, with A' = dA/dr of Sec. 4), through the
 * weights U Fs / (c tau) (Eq. ui_area) and through h-bar (dtaps, from
 * pat_system_kernel_dc for the plan's tap window, device doubles[n_taps]).
 * The bins of every pair stay those of the plan (the derivative of the
 * piecewise-smooth operator between bin changes).  x: device float[N];
 * ds: device float[K][L] (overwritten); ws: pat_workspace_bytes(plan,
 * PAT_OP_FORWARD_DC) bytes.  PAT_ERR_UNSUPPORTED for the point method or when
 * the doubled shared-memory windows do not fit. */
pat_status pat_forward_dc(pat_plan *plan, const float *x, const double *dtaps, float *ds, void *ws, size_t ws_bytes,
                          void *stream);

/* Projected FISTA for the Tikhonov non-negative least squares problem of
 * Eq. (nnls_tik):  min_{p >= 0} 1/2 |A p - s|^2 + 1/2 lambda_R |p|^2.
 * s device float[K][L]; x device float[N]: initial guess in, solution out.
 * step <= 0 estimates 1 / |A^T A + lambda_R| by 20 power iterations.
 * ws: pat_workspace_bytes(plan, PAT_OP_RECON) bytes.  Enqueues 2 operator
 * applications per iteration; synchronises `stream` only for the step
 * estimate.  The FISTA scalars live on the device, so every iteration is the
 * same launch sequence: on a capturable stream (not the legacy default
 * stream, not one the caller is capturing) with iters >= 2 it is captured
 * once into a CUDA graph and the graph is launched iters times; otherwise the
 * launches are enqueued directly (same arithmetic). */
pat_status pat_recon(pat_plan *plan, const float *s, float *x, int32_t iters, float lambda_R, float step, void *ws,
                     size_t ws_bytes, void *stream);

/* pat_recon for nprob independent problems of any sizes (one plan each,
 * distinct plans): arrays of nprob plans, measurements s[i], solutions x[i]
 * (initial guesses in), lambda_R[i], step[i] (NULL or <= 0: estimated per
 * problem), workspaces ws[i] of ws_bytes[i] >= pat_workspace_bytes(plans[i],
 * PAT_OP_RECON).  On a capturable stream one iteration of every problem is
 * captured into one CUDA graph, each problem on its own branch (fork and join
 * on internal streams), so small problems overlap on the GPU; the graph is
 * launched iters times.  Results equal those of pat_recon per problem.
 * Synchronises `stream` for the step estimates only. */
pat_status pat_recon_batch(pat_plan *const *plans, int32_t nprob, const float *const *s, float *const *x,
                           int32_t iters, const float *lambda_R, const float *step, void *const *ws,
                           const size_t *ws_bytes, void *stream);

/* Autotuner of the launch shapes of one plan: times the forward geometric
 * kernel with b0, b0/2 and b0/4 voxel bricks per CTA (b0 the plan's default,
 * a power of two up to one 8 x 8 x 8-brick super-tile; finer runs are never
 * below one brick per warp) and the adjoint gather with 2, 4 and 8 voxel
 * bricks per CTA, each three times (the first run discarded) on x (device
 * float[N]) and ws (pat_workspace_bytes(plan, PAT_OP_AUTOTUNE) bytes,
 * contents overwritten), and keeps the fastest pair for later calls
 * (pat_plan_info fwd_blocks and adj_blocks report it).  Costs about 9
 * operator halves; synchronises `stream`, which must not be under capture.
 * Results of later calls differ from the untuned ones only by the order of
 * floating-point additions. */
pat_status pat_plan_autotune(pat_plan *plan, const float *x, void *ws, size_t ws_bytes, void *stream);

/* s = A x like pat_forward, for callers that cannot allocate device memory
 * (for example code running where cudaMalloc is forbidden or unavailable,
 * such as inside a host callback or a plug-in that must not touch the
 * allocator).  There is no counterpart in the paper: it is a deployment
 * variant of pat_forward.  The forward workspace comes from a fixed scratch
 * array of PAT_STATIC_SCRATCH_BYTES (16 MiB) that the library places in
 * device memory at module load; every GPU that loads the library keeps it
 * until the process exits.  Plans whose pat_workspace_bytes(plan,
 * PAT_OP_FORWARD) exceeds that size are rejected with PAT_ERR_WORKSPACE.
 * The first call on each device looks the array up (cudaGetSymbolAddress
 * with that device current); make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents (each
 * call clears what must start at zero), so calls that overlap on the GPU
 * (different streams, or different host threads) race: serialise them.  The
 * call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine. */
#define PAT_STATIC_SCRATCH_BYTES (16u << 20)
pat_status pat_forward_static(pat_plan *plan, const float *x, float *s, void *stream);

/* Arithmetic peaks of the current device, measured by dependent-chain
 * kernels (8 independent chains per thread, 8 CTAs of 256 threads per SM,
 * one warm-up launch then one timed launch each, about 10 ms per figure),
 * in operations per second: FP32 fused multiply-add (2 flops each), the same
 * on packed register pairs (__ffma2_rn, 4 flops per instruction), FP64 fused
 * multiply-add, and rsqrtf on the special-function unit (1 op each).  The
 * figures are those of the clocks at the time of the call.  Runs on `stream`
 * and synchronises with it; allocates and frees a small device buffer.
 * PAT_ERR_INVALID_ARG for a null out, PAT_ERR_CUDA on any CUDA failure. */
typedef struct pat_peaks {
    double fp32_ffma_flops, fp32_ffma2_flops, fp64_dfma_flops, sfu_rsqrt_ops;
} pat_peaks;
pat_status pat_measure_peaks(pat_peaks *out, void *stream);

/* Thread-local description of the last failure ("" if none). */
const char *pat_last_error(void);

/* Library version, e.g. 100 for 0.1.0. */
int32_t pat_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PAT_H */
