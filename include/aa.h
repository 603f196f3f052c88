/*
 * aa.h -- C ABI of the GB300 (sm_103a) low-synchronization Anderson
 * acceleration library (libaa).
 *
 * Method: Anderson acceleration (Algorithm 1 of Lockhart et al., arXiv
 * 2110.09667) whose least-squares problem (Algorithm 2) is solved through a
 * QR factorization of the residual-difference history F_i that is updated
 * in place each iteration: QRDelete drops the oldest column by Givens
 * rotations, QRAdd appends Delta f_{i-1} with one of four orthogonalization
 * schemes -- MGS (Algorithm 3), ICWY (Algorithm 4), CGS-2 (Algorithm 5),
 * DCGS-2 (Algorithm 6).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are device pointers (cudaMalloc / torch CUDA
 *    tensors) on the current device, 16-byte aligned, holding n contiguous
 *    FP64 values unless stated otherwise.  *_host pointers are host memory.
 *  - All device work is enqueued on the context's stream (aa_config.stream,
 *    a cudaStream_t; NULL means the legacy default stream).  Calls return
 *    after enqueueing, except where a host output is requested: those
 *    synchronize the stream before returning.
 *  - Return value: 0 (AA_OK) on success, 1 (AA_NOTCONVERGED) from aa_solve
 *    when max_iters is reached, a negative AA_E* code on error.  No C++
 *    exception crosses the ABI.  aa_last_error() gives a message.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - After a call returns an error that the device reported (AA_ETIMEOUT,
 *    AA_ENONFINITE) the history is undefined: aa_step, aa_qradd and aa_lsq
 *    return AA_ESTATE until aa_reset (aa_solve resets by itself).
 *  - The caller owns x, G(x), f and user data; the context owns the history
 *    (Q, R, T, dG, f_{i-1}, G(x_{i-1})) and its reduction scratch.
 */
#ifndef AA_H_
#define AA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define AA_OK 0
#define AA_NOTCONVERGED 1
#define AA_EINVAL (-1)     /* bad argument (size, alignment, enum, NULL) */
#define AA_ENOMEM (-2)     /* device or host allocation failed */
#define AA_ECUDA (-3)      /* a CUDA runtime call failed */
#define AA_EBREAKDOWN (-4) /* QRAdd: new column numerically in span(Q); history cleared */
#define AA_ENONFINITE (-5) /* NaN/Inf in a residual or norm */
#define AA_ETIMEOUT (-6)   /* a bounded device-side wait ran out */
#define AA_ECALLBACK (-7)  /* the user's G callback returned non-zero */
#define AA_ESTATE (-8)     /* call not valid in the context's current state */

/* Orthogonalization scheme used by QRAdd (Sec. 3 of the paper). */
typedef enum { AA_MGS = 0, AA_ICWY = 1, AA_CGS2 = 2, AA_DCGS2 = 3 } aa_orth;

/* Storage type of the history Q and dG.  Dot products, norms, R, T and
 * gamma stay FP64 in every case; x, G(x), f and Delta f stay FP64. */
typedef enum { AA_STORE_FP64 = 0, AA_STORE_FP32 = 1, AA_STORE_BF16 = 2 } aa_storage;

/* Flags (aa_config.flags). */
#define AA_FLAG_DCGS2_SCALED 0x1u  /* DCGS-2: R_{0:k-2,k-1} += R_{k-1,k-1} s instead of += s */
#define AA_FLAG_ICWY_GRAM 0x2u     /* ICWY: after a delete, refresh T from a Gram reduction of
                                      the rotated Q (fused into the first pass, k <= 24) instead
                                      of rotating T at the m x m level */
#define AA_FLAG_TIMING 0x4u        /* record CUDA events around every pass (aa_pass_times) */
#define AA_FLAG_FP32_DOTS 0x8u     /* FP64 storage: the dot products of the first pass of each
                                      QR update (and of the CGS-2 middle pass), when there are
                                      more than four, run on the FP32 pipe: exact products of
                                      (hi, lo) float splits of the FP64 operands (each scaled by
                                      a power of two, 2^-48 relative), compensated float-pair
                                      sums over 64 rows per lane, folded into FP64.  Squared
                                      norms of f and Delta f stay FP64 (they carry the NaN/Inf
                                      test); Q, v, x, R, T and gamma stay FP64.  The scale of f
                                      and Delta f is taken from the previous ||f|| (aa_step) or
                                      ||Delta f|| (aa_qradd): a vector more than about 2^90
                                      smaller or 2^47 larger than that loses its smallest or
                                      overflows its cross products.  No counterpart in the
                                      paper. */
#define AA_FLAG_DF_ARITH 0x10u     /* FP64 storage: the first pass of each QR update (QRDelete
                                      rotation, first block of dot products) on the FP32/INT
                                      pipes in (hi, lo) float arithmetic, about 2^-48 relative
                                      per operation instead of 2^-53; the differences f, df, dg,
                                      the projection and the update stay FP64, and so do Q, dG,
                                      x in memory and R, T, gamma.  Not with AA_FLAG_FP32_DOTS
                                      or FP32/BF16 storage (AA_EINVAL).  No counterpart in the
                                      paper. */

typedef struct aa_config {
  int64_t n;          /* vector length, >= 1 */
  int32_t m;          /* history depth, 1..64 */
  int32_t orth;       /* aa_orth */
  int32_t storage;    /* aa_storage */
  int32_t max_iters;  /* aa_solve: iteration cap (>= 0) */
  double tol;         /* aa_solve: stop when ||G(x_i) - x_i||_2 / scale < tol (stop_kind 0)
                         or ||x_{i+1} - x_i||_2 < tol (stop_kind 1, Algorithm 1 as printed) */
  double scale;       /* > 0; typically ||b||_2 */
  int32_t stop_kind;  /* 0 or 1 */
  int32_t dcgs2_min_mi; /* DCGS-2 reorthogonalises when m_i > this; the paper uses 3 */
  double breakdown_tol; /* breakdown when rho <= breakdown_tol * ||Delta f||; default 1e-14 when 0 */
  uint64_t flags;     /* AA_FLAG_* */
  void *stream;       /* cudaStream_t */
} aa_config;

/* Fills cfg with defaults: m=5, MGS, FP64, max_iters=100, tol=1e-8, scale=1,
 * stop_kind=0, dcgs2_min_mi=3, breakdown_tol=1e-14, flags=0, stream=NULL. */
void aa_config_default(aa_config *cfg, int64_t n);

typedef struct aa_ctx aa_ctx;

/* Per-context counters, cumulative since aa_create / aa_reset. */
typedef struct aa_stats {
  int64_t iters;          /* aa_solve: iterations taken (x_0 is iterate 0) */
  int64_t steps;          /* aa_step calls */
  int64_t reductions;     /* grid-wide reduction passes (the paper's "syncs") */
  int64_t launches;       /* kernels launched by the library */
  int64_t breakdowns;     /* history restarts */
  double fnorm;           /* ||f_i||_2 of the last step */
  double g_ms, aa_ms;     /* aa_solve: time in G and in the AA passes (CUDA events) */
} aa_stats;

/* Create a context: allocates and zeroes the history on the current device.
 * Errors: AA_EINVAL (n < 1, m outside 1..64, bad enum), AA_ENOMEM, AA_ECUDA. */
int aa_create(const aa_config *cfg, aa_ctx **out);

/* Destroy a context (synchronizes its stream, frees all device memory).  NULL is ignored. */
void aa_destroy(aa_ctx *ctx);

/* Forget the history (Algorithm 1 restarts at iteration 0); also clears the
 * reset-required state left by a device-reported error. */
int aa_reset(aa_ctx *ctx);

/* Test hook (no counterpart in the paper): writes `code` (0 or a negative
 * AA_E* value) into the context's device status word on its stream, as a
 * pass that failed on the device would, so that host-side error handling
 * can be exercised without a device fault.  The next call that reads the
 * status (aa_step, aa_qradd, aa_lsq) returns it.  Synchronizes. */
int aa_test_set_device_status(aa_ctx *ctx, int code);

/* Replace the stream used by later calls. */
int aa_set_stream(aa_ctx *ctx, void *stream);

/* Algorithm 2, QR part, as a unit: if the factorization already holds m
 * columns, QRDelete removes the oldest (Givens rotations); then QRAdd
 * appends v_dev with the configured scheme.  v_dev (n FP64) is only read.
 * Returns AA_EBREAKDOWN (history cleared) when the new column's norm is
 * <= breakdown_tol * ||v||.  Synchronizes the stream. */
int aa_qradd(aa_ctx *ctx, const double *v_dev);

/* Algorithm 2, last step: gamma_host[0..k-1] solves R gamma = Q^T f_dev for
 * the k columns held.  Returns k (>= 0) or a negative error.  Synchronizes. */
int aa_lsq(aa_ctx *ctx, const double *f_dev, double *gamma_host);

/* One iteration of Algorithm 1 given x_i (x_dev) and G(x_i) (gx_dev): forms
 * f_i, Delta f_{i-1}, Delta g_{i-1}, updates the QR factorization and the dG
 * history, solves the least-squares problem and writes
 * x_{i+1} = G(x_i) - dG_i gamma into xnext_dev (which must not alias x_dev
 * or gx_dev).  The first call after create/reset writes x_1 = G(x_0).
 * *fnorm_host (if not NULL) receives ||f_i||_2; then the stream is
 * synchronized.  AA_EBREAKDOWN is not returned: a breakdown clears the
 * history and the step falls back to x_{i+1} = G(x_i) (counted in stats). */
int aa_step(aa_ctx *ctx, const double *x_dev, const double *gx_dev, double *xnext_dev,
            double *fnorm_host);

/* User fixed-point map: enqueue gx_dev = G(x_dev) on `stream` and return 0;
 * any non-zero return aborts aa_solve with AA_ECALLBACK. */
typedef int (*aa_g_fn)(const double *x_dev, double *gx_dev, int64_t n, void *stream, void *user);

/* Algorithm 1 to convergence: x_dev holds x_0 on entry and the returned
 * iterate on exit.  Returns AA_OK, AA_NOTCONVERGED, or an error. */
int aa_solve(aa_ctx *ctx, aa_g_fn G, void *user, double *x_dev, aa_stats *stats);

/* Current factorization for inspection: Q_host (n x k, column-major, may be
 * NULL), R_host (k x k row-major, may be NULL), T_host (ICWY's unit-lower
 * T, k x k row-major, may be NULL); *k receives the column count. Synchronizes. */
int aa_get_qr(aa_ctx *ctx, double *Q_host, double *R_host, double *T_host, int *k);

/* Counters since create/reset. */
int aa_get_stats(const aa_ctx *ctx, aa_stats *out);

/* Per-pass device time (AA_FLAG_TIMING): ms_out[kind] and count_out[kind]
 * accumulate, for each pass kind (0 init, 1 first pass, 2 projection,
 * 3 CGS-2 middle pass, 4 MGS link, 5 update, 6 lsq, 7 mdot), the CUDA-event
 * time measured on the context's stream and the number of launches since
 * create/reset.  Both arrays hold 8 entries. */
int aa_pass_times(const aa_ctx *ctx, double *ms_out, int64_t *count_out);

/* Multi-column dot product with a deterministic two-stage grid reduction
 * (the fused multi-dot of Sec. 4): out_host[j*nv + v] = sum_i A_j[i] * V_v[i]
 * for the k columns A_j = A_dev + j*lda and nv vectors V_v = V_dev + v*ldv
 * (all FP64, columns 16-byte aligned, k*nv <= 256, lda, ldv >= n).  The
 * result is bit-identical from run to run.  Allocates its reduction scratch
 * (grid x k*nv doubles) with cudaMalloc on every call.  Synchronizes.
 * Returns AA_ETIMEOUT (and NaN products) if a bounded device wait ran out. */
int aa_mdot(const double *A_dev, int64_t lda, int k, const double *V_dev, int64_t ldv, int nv,
            int64_t n, double *out_host, void *stream);

/* Allocation-free variant of aa_mdot.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory --
 * frameworks whose own pool owns all device memory, processes running close
 * to the device's memory limit, and latency-critical loops in which
 * cudaMalloc/cudaFree would synchronize the device.  It computes the same
 * products as aa_mdot with the same deterministic reduction, but its
 * reduction scratch is a file-scope device array of about 0.76 MB (the
 * reduction state plus 304 x 256 partial sums) that every GPU which loads
 * the library holds until the process exits; it calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *  - Sizes: same limits as aa_mdot (k*nv <= 256, k + nv <= 70, lda, ldv >= n,
 *    columns 16-byte aligned); larger requests return AA_EINVAL.
 *  - Output: out_dev (device, k*nv FP64, out_dev[j*nv + v]) is written on
 *    `stream`; the call does not synchronize.  Since it returns before the
 *    kernel ends, a bounded device wait that ran out cannot be returned as
 *    a status: it shows as NaN in every product.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture.  The address is cached per device and
 *    looked up again when the device's current context has changed (after
 *    cudaDeviceReset, for example).
 *  - Every call shares the one array and leaves its contents behind; the
 *    call clears what must start at zero itself.  Calls whose work overlaps
 *    on the GPU (for example on two streams) race on the array: serialize
 *    them. */
int aa_mdot_noalloc(const double *A_dev, int64_t lda, int k, const double *V_dev, int64_t ldv,
                    int nv, int64_t n, double *out_dev, void *stream);

/* Copies `bytes` bytes from src to dst on `stream` (asynchronous).  No
 * counterpart in the paper: it moves iterates between page-locked host
 * memory and the device for callers that keep x on the host.  Either side
 * may be device memory or host memory from cudaHostAlloc/cudaHostRegister;
 * when the device can address both (cudaPointerGetAttributes reports a
 * device address) and both are 16-byte aligned, a kernel on every SM does
 * the copy with 16-byte loads and stores (over this part's NVLink-C2C host
 * link, faster than the copy engines); otherwise cudaMemcpyAsync does it.
 * Errors: AA_EINVAL (NULL pointer), AA_ECUDA. */
int aa_copy(void *dst, const void *src, size_t bytes, void *stream);
/* 1 if aa_copy(dst, src, ...) takes the kernel path (the device addresses
 * both sides, 16-byte aligned), 0 if it hands the copy to cudaMemcpyAsync. */
int aa_copy_path(const void *dst, const void *src);

/* ---------------------------------------------------------- test problems
 * Built-in fixed-point maps (aa_g_fn-compatible) for the seeded stencil
 * workloads.  `user` points to the matching parameter struct; b/src are
 * device pointers. */
typedef struct aa_jacobi2d {  /* 2D 5-point anisotropic Jacobi: G = x + D^{-1}(b - A x) */
  int64_t nx, ny; double eps; const double *b_dev;
} aa_jacobi2d;
typedef struct aa_jacobi3d {  /* 3D 7-point weighted Jacobi: G = x + omega D^{-1}(b - A x) */
  int64_t nx, ny, nz; double ey, ez, omega; const double *b_dev;
} aa_jacobi3d;
typedef struct aa_bratu2d {   /* nonlinear Jacobi for -Lap u = lambda e^u + src, h = 1/(s+1) */
  int64_t s; double lambda; const double *src_dev; /* src may be NULL */
} aa_bratu2d;

int aa_g_jacobi2d(const double *x_dev, double *gx_dev, int64_t n, void *stream, void *user);
int aa_g_jacobi3d(const double *x_dev, double *gx_dev, int64_t n, void *stream, void *user);
int aa_g_bratu2d(const double *x_dev, double *gx_dev, int64_t n, void *stream, void *user);

/* ------------------------------------------------------------ batched form
 * Many independent AA(m) solves of the 2D Bratu nonlinear-Jacobi map
 * (Sec. 5.2), u <- (sum of neighbours + h^2 (lambda e^u + src)) / 4 on
 * s x s grids, h = 1/(s+1), zero boundary, in ONE persistent kernel launch
 * (captured in a CUDA graph): each CTA pops the next solve from a queue
 * (largest first) and runs the whole Anderson loop with ICWY QR updates
 * (Algorithm 4) and block-level reductions.  Q and dG are stored in FP32,
 * x/G(x)/f in FP64, R, T and gamma in FP64.  Stop: ||G(x_i) - x_i||_2 /
 * ||G(0)||_2 < tol, or max_iters. */
typedef struct aa_batch_desc {
  int32_t count;          /* number of solves, >= 1 */
  const int64_t *side;    /* host, count entries: grid side s_i (n_i = s_i^2), 1..46340 */
  const double *lambda;   /* host, count entries */
  const double *src_host; /* host, sum n_i values (solve i's block in input order), or NULL */
  int32_t m;              /* history depth 1..16 */
  double tol;             /* default 1e-8 when <= 0 */
  int32_t max_iters;      /* default 100000 when <= 0 */
  int32_t block, ctas_per_sm;  /* launch shape hints (aa_batch_solve takes them explicitly) */
} aa_batch_desc;

typedef struct aa_batch aa_batch;

/* Allocates the arena (about 120 bytes per unknown for m = 10) and uploads
 * the per-solve parameters.  AA_EINVAL / AA_ENOMEM. */
int aa_batch_create(const aa_batch_desc *desc, aa_batch **out);
void aa_batch_destroy(aa_batch *b);
/* Optional initial guesses (host, sum n_i values in input order); NULL
 * returns to x_0 = 0.  A solve whose ||G(x_0) - x_0|| is not below
 * ||G(0)|| restarts from x_0 = 0 (reported per solve). */
int aa_batch_set_x0(aa_batch *b, const double *x0_host);
/* Runs every solve: one persistent launch of `block` threads (128, 256 or
 * 512) x ctas_per_sm (1..4) CTAs per SM on `stream`; *ms_out (if not NULL)
 * receives its CUDA-event time.  Synchronizes. */
int aa_batch_solve(aa_batch *b, int block, int ctas_per_sm, void *stream, double *ms_out);
/* Per-solve iterations, final ||f||/||G(0)|| and status (0 converged, 1 cap
 * reached, AA_ENONFINITE) in input order; any pointer may be NULL. */
int aa_batch_results(aa_batch *b, int32_t *iters, double *resid, int32_t *status);
/* Per-solve flag (input order): 1 if the x_0 given by aa_batch_set_x0 was
 * rejected by the residual test and the solve restarted from x_0 = 0. */
int aa_batch_fallbacks(aa_batch *b, int32_t *fallback);
/* Per-solve start and stop times of the last aa_batch_solve (input order),
 * in ms from the earliest start, read from the device's global timer: the
 * completion profile of the persistent launch (load balance, tail).  Either
 * pointer may be NULL, not both.  No counterpart in the paper. */
int aa_batch_times(aa_batch *b, double *start_ms, double *end_ms);
/* Solution of solve idx (host, n_idx doubles). */
int aa_batch_solution(aa_batch *b, int idx, double *x_host);
/* Total arena rows (sum of n_i rounded up to 64 each). */
int64_t aa_batch_rows(const aa_batch *b);
/* Change the iteration cap of later aa_batch_solve calls. */
int aa_batch_set_max_iters(aa_batch *b, int max_iters);

/* e^u for n device doubles computed on the FP32 pipe (the exponential the
 * batched Bratu map uses): Tang's table-driven method (reduction by ln2/128,
 * a 128-entry table of 2^(j/128) and a degree-5 polynomial) in (hi, lo)
 * float arithmetic, relative error at most about 3 |u| 2^-48 + 2^-45 for
 * |u| < 86.  out_dev may equal u_dev. */
int aa_exp_fp32pipe(int64_t n, const double *u_dev, double *out_dev, void *stream);

/* ------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper): the kernels that train
 * and run the MLP mapping a parametric problem's parameters to an initial
 * guess x_0.  All pointers are device pointers, all matrices row-major with
 * the given leading dimensions (elements); every call is asynchronous on
 * `stream` and returns AA_EINVAL for bad sizes, null or misaligned pointers
 * and AA_ECUDA for a launch failure.
 * ---------------------------------------------------------------------- */

/* C = A B^T on the tensor cores: A [M x K] and B [N x K] BF16 (K, lda, ldb
 * multiples of 8, A and B 16-byte aligned), FP32 accumulation.  epi bits:
 * 1 add bias[N] (fp32), 2 GELU, 4 store C as BF16 (else FP32), 8 also store
 * the pre-GELU value to pre (fp32, leading dimension ldp), 16 add to the
 * FP32 C already in place (not with 4). */
int aa_gemm_bf16_nt(int M, int N, int K, const void *A, int lda, const void *B, int ldb, void *C,
                    int ldc, const float *bias, float *pre, int ldp, int epi, void *stream);
/* The same product on the fifth-generation tensor cores: tcgen05.mma with
 * the FP32 accumulator in tensor memory, operands brought into shared memory
 * by the tensor-memory accelerator (128-byte swizzle), one 128 x 256 (or
 * 128 x 128) tile of C per CTA.  Same arguments, layout rules and epi bits as
 * aa_gemm_bf16_nt, and ldc >= N (ldp >= N with epi bit 8).  Rows of C are
 * the same sums in another order: results agree with aa_gemm_bf16_nt to the
 * FP32 accumulation bound.  Every device-side wait is bounded (one second);
 * a CTA that gives up writes NaN over its tile and is reported by
 * aa_gemm_tc_status. */
int aa_gemm_bf16_nt_tc(int M, int N, int K, const void *A, int lda, const void *B, int ldb, void *C,
                       int ldc, const float *bias, float *pre, int ldp, int epi, void *stream);
/* Synchronises `stream`; AA_ETIMEOUT (and the record cleared) if a CTA of an
 * aa_gemm_bf16_nt_tc launch gave up a bounded wait since the last call,
 * else AA_OK. */
int aa_gemm_tc_status(void *stream);
/* out[c][r] = in[r][c] for a [rows x cols] BF16 matrix. */
int aa_transpose_bf16(int rows, int cols, const void *in, int ldi, void *out, int ldo,
                      void *stream);
/* grad[i] *= GELU'(pre[i]) in place (grad BF16, pre FP32, n elements). */
int aa_gelu_bwd(int64_t n, const float *pre, void *grad, void *stream);
/* Mean-squared error of y against t (n FP32 each): dy = 2 (y - t) * scale
 * (BF16) and the per-block sums of (y - t)^2 in block_loss[nblocks] (FP64,
 * summed by the caller in block order). */
int aa_mse(int64_t n, const float *y, const float *t, float scale, void *dy, double *block_loss,
           int nblocks, void *stream);
/* out[c] = sum over r of g[r][c] (BF16 in, FP32 out): bias gradients. */
int aa_colsum_bf16(int rows, int cols, const void *g, int ld, float *out, void *stream);
/* Adam step (Kingma and Ba 2015) on n FP32 master weights w with moments
 * m, v and gradient g; refreshes the BF16 copy w_bf16 when not NULL.
 * step counts from 1 (bias corrections). */
int aa_adam(int64_t n, float *w, void *w_bf16, const float *g, float *m, float *v, float lr,
            float beta1, float beta2, float eps, int step, float weight_decay, void *stream);
/* Momentum SGD on n FP32 master weights: mom = momentum mom + g + wd w,
 * w -= lr mom; refreshes w_hi = bf16(w) and w_lo = bf16(w - w_hi) when not
 * NULL (the split copy carries about 16 significant bits). */
int aa_sgd(int64_t n, float *w, void *w_hi, void *w_lo, const float *g, float *mom, float lr,
           float momentum, float weight_decay, void *stream);
/* y = bf16(x) for n values. */
int aa_f32_to_bf16(int64_t n, const float *x, void *y, void *stream);
/* hi = bf16(x), lo = bf16(x - hi) for n values. */
int aa_f32_split_bf16(int64_t n, const float *x, void *hi, void *lo, void *stream);

/* Self-test of the bounded device-side wait used by every streaming pass:
 * one kernel waits on an mbarrier that nothing completes, gives up after the
 * wait's iteration limit (about a second) and reports it.  Returns
 * AA_ETIMEOUT when the wait ran out and came back as a status (the expected
 * result; the context stays usable), AA_OK if the wait completed, AA_ECUDA or
 * AA_ENOMEM on a CUDA failure.  Synchronizes `stream`.  No counterpart in the
 * paper. */
int aa_selftest_wait_timeout(void *stream);

/* Message for the last error on this thread. */
const char *aa_last_error(void);
const char *aa_strerror(int code);

/* Library version string. */
const char *aa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AA_H_ */
