/*
 * krp.h -- C ABI of the GB300 (sm_103a) Khatri-Rao random projection library.
 *
 * What it computes (Saibaba, Verma, Ballard, "Improved Analysis of Khatri-Rao
 * Random Projections and Applications"):
 *   - the mode-n KRP sketch  Y_n = X_(n) (Omega_d kr ... kr Omega_{n+1} kr
 *     Omega_{n-1} kr ... kr Omega_1)  of a dense d-way tensor, without forming
 *     the Khatri-Rao product (Sec. 5.1, Alg. 7 MTTKRP step);
 *   - all d sketches from one shared factor set by a dimension tree
 *     (RHOSVD-KRP-MEMO, Sec. 5.1);
 *   - randomized HOSVD / ST-HOSVD with KRP sketches (Alg. 7, Alg. 8): FP64
 *     thin QR of every sketch, multi-TTM core G = X x_1 Q_1^T ... x_d Q_d^T,
 *     optional FP64 rank-r truncation of the core and FP64 residual;
 *   - the single-pass randomized SVD of a block Hankel matrix with KRP
 *     sketches (Alg. 6, Eq. (4.1)).
 *
 * Conventions used by every entry point
 *   Layout.  A d-way tensor X of dims (n_1..n_d) is mode-1 fastest: element
 *     (i_1..i_d), 0-based, sits at sum_j i_j * prod_{m<j} ld_m, where ld
 *     (the per-mode leading sizes, ld_m >= n_m) is the argument `ld` of the
 *     entry points that take X; ld = NULL means ld_m = n_m (dense: a
 *     C-contiguous torch tensor of shape (n_d, ..., n_1)).  A padded X (some
 *     ld_m > n_m) must be device memory; it is first packed into a dense
 *     copy in the workspace (one extra read and write of X).  For KRP_BF16X2
 *     both planes have the same padding and the lo plane starts prod_m ld_m
 *     elements after the hi plane.
 *     Matrices (factors Omega_j, sketches Y_n, bases Q_n) are column-major with
 *     leading dimension equal to their row count.
 *   Memory.  Unless stated otherwise, data pointers are device pointers of the
 *     context's device.  The caller allocates and owns inputs and outputs; the
 *     context owns its workspace (grown on demand with cudaMalloc between
 *     calls).  krp_tucker_* and krp_block_hankel_lowrank also accept host
 *     pointers for X / blocks and for their outputs: they are detected with
 *     cudaPointerGetAttributes and staged through the workspace.
 *   Streams.  All work is enqueued on the context's stream (set at creation
 *     or with krp_set_stream) and is asynchronous unless stated otherwise.
 *   Errors.  Arguments are validated before any launch; on failure the call
 *     returns a non-zero krp_status, launches nothing and records a message
 *     readable with krp_last_error.  No entry point aborts or throws.
 *   Threads.  A context may be used by one host thread at a time.
 *   Precision.  KRP_F32 inputs keep FP32-level error: the passes over X run
 *     on tcgen05 tensor cores as three TF32 products of exact hi/lo splits
 *     (X F ~ X_h F_h + X_h F_l + X_l F_h) where n_1 % 4 == 0, X is 16-byte
 *     aligned and the widths fit (l <= 64; c_1 <= 32 for the residual), and
 *     on FP32 CUDA cores otherwise; KRP_BF16 inputs run the contractions over
 *     X on tcgen05 with BF16 operands and FP32 accumulation.  QR, truncation
 *     and the residual's sums are FP64.
 */
#ifndef KRP_H_
#define KRP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KRP_ABI_VERSION 2
#define KRP_MAXD 8

typedef enum krp_status {
  KRP_OK = 0,
  KRP_EINVAL = 1,        /* invalid argument (shape, pointer, dtype, flag) */
  KRP_ENOMEM = 2,        /* workspace allocation failed */
  KRP_ECUDA = 3,         /* a CUDA runtime/driver call failed */
  KRP_EUNSUPPORTED = 4,  /* valid request the library does not implement */
  KRP_ETIMEOUT = 5,      /* a bounded device-side wait expired */
  KRP_ENUMERIC = 6       /* NaN/Inf met in a FP64 stage */
} krp_status;

typedef enum krp_dtype {
  KRP_F32 = 0,
  KRP_BF16 = 1,
  KRP_FP8_E4M3 = 2,  /* reserved */
  KRP_F64 = 3,
  /* X as a BF16 hi/lo pair: 2N BF16 values, the hi plane (N) then the lo
   * plane (N), X ~ hi + lo with |X - hi - lo| <= 2^-17 |X| (krp_split_bf16x2
   * builds it from FP32).  Contractions over X run on tensor cores with both
   * planes (FP32 accuracy of X at 4 bytes per element); factors are BF16. */
  KRP_BF16X2 = 4
} krp_dtype;

/* Flags of krp_tucker_rhosvd / krp_tucker_sthosvd. */
#define KRP_MEMO 0x1u     /* one shared factor set + dimension tree (MEMO variant) */
#define KRP_TRUNCATE 0x2u /* truncate the rank-l result to ranks r_i */
#define KRP_RESIDUAL 0x4u /* compute ||X - X_hat||_F / ||X||_F (extra pass over X) */
#define KRP_TIMINGS 0x8u  /* fill krp_tucker_out.times (events between phases; synchronises) */

/* Draw ids of the factor sets used by the Tucker pipelines (see
 * krp_gen_factors): memoized set = 0, fresh set of mode i = 1 + i, ST-HOSVD
 * step i = 64 + i.  Stream tags: 0 = Omega (right sketch), 1 = Psi (left). */
#define KRP_DRAW_MEMO 0u
#define KRP_DRAW_FRESH_BASE 1u
#define KRP_DRAW_STHOSVD_BASE 64u
#define KRP_TAG_OMEGA 0u
#define KRP_TAG_PSI 1u

typedef struct krp_ctx_s* krp_ctx;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Errors: KRP_EINVAL
 * (null out, bad device), KRP_ECUDA. */
krp_status krp_create(krp_ctx* out, int device, void* cuda_stream);

/* Synchronise the context's stream, free its workspace and the context. */
krp_status krp_destroy(krp_ctx ctx);

/* Switch the stream later work is enqueued on. */
krp_status krp_set_stream(krp_ctx ctx, void* cuda_stream);

/* Limit, in nanoseconds, of every bounded device-side wait of the context's
 * tensor-core kernels (their mbarrier waits on TMA data, MMA completion and
 * the other warp roles); 0 restores the default of 1 s.  A wait that runs
 * out makes its kernel stop: it records KRP_ETIMEOUT in the context's status
 * word (the first error recorded is kept), lets the copies and MMAs it has
 * issued complete (those waits keep the 1 s default), frees its tensor
 * memory and returns; the pipeline entry points then return KRP_ETIMEOUT and
 * clear the word.  Diagnostics: a limit shorter than the kernels' own
 * progress (e.g. 1 ns) exercises that path; the paper has no counterpart.
 * Synchronises the context's stream.  Errors: KRP_EINVAL (null ctx),
 * KRP_ECUDA. */
krp_status krp_set_wait_limit(krp_ctx ctx, uint64_t ns);

/* Message of the last failed call on `ctx` ("" if none).  Owned by ctx. */
const char* krp_last_error(krp_ctx ctx);

/* Static name of a status code. */
const char* krp_status_string(krp_status s);

/* KRP_ABI_VERSION of the loaded library. */
int krp_abi_version(void);

/* Number of kernels this context has launched so far (for launch counting). */
uint64_t krp_launch_count(krp_ctx ctx);

/* ---- a1: sketching factors (Def. of KRP, Sec. 2.5) ------------------------ */

/* Draw i.i.d. N(0,1) factors Omega_j (rows[j] x ell, column-major) on the
 * device from Philox4x32-10 (10 rounds, Salmon et al. SC'11) and Box-Muller:
 *   key = (seed mod 2^32, seed >> 32); entry (i,k) has e = i + rows[j]*k and
 *   counter (e >> 2, j, draw_id, tag); the 4 output words of a counter give
 *   entries e&~3 .. e|3 as z0 = rho(w0)cos(2pi u(w1)), z1 = rho(w0)sin(..),
 *   z2 = rho(w2)cos(2pi u(w3)), z3 = rho(w2)sin(..), u(w) = (w+0.5)/2^32,
 *   rho(w) = sqrt(-2 ln u(w)), computed in FP64, then rounded to out_type
 *   (KRP_F32: RN; KRP_BF16: RN to FP32 then RN-even to bfloat16; KRP_F64).
 * omega[j] may be NULL to skip factor j.  Column k of a factor does not depend
 * on ell (prefix-consistent).  Errors: KRP_EINVAL (d out of 1..KRP_MAXD,
 * rows[j] < 1, ell < 1, bad dtype). */
krp_status krp_gen_factors(krp_ctx ctx, uint64_t seed, uint32_t draw_id,
                           uint32_t tag, int d, const int64_t* rows, int ell,
                           krp_dtype out_type, void* const* omega);

/* The raw Philox4x32-10 words for counters (first_block + b, c1, c2, c3),
 * b = 0..nblocks-1, under the key of `seed`; out (device) receives 4*nblocks
 * uint32 in counter order.  Used to check the stream bit-exactly. */
krp_status krp_philox_words(krp_ctx ctx, uint64_t seed, uint32_t c1,
                            uint32_t c2, uint32_t c3, uint64_t first_block,
                            int64_t nblocks, uint32_t* out);

/* ---- a2: one mode-n sketch (Alg. 7, MTTKRP step) -------------------------- */

/* Y (dims[n] x ell, FP32, column-major) = X_(n) K_n with
 * K_n = Omega_d kr ... kr Omega_{n+1} kr Omega_{n-1} kr ... kr Omega_1.
 * X: xt = KRP_F32, KRP_BF16 or KRP_BF16X2; omega[j] (j != n) is dims[j] x
 * ell of type omt (KRP_F32 for F32 X, KRP_BF16 for BF16 and BF16X2 X);
 * omega[n] is ignored.  The tensor-core forms need n_1 % 8 == 0 and a
 * 16-byte aligned X (KRP_EINVAL otherwise).  n is
 * 0-based.  d in 2..KRP_MAXD, 1 <= ell <= 256.  The product is never formed:
 * the contraction runs over X once (two-stage: one factor by GEMM, the rest
 * as Hadamard-weighted reductions).  Errors: KRP_EINVAL, KRP_ENOMEM, KRP_ECUDA. */
krp_status krp_sketch_mode(krp_ctx ctx, const void* X, krp_dtype xt, int d,
                           const int64_t* dims, const int64_t* ld, int n,
                           const void* const* omega, krp_dtype omt, int ell,
                           float* Y);

/* ---- a3: all d sketches with one factor set (RHOSVD-KRP-MEMO, Sec. 5.1) ---- */

/* Y[n] (dims[n] x ell) for n = 0..d-1 from the shared factors omega[0..d-1],
 * by a dimension tree that contracts the first mode once and reuses the
 * partial result for every mode but the first (cost 4 N ell flops, Sec. 5.1).
 * Arguments as in krp_sketch_mode.  tree_split (tensor-core forms, one pass
 * over X): the tree's second dimension is the modes 2..tree_split+1 merged
 * (1 <= tree_split <= d-1), contracted in the same pass as mode 1, and its
 * sketch is split into those modes' sketches afterwards; -1 lets the library
 * pick it: the first call for a given (dims, ell, dtype) times every split
 * whose merged dimension has at most 2^20 rows (the call then synchronises
 * the stream) and the context keeps the fastest for later calls.  The FP32
 * form ignores tree_split.  Errors: as krp_sketch_mode, and KRP_EINVAL for a
 * tree_split out of range. */
krp_status krp_sketch_all_modes(krp_ctx ctx, const void* X, krp_dtype xt,
                                int d, const int64_t* dims, const int64_t* ld,
                                const void* const* omega, krp_dtype omt,
                                int ell, float* const* Y, int tree_split);

/* ---- a4: FP64 thin QR (Alg. 1 step 3) ------------------------------------ */

/* FP64 thin QR of `count` FP32 matrices Y[b] (m[b] x l[b], column-major,
 * m >= l) into Q[b] (FP64, m x l, column-major, diag(R) >= 0): shifted
 * CholeskyQR3 for l <= 64 (columns whose pivot collapses are refilled and
 * re-orthogonalised, so Q stays orthonormal for rank-deficient Y),
 * Householder above.  R[b] (l x l, FP64, column-major) may be NULL.
 * Errors: KRP_EINVAL (m < l, l > 256),
 * KRP_ENUMERIC (non-finite input; reported after a stream synchronisation). */
krp_status krp_qr(krp_ctx ctx, int count, const float* const* Y,
                  const int64_t* m, const int* l, double* const* Q,
                  double* const* R);

/* The same FP64 thin QR as krp_qr, for one FP32 matrix, without allocating any
 * device memory.  The paper has no counterpart: this is a service for callers
 * that may not call cudaMalloc while they run -- code inside a framework whose
 * caching allocator owns the device memory, loops that cannot afford the
 * device-wide synchronisation of cudaMalloc/cudaFree, programs that reserve
 * their memory budget up front.  It needs no context: it runs on the calling
 * thread's current device and enqueues on `cuda_stream` (a cudaStream_t, NULL
 * = legacy default stream); Y (m x l), Q (m x l) and the optional R (l x l)
 * are device pointers, column-major.
 * Scratch: one fixed __device__ array of KRP_QR_NOALLOC_MAX_DOUBLES doubles
 * (4 MiB) built into the library, resident on every GPU that loads it until
 * the process exits.  A call needs m*l + 4*l*l + 2 of those doubles; larger
 * requests, l outside 1..64, m < l and NULL Y/Q return KRP_EINVAL before any
 * launch.  Every call looks the array's device address up with
 * cudaGetSymbolAddress in the current device's context (nothing is cached, so
 * a device reset does not leave a stale address); the first call on a device
 * may load the library's device code there, so make it before any stream
 * capture.  All calls share the array and it keeps the last call's
 * contents (the accumulators a call needs zeroed are cleared by the call), so
 * calls whose work can overlap on the GPU -- on different streams, or from
 * different threads -- race and must be serialised by the caller.  The call
 * is asynchronous and does not check the input for NaN/Inf: for non-finite
 * input Q and R are undefined and the call still returns KRP_OK (krp_qr
 * reports KRP_ENUMERIC instead).  CUDA launch failures return KRP_ECUDA. */
#define KRP_QR_NOALLOC_MAX_DOUBLES 524288
krp_status krp_qr_noalloc(const float* Y, int64_t m, int l, double* Q,
                          double* R, void* cuda_stream);

/* Launch trace (diagnostics): between krp_trace_begin and krp_trace_end the
 * context records a CUDA event after every kernel it launches, on the stream
 * of the launch (its own stream, or the second stream that runs the FP32
 * form's QR beside the TTMs; not inside captured graphs).  krp_trace_end
 * synchronises and writes a JSON list [["launch name", ms], ...] into json
 * (cap bytes): the time from the previous event on the same stream, i.e.
 * each launch's duration on its stream including any copy or memset
 * enqueued just before it.  KRP_EINVAL if the buffer is too small. */
krp_status krp_trace_begin(krp_ctx ctx);
krp_status krp_trace_end(krp_ctx ctx, char* json, size_t cap);

/* hi[e] = bf16_rn(X[e]), lo[e] = bf16_rn(X[e] - hi[e]) for e < n; out holds
 * 2n BF16 values (hi plane then lo plane), the KRP_BF16X2 layout.  X and out
 * are device pointers (out 16-byte aligned).  The paper streams X in one
 * precision; this split form is not in it. */
krp_status krp_split_bf16x2(krp_ctx ctx, const float* X, int64_t n, void* out);

/* ---- a5: multi-TTM core (Alg. 7 last step) ------------------------------- */

/* G = X x_1 Q_1^T x_2 Q_2^T ... x_d Q_d^T, G of dims (cols[0..d-1]) FP32,
 * mode-1 fastest.  Q[j] is FP64 dims[j] x cols[j] column-major.  X as in
 * krp_sketch_mode (KRP_F32, KRP_BF16 or KRP_BF16X2); with BF16 X the first
 * two contractions run on tensor cores with Q_1 (and the intermediate) as
 * BF16 hi/lo pairs.  All pointers are device pointers.  Errors: KRP_EINVAL,
 * KRP_ENOMEM, KRP_ECUDA. */
krp_status krp_multi_ttm(krp_ctx ctx, const void* X, krp_dtype xt, int d,
                         const int64_t* dims, const int64_t* ld,
                         const double* const* Q, const int* cols, float* G);

/* ---- a7, a8 as separate steps (for sharded use: one slab of X per GPU) ---- */

/* Rank truncation of a Tucker core by an FP64 HOSVD of the core: per mode i
 * the leading ranks[i] left singular vectors U_i of the unfolding G_(i)
 * (from the eigenvectors of the ell[i] x ell[i] Gram matrix), then
 * core_out = G x_1 U_1^T ... x_d U_d^T and factors_out[i] = factors[i] U_i.
 * (Sec. 2.2 HOSVD applied to the small core; equal to the HOSVD of the
 * rank-ell approximation because every factors[i] is orthonormal.)
 *   core:        device FP32, ell[0] x ... x ell[d-1], mode-1 fastest (read)
 *   factors[i]:  device FP64, dims[i] x ell[i], column-major (read)
 *   core_out:    device FP32, ranks[0] x ... x ranks[d-1] (written)
 *   factors_out[i]: device FP64, dims[i] x ranks[i] (written)
 * Requires 1 <= ranks[i] <= ell[i] <= min(64, dims[i]).  Synchronises the
 * context stream; KRP_ENUMERIC if a non-finite value is met. */
krp_status krp_core_truncate(krp_ctx ctx, int d, const int64_t* dims, const int* ell,
                             const int* ranks, const float* core,
                             const double* const* factors, float* core_out,
                             double* const* factors_out);

/* Residual sums of a Tucker approximation X_hat = core x {factors}:
 *   sums[0] = ||X - X_hat||_F^2,  sums[1] = ||X||_F^2   (FP64, host array)
 * by one streaming pass over X (Sec. 5.2 error; the same computation as
 * KRP_RESIDUAL).  For a slab of X along the last mode, pass the slab's dims
 * and the matching rows of the last factor: the sums of all slabs add up to
 * the whole tensor's.
 *   X: device, dims, mode-1 fastest, dtype xt (F32, BF16 or BF16X2)
 *   core: device FP32, core_dims; factors[i]: device FP64 dims[i] x core_dims[i]
 * Synchronises the context stream. */
krp_status krp_residual(krp_ctx ctx, const void* X, krp_dtype xt, int d,
                        const int64_t* dims, const int64_t* ld, const int* core_dims,
                        const float* core, const double* const* factors, double* sums);

/* ---- a6-a8: randomized Tucker pipelines (Alg. 7, Alg. 8) ------------------ */

typedef struct krp_phase_times {
  double rng_ms, sketch_ms, qr_ms, core_ms, truncate_ms, residual_ms, total_ms;
} krp_phase_times;

typedef struct krp_tucker_out {
  /* in: output buffers sized for the output ranks (l_i = r_i + oversample,
   * or r_i with KRP_TRUNCATE); device or host memory */
  float* core;                   /* prod of output ranks, mode-1 fastest */
  double* factors[KRP_MAXD];     /* n_i x rank_i, column-major */
  /* out */
  int d;
  int64_t core_dims[KRP_MAXD];
  double rel_residual;           /* with KRP_RESIDUAL, else -1 */
  double x_norm;                 /* ||X||_F (with KRP_RESIDUAL, else -1) */
  double core_norm;              /* ||G||_F */
  krp_phase_times times;         /* with KRP_TIMINGS */
} krp_tucker_out;

/* RHOSVD-KRP (Alg. 7): per mode i a fresh factor set (draw 1+i) of sketch
 * size l_i = ranks[i] + oversample, sketch Y_i, FP64 QR -> Q_i; then the core
 * G = X x {Q_i^T}.  With KRP_MEMO one shared set (draw 0, l = max l_i) and
 * the dimension tree (krp_sketch_all_modes).  KRP_TRUNCATE: rank-r_i
 * truncation by an FP64 HOSVD of the core (U_i = leading r_i left singular
 * vectors of G_(i), G <- G x {U_i^T}, Q_i <- Q_i U_i).  KRP_RESIDUAL: FP64
 * ||X - X_hat||_F / ||X||_F by streaming reconstruction.  Needs l_i <= n_i
 * (l_i <= 64 with KRP_TRUNCATE).  X is KRP_F32, KRP_BF16 or KRP_BF16X2 (for
 * the last two the factors are drawn in BF16).  KRP_TIMINGS fills
 * out->times from CUDA events recorded between the phases (the call then
 * synchronises the stream).  Errors: KRP_EINVAL (shapes,
 * ranks, flags, dtype, NULL buffers), KRP_ENOMEM, KRP_ECUDA; KRP_ETIMEOUT if
 * a bounded device-side wait expired and KRP_ENUMERIC if an FP64 stage met a
 * non-finite value (both read from the context's device status word after
 * a stream synchronisation). */
krp_status krp_tucker_rhosvd(krp_ctx ctx, const void* X, krp_dtype xt, int d,
                             const int64_t* dims, const int64_t* ld,
                             const int* ranks, int oversample, uint64_t seed,
                             unsigned flags, krp_tucker_out* out);

/* RSTHOSVD-KRP (Alg. 8), modes in the order 1..d: step i sketches the current
 * core with factors of draw 64+i (l_j x l_i for j < i, n_j x l_i for j > i),
 * QR -> Q_i, G <- G x_i Q_i^T.  Flags as above except KRP_MEMO (ignored). */
krp_status krp_tucker_sthosvd(krp_ctx ctx, const void* X, krp_dtype xt, int d,
                              const int64_t* dims, const int64_t* ld,
                              const int* ranks, int oversample, uint64_t seed,
                              unsigned flags, krp_tucker_out* out);

/* ---- a9-a10: block Hankel single-pass low-rank approximation (Alg. 6) ------ */

/* M is the (m s) x (n s) block Hankel matrix with block (i, j) = H_{i+j-1}
 * (1-based), given as `blocks`: 2s-1 column-major m x n blocks stored one
 * after another (FP32 or BF16).  With Omega = Omega1 kr Omega2 (s x l_r,
 * n x l_r; tag 0) and Psi = Psi1 kr Psi2 (s x l_l, m x l_l; tag 1), draw 0:
 *   Y = M Omega  = sum_k (E_k Omega1) kr (H_k Omega2)     (Eq. (4.1))
 *   Z = M^T Psi  = sum_k (E_k^T Psi1) kr (H_k^T Psi2)
 *   Y = QR;  W = (Psi^T Q)^+ Z^T;  W = U_W S V^T;  U = Q U_W;
 * returns U (m s x r), S (r), V (n s x r), FP64 column-major (device or host).
 * ell_l = 0 selects ceil(1.5 ell_r).  Needs 1 <= r <= ell_r <= ell_l,
 * ell_r <= m s, ell_l <= n s, ell_r <= 64, ell_l <= 256.  Synchronises the
 * stream.
 * Errors: KRP_EINVAL (sizes, dtype, NULL buffers), KRP_ENOMEM, KRP_ECUDA,
 * KRP_ENUMERIC (an FP64 stage met a non-finite value). */
krp_status krp_block_hankel_lowrank(krp_ctx ctx, const void* blocks,
                                    krp_dtype bt, int m, int n, int s, int r,
                                    int ell_r, int ell_l, uint64_t seed,
                                    double* U, double* S, double* V);

/* Alg. 6 on a two-level block Hankel matrix (Sec. 4.3, multilevel block
 * structure with L = 2): M is (m s1 s2) x (n s1 s2); block (i1, j1) of M
 * (1-based, s1 x s1 of them) is itself an s2 x s2 block Hankel matrix whose
 * block (i2, j2) is H_{i1+j1-1, i2+j2-1}, m x n, i.e.
 *   M = sum_{k1, k2} E_{k1} kron E_{k2} kron H_{k1,k2}.
 * `blocks` holds the (2 s1 - 1)(2 s2 - 1) column-major m x n blocks, block
 * (k1, k2) (0-based) at position k1 + (2 s1 - 1) k2; row index of M is
 * a + m (i2 + s2 i1) (0-based).  With Omega = Omega1 kr Omega2 kr Omega3
 * (s1, s2, n rows x l_r; factors 0, 1, 2 of tag 0) and Psi = Psi1 kr Psi2 kr
 * Psi3 (s1, s2, m rows x l_l; tag 1), draw 0:
 *   Y = M Omega = sum_{k1,k2} (E_{k1} Omega1) kr (E_{k2} Omega2) kr (H_{k1,k2} Omega3)
 * (the two-level form of Eq. (4.1)), Z = M^T Psi likewise with the blocks
 * transposed, then the steps of krp_block_hankel_lowrank: returns U
 * (m s1 s2 x r), S (r), V (n s1 s2 x r), FP64 column-major (device or host).
 * ell_l = 0 selects ceil(1.5 ell_r).  Needs 1 <= r <= ell_r <= ell_l,
 * ell_r <= 64, ell_l <= 256, ell_r <= m s1 s2, ell_l <= n s1 s2.  Synchronises
 * the stream.  Errors: KRP_EINVAL, KRP_ENOMEM, KRP_ECUDA, KRP_ENUMERIC. */
krp_status krp_block_hankel2_lowrank(krp_ctx ctx, const void* blocks,
                                     krp_dtype bt, int m, int n, int s1, int s2,
                                     int r, int ell_r, int ell_l, uint64_t seed,
                                     double* U, double* S, double* V);

/* The two sketches of Alg. 6 alone (device pointers): Y (m s x ell_r) and
 * Z (n s x ell_l), FP32, from given factors (FP32 or BF16 like the blocks;
 * omega1 s x ell_r, omega2 n x ell_r, psi1 s x ell_l, psi2 m x ell_l, all
 * column-major).  Asynchronous.  Errors: KRP_EINVAL, KRP_ENOMEM, KRP_ECUDA. */
krp_status krp_block_hankel_sketch(krp_ctx ctx, const void* blocks,
                                   krp_dtype bt, int m, int n, int s,
                                   const void* omega1, const void* omega2,
                                   int ell_r, const void* psi1,
                                   const void* psi2, int ell_l, float* Y,
                                   float* Z);

/* Nystrom approximation of a symmetric positive semidefinite block Hankel
 * matrix M (Sec. 4.1, the remark after Alg. 6):
 *   M_nys = (M Omega) (Omega^T M Omega)^+ (M Omega)^T,  Omega = Omega1 kr Omega2,
 * with the column-sketch factors of krp_block_hankel_lowrank (Omega1 s x ell,
 * Omega2 m x ell, tag 0, draw 0), so Y = M Omega is that call's Y for
 * ell_r = ell.  Y = QR (FP64), C = Omega^T Y = (Omega^T Q) R formed
 * structurally and symmetrised, C = V diag(c) V^T; the pseudoinverse treats
 * c_i <= rcond * c_1 as zero (rcond <= 0 selects 1e-5); the eigenpairs of
 * M_nys = Q (R C^+ R^T) Q^T come from the ell x ell matrix R C^+ R^T.
 *   blocks: 2s-1 column-major m x m blocks (FP32 or BF16), each symmetric
 *           and M positive semidefinite (the caller's promise; not checked)
 *   U:      m s x r FP64 column-major, the top r eigenvectors of M_nys
 *   Lambda: r FP64, their eigenvalues, descending
 * Device or host pointers (host ones are staged).  Needs 1 <= r <= ell <=
 * min(64, m s) and rcond < 1.  Synchronises the stream.  Errors: KRP_EINVAL,
 * KRP_ENOMEM, KRP_ECUDA, KRP_ENUMERIC (an FP64 stage met a non-finite
 * value). */
krp_status krp_block_hankel_nystrom(krp_ctx ctx, const void* blocks,
                                    krp_dtype bt, int m, int s, int r, int ell,
                                    double rcond, uint64_t seed, double* U,
                                    double* Lambda);

/* Eigensystem realization from the rank-r result of krp_block_hankel_lowrank
 * (the use Sec. 4.2 makes of Alg. 6): with M ~ U S V^T, O = U S^{1/2} and
 * G^+ = V S^{-1/2}, the state matrix is
 *   A = O_top^+ H_up G^+,
 * O_top the first (s-1) m rows of O and H_up the block Hankel matrix shifted
 * by one block (block (i, j) = h_{i+j}, i = 1..s-1, j = 1..s, 1-based, i.e.
 * blocks 2..2s-1).  A is determined up to a similarity transform; its
 * eigenvalues are the realized system's.  The least-squares step uses the
 * normal equations with a Cholesky factor in FP64 (O_top's condition number
 * is that of S^{1/2} on the orthonormal rows of U, small for a decaying
 * Hankel spectrum), the eigenvalues Householder reduction to Hessenberg form
 * and the Francis double-shift QR iteration in FP64 (Golub & Van Loan).
 *   blocks: 2s-1 column-major m x n blocks as for krp_block_hankel_lowrank
 *           (KRP_F32 or KRP_BF16); U (m s x r), S (r), V (n s x r): FP64
 *   A:      r x r FP64 column-major (may be NULL)
 *   eig_re, eig_im: r FP64 each, the eigenvalues in deflation order (complex
 *           pairs adjacent, positive imaginary part first)
 * All pointers are device pointers.  Needs s >= 2 and 1 <= r <= min(64,
 * (s-1) m, s n).  Synchronises the stream.  Errors: KRP_EINVAL, KRP_ENOMEM,
 * KRP_ECUDA, KRP_ENUMERIC (O_top rank-deficient, a non-finite value, or an
 * eigenvalue that did not converge in 100 iterations). */
krp_status krp_era_realize(krp_ctx ctx, const void* blocks, krp_dtype bt, int m,
                           int n, int s, int r, const double* U, const double* S,
                           const double* V, double* A, double* eig_re,
                           double* eig_im);

/* ---- Hadamard products of Tucker tensors (Sec. 5, its opening) ----------- */

/* RHOSVD-KRP-MEMO of Z = X * Y (elementwise), X = G x {U_j}, Y = H x {V_j},
 * without forming Z: Z is the Tucker tensor with core G (x) H (index
 * c_j = a_j + r_j b_j) and factors W_j[i, c_j] = U_j[i, a_j] V_j[i, b_j], so
 * with one Philox factor set Omega_j (n_j x l, FP64, draw 0, tag 0 -- the
 * MEMO set of krp_tucker_rhosvd):
 *   Y_n = W_n MTTKRP_n(G (x) H, {W_j^T Omega_j}),  Y_n = Q_n R_n,
 *   core = (G (x) H) x_1 (Q_1^T W_1) ... x_d (Q_d^T W_d),
 *   rel_error = sqrt(max(0, ||Z||^2 - ||core||^2)) / ||Z|| with
 *   ||Z||^2 = <G (x) H, (G (x) H) x_j (W_j^T W_j)> (cancellation limits it to
 *   errors above ~1e-7).
 *   G: r_1 x ... x r_d, H: s_1 x ... x s_d (FP64, mode-1 fastest);
 *   U[j]: n_j x r_j, V[j]: n_j x s_j (FP64 column-major); core: l^d FP64;
 *   factors[j]: n_j x l FP64 column-major (orthonormal); rel_error: host
 *   double, may be NULL.
 * Device pointers except rel_error.  Needs 1 <= l <= min(64, n_j) and
 * prod_j r_j s_j <= 2^25.  Synchronises the stream.  Errors: KRP_EINVAL,
 * KRP_ENOMEM, KRP_ECUDA, KRP_ENUMERIC. */
krp_status krp_tucker_hadamard(krp_ctx ctx, int d, const int64_t* dims,
                               const int* rg, const double* G,
                               const double* const* U, const int* rh,
                               const double* H, const double* const* V,
                               int ell, uint64_t seed, double* core,
                               double* const* factors, double* rel_error);

/* ---- Sensor placement from Tucker factors (Sec. 6) ------------------------ */

/* Training phase: for each mode i, the column-pivoted Householder QR of
 * Q_i^T (l_i x N_i) picks l_i grid indices (the first l_i pivots, in the
 * order picked: at step k the column of largest remaining norm over rows
 * k..l_i-1, ties to the lowest position, decided in FP64), and the
 * interpolation factor is A_i = Q_i (P_i^T Q_i)^{-1}, P_i^T Q_i = Q_i[idx_i, :]
 * (Gauss-Jordan elimination with partial pivoting, FP64).
 *   Q[i]:   N_i x l_i FP64 column-major with orthonormal columns (e.g. the
 *           factors returned by krp_tucker_rhosvd)
 *   idx[i]: l_i int32, the sensor indices of mode i (0-based)
 *   A[i]:   N_i x l_i FP64 column-major
 * All device pointers.  Needs 1 <= d <= KRP_MAXD and 1 <= l_i <= min(64, N_i).
 * Synchronises the stream.  Errors: KRP_EINVAL, KRP_ENOMEM, KRP_ECUDA,
 * KRP_ENUMERIC (P_i^T Q_i singular). */
krp_status krp_sensor_select(krp_ctx ctx, int d, const int64_t* dims,
                             const int* ells, const double* const* Q,
                             int* const* idx, double* const* A);

/* Test phase: T ~ T_hat x_1 A_1 ... x_d A_d from the measurements
 * T_hat = T(idx_1, ..., idx_d) (l_1 x ... x l_d FP32, mode-1 fastest) with the
 * factors of krp_sensor_select; out (N_1 x ... x N_d FP32, mode-1 fastest).
 * The expansion runs in FP64 (one small TTM per mode).  Device pointers;
 * asynchronous.  Errors: KRP_EINVAL, KRP_ENOMEM, KRP_ECUDA. */
krp_status krp_sensor_reconstruct(krp_ctx ctx, int d, const int64_t* dims,
                                  const int* ells, const double* const* A,
                                  const float* T_hat, float* out);

/* ---- a11: batches of small uneven 3-way tensors -------------------------- */

/* One tensor of a batch (all device pointers). */
typedef struct krp_tucker_item {
  const void* X;          /* in: n1 x n2 x n3, mode-1 fastest, the batch dtype */
  int64_t dims[3];        /* in: 1 <= n_i <= 256 */
  int ranks[3];           /* in: r_i; l_i = r_i + oversample <= min(32, n_i) */
  uint64_t seed;          /* in: Philox key of this tensor's factor set */
  float* core;            /* in: output, prod of output ranks, mode-1 fastest */
  double* factors[3];     /* in: outputs, n_i x rank_i column-major FP64 */
  double rel_residual;    /* out: with KRP_RESIDUAL, else -1 */
} krp_tucker_item;

/* RHOSVD-KRP-MEMO (Alg. 7 with one factor set per tensor, draw 0 of key
 * `seed`, i.e. exactly what krp_tucker_rhosvd with KRP_MEMO computes for that
 * tensor alone) of `count` 3-way tensors of different shapes and ranks, each
 * phase one launch over the whole batch (persistent kernels whose warps take
 * work units of mode-3 slabs from an atomic counter; with KRP_BF16 the
 * contractions run on warp-level tensor-core MMAs; QR and eigenproblems as
 * job arrays).  Dims n_i <= 256, l_i = rank_i + oversample <= min(32, n_i).
 * Flags: KRP_TRUNCATE, KRP_RESIDUAL (KRP_MEMO implied).  The first call with
 * a given set of descriptors (pointers, shapes, ranks, seeds, flags)
 * allocates the batch's scratch, picks the slabs per work unit by timing,
 * and records the phase
 * sequence as a CUDA graph; later calls with identical descriptors replay
 * the graph.  The call synchronises the stream and fills rel_residual.  The
 * plan and its scratch stay with the context until a call with other
 * descriptors or krp_destroy.  The paper describes single tensors only; the
 * batched form has no counterpart there.  Errors: KRP_EINVAL (shapes, ranks,
 * host pointers, dtype), KRP_ENOMEM, KRP_ECUDA, KRP_ENUMERIC. */
krp_status krp_tucker_rhosvd_batched(krp_ctx ctx, krp_dtype xt, int count,
                                     krp_tucker_item* items, int oversample,
                                     unsigned flags);

/* One block Hankel matrix of a batch (device pointers), as for
 * krp_block_hankel_lowrank: 2s-1 column-major m x n blocks, target rank r,
 * sketch sizes ell_r, ell_l (0 = ceil(1.5 ell_r)), Philox key seed. */
typedef struct krp_hankel_item {
  const void* blocks;
  int m, n, s, r, ell_r, ell_l;
  uint64_t seed;
  double* U;              /* out: m s x r */
  double* S;              /* out: r */
  double* V;              /* out: n s x r */
} krp_hankel_item;

/* Alg. 6 for `count` block Hankel matrices of different sizes, each phase one
 * launch over the batch; item b computes what krp_block_hankel_lowrank
 * computes for it alone.  As for krp_tucker_rhosvd_batched, the first call
 * with given descriptors builds a plan and records a CUDA graph that later
 * identical calls replay (ell_l = 0 is replaced in the descriptor by its
 * value).  Needs ell_r <= 64.  Synchronises the stream.  The paper describes
 * single matrices only; the batched form has no counterpart there.  Errors:
 * KRP_EINVAL (sizes, dtype, host pointers), KRP_ENOMEM, KRP_ECUDA,
 * KRP_ENUMERIC. */
krp_status krp_block_hankel_batched(krp_ctx ctx, krp_dtype bt, int count,
                                    krp_hankel_item* items);

/* Work split of the context's current batch plan: slabs per sketch unit
 * (picked by timing), number of sketch units (warp work items), and the
 * sketch kernel's grid; KRP_EINVAL if there is none. */
krp_status krp_tucker_batch_plan_info(krp_ctx ctx, int* slabs_per_unit,
                                      int* units, int* grid);

#ifdef __cplusplus
}
#endif

#endif /* KRP_H_ */
