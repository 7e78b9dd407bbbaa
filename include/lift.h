/*
 * liftblas -- C-ABI of the GB300 (sm_103a) kernels for the fused map/reduce
 * programs of Steuwer, Fensch and Dubach, "Patterns and Rewrite Rules for
 * Systematic Code Generation" (arXiv 1502.02389):
 *
 *   scal(a, x)          = map(mult(a), x)                          Fig. 5
 *   asum(x)             = reduce(add, 0) . map(abs, x)             Fig. 5
 *   dot(x, y)           = reduce(add, 0) . map(mult) . zip(x, y)   Fig. 5
 *   gemv(A, x, y, a, b) = y <- a*A*x + b*y, map(dot) over rows     Fig. 5, Sec. 5.1
 *
 * and, built the same way: the mixed-precision asum / dot (bf16, fp8-e4m3
 * with block scales), the compensated fp32 asum / dot, nrm2, sum and axpy
 * (other user functions in the same patterns, Sec. 4.2), gemv-T (gemv over
 * the reorder-stride transpose, Sec. 3.2), BlackScholes (the map of Fig. 6),
 * a batched persistent launch of many asum / dot / scal / gemv calls, and
 * the variant policies (a tuned table and a learned cost model).
 *
 * Each kernel variant is one low-level expression derived from these with
 * the rewrite rules of Fig. 3 and Fig. 4; its integer parameters (split
 * tile, vector width, reorder-stride, tree depth, combine passes, staging)
 * are compile-time template parameters.  lift_variant_describe lists them.
 *
 * Conventions for every entry point:
 *  - All array pointers are DEVICE pointers, owned by the caller; the
 *    library never frees or keeps them.  Arrays are contiguous (no BLAS inc
 *    strides); gemv's A is row-major with leading dimension lda >= N.
 *  - Sizes are int64_t element counts.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call is asynchronous on that stream: the status
 *    returned reports argument validation and launch errors only.
 *  - Nothing aborts or throws across the ABI.  Invalid arguments return
 *    LIFT_ERR_INVALID_ARG before any launch: n < 0, M < 0, N < 0, lda < N,
 *    or a NULL pointer for an array that would be read or written.
 *  - n == 0 is valid: a reduction writes 0; gemv with N == 0 computes
 *    y <- b*y, and with M == 0 does nothing.
 *  - A pointer that is not aligned for a variant's vector width or for
 *    TMA bulk copies (16 B) makes the library use the same variant family's
 *    guarded scalar-load form instead; it is not an error.
 *  - The reductions use a per-device workspace allocated by lift_init
 *    (partials, ticket counters, a status word), one slot per stream for up
 *    to 8 streams of a device; calls on the same stream are ordered by it.
 *    Calls on more than 8 streams at once share slots and can race (and
 *    after 4096 distinct stream handles the assignment starts afresh).
 *  - Most kernels are launched as programmatic dependents of the kernel
 *    before them on the stream: their CTAs may be scheduled while that
 *    kernel still runs, but each waits for it to complete (and for its
 *    writes to be visible) before touching memory, so calls on one stream
 *    stay ordered exactly as stream order promises.
 *  - lift_last_error() returns a detail message for the last failure of the
 *    calling thread.
 */
#ifndef LIFT_H
#define LIFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LIFT_OK = 0,
  LIFT_ERR_INVALID_ARG = 1,
  LIFT_ERR_UNSUPPORTED = 2,
  LIFT_ERR_CUDA = 3,
  LIFT_ERR_NO_MEMORY = 4,
  LIFT_ERR_TIMEOUT = 5,
  LIFT_ERR_NOT_INITIALIZED = 6
} lift_status;

typedef enum { LIFT_F32 = 0, LIFT_BF16 = 1, LIFT_FP8_E4M3 = 2 } lift_dtype;

/* Operation ids: the four Fig. 5 programs, the mixed-precision reductions
 * (stored bf16 or fp8-e4m3 inputs), the user-function programs, gemv-T,
 * BlackScholes and the compensated fp32 reductions.  Each has its own list
 * of variants (lift_variant_count / lift_variant_describe). */
typedef enum {
  LIFT_OP_ASUM = 0,
  LIFT_OP_DOT = 1,
  LIFT_OP_SCAL = 2,
  LIFT_OP_GEMV = 3,
  LIFT_OP_ASUM_BF16 = 4,
  LIFT_OP_DOT_BF16 = 5,
  LIFT_OP_ASUM_FP8 = 6,
  LIFT_OP_DOT_FP8 = 7,
  LIFT_OP_NRM2 = 8,
  LIFT_OP_SUM = 9,
  LIFT_OP_AXPY = 10,
  LIFT_OP_GEMV_T = 11,
  LIFT_OP_BLACKSCHOLES = 12,
  LIFT_OP_ASUM_COMP = 13,
  LIFT_OP_DOT_COMP = 14,
  LIFT_NUM_OPS = 15
} lift_op;

/* The cost model can cover op ids 0 .. LIFT_MLP_OPS-1 (a weights file says
 * how many it covers); the MLP policy falls back to the FIXED choice for the
 * others. */
#define LIFT_MLP_OPS 15

/* ------------------------------------------------------------------------
 * Library state
 * ------------------------------------------------------------------------ */

/* Set up `device`: query its SM count and allocate the reduction workspace
 * on it: 8 slots of partials and tickets (about 17 MiB each), one per
 * stream that launches work on the device (a stream takes the next slot on
 * its first call; beyond 8 streams slots are shared in turn), so calls on
 * up to 8 streams may run at the same time.  A CUDA graph keeps the slot of
 * the stream it was captured on.  Must be called (once per device) before
 * any other call on that device, outside CUDA graph capture.  Calling it
 * again is a no-op; calls from several threads at once set the device up
 * once.
 * The first call also reads two environment overrides:
 *   LIFT_POLICY  = fixed | table:<path> | mlp[:<path>] | mlp_tune[:<path>]
 *                  (the learned policies default to the weights file
 *                  data/mlp_gb300.txt beside the library);
 *   LIFT_VARIANT = comma-separated variant names, each forced for its op.
 * An unknown policy, an unreadable file or an unknown variant name makes
 * this and every later lift_init return LIFT_ERR_INVALID_ARG.
 * Returns LIFT_ERR_CUDA / LIFT_ERR_NO_MEMORY on failure. */
lift_status lift_init(int device);

/* Free the workspaces of every initialised device.  Synchronises them. */
lift_status lift_finalize(void);

const char* lift_status_string(lift_status s);
const char* lift_last_error(void);

/* Number of SMs of the current device (0 if not initialised). */
int lift_sm_count(void);

/* Read (and, if `clear`, reset) the current device's status word, where
 * kernels record a device-side wait that gave up (LIFT_ERR_TIMEOUT).
 * Synchronises with the device.  When `clear` is set and a failure was
 * recorded, it also waits for the whole device and returns every one-pass
 * "last CTA" ticket of the workspace to 0 (do not call it then while
 * another host thread launches on the device).  Returns 0, a lift_status
 * code, or LIFT_ERR_NOT_INITIALIZED / LIFT_ERR_CUDA for the read itself. */
int lift_read_status(int clear);

/* ------------------------------------------------------------------------
 * fp32 programs (Fig. 5).  The policy picks the variant (see
 * lift_set_policy).
 * ------------------------------------------------------------------------ */

/* asum: *result = sum_i |x_i| (Fig. 5: reduce(add,0) . map(abs)).
 * x: n floats; result: one float (device).  Accumulates in fp32 per
 * thread and combines the per-CTA partials in FP64. */
lift_status lift_asum(const float* x, int64_t n, float* result, void* stream);

/* dot: *result = sum_i x_i * y_i (Fig. 5: reduce(add,0) . map(mult) . zip). */
lift_status lift_dot(const float* x, const float* y, int64_t n, float* result, void* stream);

/* scal: y_i = alpha * x_i, one correctly rounded fp32 multiply per element
 * (Fig. 5 and Fig. 2: map(mult(alpha))).  y == x (in place) is allowed;
 * other overlaps are not. */
lift_status lift_scal(int64_t n, float alpha, const float* x, float* y, void* stream);

/* gemv: y_i <- alpha * sum_j A[i*lda + j] * x_j + beta * y_i, i < M, j < N
 * (Fig. 5, "as defined by the BLAS library", Sec. 5.1).  A row-major M x N
 * with lda >= N; x: N floats; y: M floats, read only when beta != 0.
 * Per row: z = fl(alpha * dot); y = fl(z + fl(beta * y)). */
lift_status lift_gemv(int64_t M, int64_t N, float alpha, const float* A, int64_t lda,
                      const float* x, float beta, float* y, void* stream);

/* ------------------------------------------------------------------------
 * More programs through the same kernel templates: the code generator of
 * the paper only knows reduce-seq and the maps (Sec. 4.2, "Reduction"), so
 * any user function plugs into the same kernels.
 *   nrm2(x)       = map(sqrt) . reduce(add, 0) . map(square, x):
 *                   sqrt(sum x_i^2), the sum combined in FP64 and its
 *                   correctly rounded FP64 square root rounded once to fp32
 *   sum(x)        = reduce(add, 0)(x)
 *   axpy(a, x, y) = map(add) . zip(map(mult(a), x), y): y_i <- fl(fl(a x_i) + y_i),
 *                   in place in y (y == x allowed; other overlaps are not)
 * Arguments, errors and conventions as for asum / scal.
 * ------------------------------------------------------------------------ */
lift_status lift_nrm2(const float* x, int64_t n, float* result, void* stream);
lift_status lift_sum(const float* x, int64_t n, float* result, void* stream);
lift_status lift_axpy(int64_t n, float alpha, const float* x, float* y, void* stream);
lift_status lift_nrm2_v(int variant, const float* x, int64_t n, float* result, double* result_f64,
                        void* stream);
lift_status lift_sum_v(int variant, const float* x, int64_t n, float* result, double* result_f64,
                       void* stream);
lift_status lift_axpy_v(int variant, int64_t n, float alpha, const float* x, float* y,
                        void* stream);

/* ------------------------------------------------------------------------
 * gemv-T: y_j <- alpha * sum_i A[i*lda + j] * x_i + beta * y_j, j < N, i < M
 * (the transposed gemv; x: M floats, y: N floats, read only when beta !=
 * 0).  In the pattern language the columns of A are the rows of
 * split^M . reorder-stride^N . join(A) (Sec. 3.2), so this is the Fig. 5
 * gemv over a reordered matrix.  Each column is folded in fp32 over RB
 * uniform blocks of rows; the RB block partials are added in fp32, in block
 * order (one-pass variants, by the last CTA of each column block) or by a
 * warp per column, lane l adding partials l, l+32, ... followed by a
 * halving tree over the lanes (two-pass variants, a second kernel); then
 * z_j = fl(alpha * sum), y_j = fl(z_j + fl(beta * y_j)).  M == 0 gives
 * y <- beta * y.  Uses the lift_init workspace (RB * N partial slots and,
 * one pass, one counter per column block).  The staged variants (info
 * stages > 0) copy row segments into shared memory with bulk copies and
 * give the two-pass variants' bits for the same blocks; they run as
 * themselves when A and x are 16-byte aligned and N and lda are multiples
 * of 4, and a call that is not runs the 4-byte-load variant 0 instead.
 * Errors: LIFT_ERR_UNSUPPORTED when RB * N exceeds the workspace; a staged
 * copy wait that runs out records LIFT_ERR_TIMEOUT in the status word
 * (lift_read_status) and leaves the affected y_j NaN.
 * lift_gemv_t_blocks reports the rows per block and the number of blocks a
 * variant uses for an M x N call.
 * ------------------------------------------------------------------------ */
/* lift_gemv_segments: how a gemv variant splits each row.  The split-row
 * variants (names "gemv_split_*"; Fig. 3 partial reduction applied to the
 * row's reduce) give each row *segments CTAs of *seg_len elements (a
 * multiple of the variant's threads x vector width; the last segment is
 * ragged) and add the segment partials in fp32 with a warp per row, lane l
 * adding partials l, l+32, ..., then a halving tree over the lanes; every
 * other gemv variant reports *seg_len = N, *segments = 1.  Host only; needs
 * lift_init for the device (the split depends on its SM count).  Errors:
 * LIFT_ERR_INVALID_ARG for a bad variant, M < 1, N < 0 or NULL outputs. */
lift_status lift_gemv_segments(int variant, int64_t M, int64_t N, int64_t* seg_len,
                               int64_t* segments);

lift_status lift_gemv_t(int64_t M, int64_t N, float alpha, const float* A, int64_t lda,
                        const float* x, float beta, float* y, void* stream);
lift_status lift_gemv_t_v(int variant, int64_t M, int64_t N, float alpha, const float* A,
                          int64_t lda, const float* x, float beta, float* y, void* stream);
lift_status lift_gemv_t_blocks(int variant, int64_t M, int64_t N, int64_t* rows_per_block,
                               int64_t* blocks);

/* ------------------------------------------------------------------------
 * Sharded reductions (the paper has no counterpart; one of the library's
 * uses over several GPUs).  A rank reduces its shard of the vector(s) to
 * one FP64 value -- the FP64 sum of its CTAs' fp32 partials, the value
 * lift_asum / lift_dot round to fp32 -- and the ranks exchange those 8-byte
 * partials (an all-gather: the one data exchange a sharded asum or dot
 * needs).  lift_combine_partials adds the gathered partials in index (rank)
 * order in FP64 and rounds once to fp32, so every rank gets the same result
 * whatever the order the partials arrived in.
 * x, y: the shard (device, n floats); partial: one double (device),
 * written.  partials: `count` doubles (host); result: one float (host);
 * result_f64 (optional, host): the FP64 sum.  The shard calls use the
 * policy's variant and the lift_init workspace; lift_combine_partials is
 * host-only and needs no device.  Errors: LIFT_ERR_INVALID_ARG for bad
 * sizes or NULL pointers.
 * ------------------------------------------------------------------------ */
lift_status lift_asum_partial(const float* x, int64_t n, double* partial, void* stream);
lift_status lift_dot_partial(const float* x, const float* y, int64_t n, double* partial,
                             void* stream);
lift_status lift_combine_partials(const double* partials, int64_t count, float* result,
                                  double* result_f64);

/* ------------------------------------------------------------------------
 * Compensated fp32 asum and dot: the Fig. 5 programs with an error-free
 * fold.  Every term is added to a per-lane (sum, compensation) pair with
 * TwoSum; for dot the product's rounding error, fma(x, y, -fl(x y)), is
 * added to the compensation too (TwoProduct, Ogita, Rump and Oishi 2005).
 * The pairs are merged with TwoSum across lanes, the warp and the CTA, the
 * per-CTA values sum + compensation are added in FP64 and rounded once to
 * fp32.  The result is within about one unit of fp32 roundoff of the exact
 * value (plus a second-order term), also when the sum cancels.
 * x, y: n floats (device); result: one float (device); result_f64
 * (optional): the FP64 value before the rounding.  Arguments, errors and
 * alignment fallback as for lift_asum / lift_dot; uses the lift_init
 * workspace (FP64 partial slots and one counter).
 * ------------------------------------------------------------------------ */
lift_status lift_asum_comp(const float* x, int64_t n, float* result, double* result_f64,
                           void* stream);
lift_status lift_dot_comp(const float* x, const float* y, int64_t n, float* result,
                          double* result_f64, void* stream);
lift_status lift_asum_comp_v(int variant, const float* x, int64_t n, float* result,
                             double* result_f64, void* stream);
lift_status lift_dot_comp_v(int variant, const float* x, const float* y, int64_t n, float* result,
                            double* result_f64, void* stream);

/* ------------------------------------------------------------------------
 * BlackScholes (Sec. 7 "Mathematical Finance Application", Fig. 6):
 * blackScholes(s) = map(BSComputation, s), a {call, put} pair per stock
 * price for European options with strike K, riskless rate r, volatility
 * sigma and maturity T (years) shared by all prices.  The paper does not
 * print compD1 / compD2 / compCall / compPut; they are the Black-Scholes
 * model:
 *   d1 = (ln(S/K) + (r + sigma^2/2) T) / (sigma sqrt T), d2 = d1 - sigma sqrt T
 *   call = S N(d1) - K e^{-rT} N(d2),   put = call - S + K e^{-rT}
 * with N(x) = erfc(-x/sqrt 2)/2, evaluated in fp32 (host-rounded constants
 * 1/K, (r + sigma^2/2) T, sigma sqrt T, 1/(sigma sqrt T), K e^{-rT}).
 * s: n prices (> 0 for a finite result; 0 gives call 0, put K e^{-rT});
 * call, put: n floats each (device), written; none of the three may
 * overlap.  Errors: LIFT_ERR_INVALID_ARG for n < 0, NULL arrays with n > 0,
 * or K, sigma, T not positive and finite, or r not finite.  All variants
 * give bit-identical results.
 * ------------------------------------------------------------------------ */
lift_status lift_blackscholes(int64_t n, const float* s, float strike, float rate, float volatility,
                              float years, float* call, float* put, void* stream);
lift_status lift_blackscholes_v(int variant, int64_t n, const float* s, float strike, float rate,
                                float volatility, float years, float* call, float* put,
                                void* stream);

/* ------------------------------------------------------------------------
 * Explicit variants (the autotuner's interface).  `variant` indexes the
 * op's variant list (0 .. lift_variant_count(op)-1); -1 means "ask the
 * policy".  result_f64 (optional, may be NULL) receives the FP64 value of
 * the final combine before its rounding to fp32.
 * ------------------------------------------------------------------------ */
lift_status lift_asum_v(int variant, const float* x, int64_t n, float* result,
                        double* result_f64, void* stream);
lift_status lift_dot_v(int variant, const float* x, const float* y, int64_t n,
                       float* result, double* result_f64, void* stream);
lift_status lift_scal_v(int variant, int64_t n, float alpha, const float* x, float* y,
                        void* stream);
lift_status lift_gemv_v(int variant, int64_t M, int64_t N, float alpha, const float* A,
                        int64_t lda, const float* x, float beta, float* y, void* stream);

/* Rewrite parameters of one variant.
 *  tile     split^tile: elements a CTA takes per pipeline step (gemv: 0)
 *  vw       asVector^vw: elements per load (1, 4 = 128-bit, 8 = 256-bit)
 *  threads  local threads per CTA (map-local width)
 *  stride   1: reorder-stride (thread t reads vector t + threads*j);
 *           0: contiguous chunk per thread
 *  tree     in-CTA iterate depth: 0 warp shuffles only, 1 + shared memory,
 *           2 + cluster distributed shared memory; gemv: 3 = stages filled
 *           by tensor copies (needs N % 256 == 0); BlackScholes: the normal
 *           distribution (0 erfcf, 1 polynomial, 2 polynomial on
 *           approximate instructions)
 *  cluster  CTAs per cluster (1 = none)
 *  passes   1: last-CTA combine in the same launch; 2: second kernel
 *  stages   0: direct vector loads; k >= 2: k-deep TMA bulk-copy ring
 *  rows     gemv: rows per warp-group step; gemv-T, compensated, mixed
 *           precision, BlackScholes: loads (rows) in flight per work-item
 *  lanes    gemv: threads that share one row (0 otherwise)
 *  final_threads  threads of the FP64 final combine
 *  grid     maps (scal, axpy, BlackScholes): 1 = one CTA per tile, the
 *           grid covers every tile and the hardware deals CTAs to SMs as
 *           earlier ones finish; 0 = a persistent grid (at most the
 *           resident CTAs) that takes the tiles round robin
 */
typedef struct {
  int op, id, tile, vw, threads, stride, tree, cluster, passes, stages, rows, lanes,
      final_threads, grid;
  char name[64];
} lift_variant_info;

int lift_variant_count(int op);
lift_status lift_variant_describe(int op, int id, lift_variant_info* out);

/* CTAs a variant launches for a problem of n elements (gemv: n = M) on
 * the current device -- the map-workgroup width of its expression. */
lift_status lift_variant_grid(int op, int id, int64_t n, int64_t* grid);

/* ------------------------------------------------------------------------
 * Mixed precision (stored bf16, or fp8-e4m3 with one fp32 scale per 4096
 * consecutive elements; the last block may be shorter).
 *   bf16: x is n uint16 bit patterns; xscale must be NULL.
 *   fp8:  x is n uint8 E4M3 bit patterns; xscale holds ceil(n/4096) floats;
 *         element i stands for q_i * xscale[i / 4096].
 * Per-thread fp32 Kahan-compensated sums of the exactly widened values
 * (bf16 -> fp32 is exact; an fp8 product is exact in fp32), one scale
 * multiply per block, FP64 combine across CTAs.  result: one float;
 * result_f64 (optional): the FP64 combine before rounding.
 * ------------------------------------------------------------------------ */
lift_status lift_asum_ex(lift_dtype t, const void* x, const float* xscale, int64_t n,
                         float* result, double* result_f64, void* stream);
lift_status lift_dot_ex(lift_dtype t, const void* x, const float* xscale, const void* y,
                        const float* yscale, int64_t n, float* result, double* result_f64,
                        void* stream);
lift_status lift_asum_ex_v(int variant, lift_dtype t, const void* x, const float* xscale,
                           int64_t n, float* result, double* result_f64, void* stream);
lift_status lift_dot_ex_v(int variant, lift_dtype t, const void* x, const float* xscale,
                          const void* y, const float* yscale, int64_t n, float* result,
                          double* result_f64, void* stream);

/* ------------------------------------------------------------------------
 * Variant policy.
 *   LIFT_POLICY_FIXED: the per-op default variant (or lift_set_variant's).
 *   LIFT_POLICY_TABLE: a tuned table (path: a text file written by the
 *                      autotuner; nearest shape in log2 size).
 *   LIFT_POLICY_MLP:   the cost model (path: weights file written by the
 *                      trainer); argmin of the predicted times.
 *   LIFT_POLICY_MLP_TUNE: the cost model with exhaustive timing as its
 *                      fallback (Sec. 6.2 explores parameter values
 *                      empirically; Sec. 6.3 names a model-guided search).
 *                      A call whose shape lies outside the range the model
 *                      was trained on (the weights file's "box"), or whose
 *                      two best predicted times are within 3 % of each
 *                      other and whose inputs span at least twice the L2,
 *                      has its candidates timed -- the model's 3 best, the
 *                      FIXED default and any variant newer than the model
 *                      -- each as a CUDA graph of 4 back-to-back launches
 *                      replayed 5 times (candidates interleaved, median),
 *                      on a private stream that first waits for the call's
 *                      stream.  The caller's arrays are only read: outputs
 *                      go to scratch (a temporary array of the output's
 *                      size for scal, axpy, BlackScholes, gemv and gemv-T,
 *                      allocated and freed around the timing).  The fastest
 *                      is cached per (op, shape, alignment); the first such
 *                      call waits for the timing (one timing runs at a time;
 *                      other threads' picks do not wait for it).  A call made while its
 *                      stream is being captured into a CUDA graph,
 *                      lift_pick and the batch never time: they use a
 *                      cached winner or the plain learned pick.  Loading
 *                      weights clears the cache.
 * Both learned policies choose only among the variants that run as
 * themselves on the call's arguments (vector loads need the pointers and,
 * for gemv and gemv-T, the row pitch aligned to the vector width); an
 * explicit or FIXED variant that cannot runs its guarded fallback.  Their
 * picks are memoised per (op, shape, pointer and pitch alignment), so a
 * repeated call shape costs a table lookup; loading weights clears the
 * memo.
 * ------------------------------------------------------------------------ */
typedef enum {
  LIFT_POLICY_FIXED = 0,
  LIFT_POLICY_TABLE = 1,
  LIFT_POLICY_MLP = 2,
  LIFT_POLICY_MLP_TUNE = 3
} lift_policy;

lift_status lift_set_policy(int policy, const char* path);
/* LIFT_POLICY_MLP_TUNE bookkeeping: shapes whose winner is cached, and the
 * launches timed so far (both since the process started; either pointer
 * may be NULL).  Host-only. */
lift_status lift_tune_stats(int64_t* tuned_shapes, int64_t* timed_launches);
/* Force `variant` for `op` (-1 clears the override). */
lift_status lift_set_variant(int op, int variant);
/* The variant the current policy would use for a dense call (aligned
 * pointers, lda = N).  M, N: gemv / gemv-T shape (else 0). */
lift_status lift_pick(int op, int64_t n, int64_t M, int64_t N, int* variant);

/* The LIFT_NUM_FEATURES cost-model features of a call, written to
 * out[0..11]: one-hot op family (asum-like one-input reductions: asum,
 * nrm2, sum, compensated asum; dot-like: dot, compensated dot; maps: scal,
 * axpy, BlackScholes; matrices: gemv, gemv-T), log2(n+1)/32, log2(M+1)/16,
 * log2(N+1)/16, one-hot element type (fp32, bf16, fp8), and, gemv and
 * gemv-T only, whether a dense row holds whole 16-byte and whole 32-byte
 * vectors (N % 4 == 0, N % 8 == 0; 0 for the other ops).  For gemv and
 * gemv-T the size feature uses n = M*N.  A weights file with d_in < 12 reads the first
 * d_in.  Host-only; needs no device.  Defined for op ids below LIFT_MLP_OPS
 * (LIFT_ERR_INVALID_ARG otherwise). */
#define LIFT_NUM_FEATURES 12
lift_status lift_features(int op, int64_t n, int64_t M, int64_t N, float* out);

/* ------------------------------------------------------------------------
 * Batched persistent launch: many asum / dot / scal / gemv calls of uneven
 * sizes in one graph-launched persistent kernel with a work queue (map over
 * the batch lowered to map-workgroup over work items).
 *
 * lift_op_desc: one call, with the arguments of the matching single-op
 * entry point (device pointers owned by the caller, valid while the batch
 * runs).  asum / dot: x (and y) of n floats, out = one float.  scal:
 * out[i] = alpha * x[i], n floats.  gemv: out <- alpha * A x + beta * out,
 * A row-major M x N with lda >= N, x of N floats, out of M floats (read
 * only when beta != 0).  variant: a variant id of that op whose tile and
 * vector width the batch adopts, or -1 for the current policy's pick
 * (FIXED, TABLE or MLP) at creation time.
 *
 * lift_batch_create validates every descriptor (op id, variant id, sizes,
 * NULL or unaligned pointers) before touching the device and returns
 * LIFT_ERR_INVALID_ARG naming the first bad op; it then splits each op into
 * work items of about 256 KiB, orders the queue largest item first and
 * copies the descriptors to device memory it allocates (freed by
 * lift_batch_destroy).  Needs lift_init; call it outside stream capture.
 * lift_batch_run launches, on `stream`, a CUDA graph (captured on its first
 * call) made of a memset node that resets the queue head and the per-op
 * counters and the persistent kernel; the results are written when the
 * stream reaches the end of the graph.  Runs of one batch must not overlap.
 * Reduction results are the FP64 sum, rounded once, of per-item fp32
 * partials taken in item order, so they do not depend on scheduling.
 * ------------------------------------------------------------------------ */
typedef struct {
  int op;
  int variant;
  int64_t n, M, N, lda;
  float alpha, beta;
  const float* x;
  const float* y;
  const float* A;
  float* out;
} lift_op_desc;

typedef struct lift_batch lift_batch;

lift_status lift_batch_create(const lift_op_desc* ops, int64_t count, lift_batch** batch);
lift_status lift_batch_run(lift_batch* batch, void* stream);
/* How the work items meet the SMs (map-workgroup over the items, two
 * schedules of the same expression; results are identical):
 *   LIFT_BATCH_QUEUE     a persistent grid (SMs x resident CTAs) whose CTAs
 *                        pop queue positions with an atomic (the default);
 *   LIFT_BATCH_PER_ITEM  one CTA per work item, CTA q taking queue position
 *                        q, dealt to the SMs by the hardware as earlier CTAs
 *                        retire (LIFT_ERR_UNSUPPORTED beyond 2^31 - 1 items).
 * A change takes effect at the next lift_batch_run (the graph is captured
 * again); if the batch has run before, the call first synchronises the
 * device so that no launch of the old graph is in flight. */
#define LIFT_BATCH_QUEUE 0
#define LIFT_BATCH_PER_ITEM 1
lift_status lift_batch_set_schedule(lift_batch* batch, int schedule);
/* The batch's schedule (-1 for a NULL batch). */
int lift_batch_schedule(const lift_batch* batch);
/* Work items, algorithmic bytes of one run, and CTAs of the launch. */
lift_status lift_batch_info(const lift_batch* batch, int64_t* items, int64_t* bytes, int64_t* grid);
/* For op i: the variant the batch adopted, the processing mode it maps to
 * (vector ops: 0..5 = (vector width, vectors per thread per tile) of
 * (1,4) (4,1) (4,2) (4,4) (8,1) (8,2), tile = 256 threads x both; gemv:
 * 0..2 = vector width 1, 4, 8), and the work-item length in elements
 * (gemv: rows).  Any output pointer may be NULL. */
lift_status lift_batch_op_choice(const lift_batch* batch, int64_t i, int* variant, int* mode,
                                 int64_t* item);
/* Synchronises the device, then frees the batch's device memory. */
lift_status lift_batch_destroy(lift_batch* batch);

/* ------------------------------------------------------------------------
 * Cost-model training kernels (FP32).  A multilayer perceptron
 * d_in -> h1 -> h2 -> V (ReLU hidden layers) predicts one log-time per
 * kernel variant from the features of a call (lift_features); it replaces
 * the paper's empirical choice of split sizes and vector widths (Sec. 6.2,
 * and the model-guided search Sec. 6.3 names as future work).
 * All pointers are device pointers owned by the caller; fp32, row-major.
 *   params: W1[d_in][h1] b1[h1] W2[h1][h2] b2[h2] W3[h2][V] b3[V]
 *           (lift_mlp_param_count floats; grads, Adam m and v: same layout)
 *   X: B x d_in features; P: B x V predictions; T, mask: B x V targets and
 *   0/1 weights; work: lift_mlp_work_count(B, h1, h2) floats that hold the
 *   forward activations for the backward pass (Z1 H1 Z2 H2, then two
 *   B x max(h1,h2) gradient buffers).
 * loss = sum(mask * (P - T)^2) * inv_measured (inv_measured = 1 / sum(mask));
 * dP = 2 * mask * (P - T) * inv_measured; Adam as in Kingma and Ba (2015)
 * with bias correction at step t >= 1.
 * ------------------------------------------------------------------------ */
int64_t lift_mlp_param_count(int d_in, int h1, int h2, int V);
int64_t lift_mlp_work_count(int64_t B, int h1, int h2);
lift_status lift_mlp_forward(int d_in, int h1, int h2, int V, const float* params, const float* X,
                             int64_t B, float* work, float* P, void* stream);
lift_status lift_mlp_loss(const float* P, const float* T, const float* mask, int64_t count,
                          float inv_measured, float* dP, float* loss, void* stream);
lift_status lift_mlp_backward(int d_in, int h1, int h2, int V, const float* params,
                              const float* X, int64_t B, float* work, const float* dP,
                              float* grads, void* stream);
lift_status lift_mlp_adam(float* params, const float* grads, float* m, float* v, int64_t count,
                          int t, float lr, float beta1, float beta2, float eps, void* stream);

/* Failure-detection probe (the paper has no counterpart).  Launches, on
 * `stream`, one warp whose first lane waits on an mbarrier that nothing
 * arrives at, giving up after `polls` polls (1 .. 2^22, the limit every
 * staged kernel uses) and recording LIFT_ERR_TIMEOUT in the device status
 * word -- the path a bulk-copy pipeline takes when its copies stall.  Faults
 * nothing and leaves the context usable; read (and clear) the outcome with
 * lift_read_status(1).  Errors: LIFT_ERR_INVALID_ARG for polls out of range,
 * LIFT_ERR_NOT_INITIALIZED without lift_init. */
lift_status lift_wait_probe(uint32_t polls, void* stream);

/* Poll limit of the staged (TMA bulk-copy) reductions' wait on each copy
 * (the paper has no counterpart): 2^22 by default; a failure-detection test
 * lowers it (0 = give up at the first wait) to drive a real reduction down
 * its timeout path without a fault.  A reduction whose wait gives up
 * records LIFT_ERR_TIMEOUT in the status word, waits with the default limit
 * for its copies still in flight, and still completes its cross-CTA
 * combine: its result is NaN and the one-pass ticket returns to 0, so the
 * next call is correct.  Process-wide; applies to launches made after the
 * call.  Errors: LIFT_ERR_INVALID_ARG for polls above 2^22. */
lift_status lift_set_wait_polls(uint32_t polls);

/* ------------------------------------------------------------------------
 * Allocation-free asum.  The paper has no counterpart: this entry point
 * exists for callers that must not have the library allocate device memory
 * -- a process whose device memory belongs to its own pool allocator under
 * a fixed budget, or a latency-critical loop that cannot pay for cudaFree's
 * device-wide synchronisation.  It computes what lift_asum computes (x: n
 * floats, result: one float, both device pointers owned by the caller) and
 * needs no lift_init: its scratch (4096 fp32 partial slots and one ticket
 * word, about 16 KiB) is a fixed array inside the library's device image,
 * held on every GPU that loads the library until the process exits.
 *  - The first call on a device looks up that array's address (with the
 *    device current) and caches it: make the first call before any stream
 *    capture.
 *  - Every call shares the array.  Each call clears the ticket on `stream`
 *    before its kernel; calls whose kernels overlap on the GPU race and
 *    give wrong results, so order them.
 *  - x needs 4-byte alignment only, as for lift_asum: a 16-byte aligned x
 *    is read with 128-bit loads, any other x with 4-byte loads of the same
 *    elements in the same order (the result is the same).
 *  - A launch that would need more than 4096 partial slots returns
 *    LIFT_ERR_UNSUPPORTED; invalid arguments (n < 0, a NULL result, a NULL
 *    x with n > 0, an x not 4-byte aligned) return LIFT_ERR_INVALID_ARG
 *    before any CUDA call.  n == 0 writes 0.
 *  - The cached address belongs to the device's context: after
 *    cudaDeviceReset, call lift_finalize (which forgets it) before the next
 *    call.
 * ------------------------------------------------------------------------ */
lift_status lift_asum_noalloc(const float* x, int64_t n, float* result, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LIFT_H */
