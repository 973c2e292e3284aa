/*
 * g3gemm.h -- C ABI of a GB300 (sm_103a) blocked general matrix multiplication.
 *
 * The operation is the one the paper "Automatic Generators for a Family of
 * Matrix Multiplication Routines with Apache TVM" (Alaejos et al.) builds its
 * family of blocked algorithms for (Section 3.1): C = C + A B with A m x k,
 * B k x n, C m x n, generalised to the usual C := beta*C + alpha*A*B.  Every
 * variant of that family computes the same product; they differ in blocking,
 * packing and which operand stays resident where (Sections 3-4, 7).  This
 * library implements the family on one GPU: a plain FP32 kernel on the CUDA
 * cores (the C-resident micro-kernel of Section 4.1) and tensor-core kernels
 * (tcgen05, TMA, TMEM) in several precisions, selected per problem shape in
 * the spirit of the paper's micro-kernel search (Section 8.4).
 *
 * Conventions for every call:
 *   - Matrices are ROW-MAJOR: element (i,p) of A is A[i*lda + p], (p,j) of B is
 *     B[p*ldb + j], (i,j) of C is C[i*ldc + j].  Leading dimensions are in
 *     elements and must satisfy lda >= max(1,k), ldb >= max(1,n),
 *     ldc >= max(1,n).  A column-major caller computes C^T = B^T A^T by
 *     swapping the operands.
 *   - A, B and C are DEVICE pointers owned by the caller; the library never
 *     frees them and keeps no reference after the call returns (a grouped plan
 *     keeps them until it is destroyed).
 *   - Calls are asynchronous on the library's current stream (g3_set_stream)
 *     or on the stream passed explicitly; none synchronises the host except
 *     g3_get_last_device_status and first-use workspace growth.
 *   - Errors: a negative g3_status is returned and nothing is launched.  An
 *     invalid argument at position i (1-based, in the order of the g3_gemm
 *     signature) returns -(100 + i), in the manner of BLAS xerbla.  Device-side
 *     failures (a bounded wait that expired) are recorded in a device status
 *     word and reported by g3_get_last_device_status().
 *   - Edge rules: m == 0 or n == 0 is a no-op; k == 0 or alpha == 0 computes
 *     C := beta*C without reading A or B; beta == 0 never reads C (NaN in C is
 *     overwritten).
 */
#ifndef G3GEMM_H
#define G3GEMM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define G3_API __attribute__((visibility("default")))
#else
#define G3_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetic of a call.  Inputs/outputs per dtype:
 *   G3_F32         A, B, C float32; FP32 FFMA on the CUDA cores.
 *   G3_F32_3XBF16  A, B, C float32; each operand split into hi + lo bfloat16
 *                  parts, C += Ahi*Bhi + Ahi*Blo + Alo*Bhi on the tensor cores
 *                  with FP32 accumulation (the lo*lo term is dropped).  For
 *                  k <= 512 the split has three parts (hi + mid + lo) and six
 *                  products (hi*hi, hi*mid, mid*hi, hi*lo, lo*hi, mid*mid):
 *                  at small k the two-part split's own error is above 2e-6
 *                  of sum |a||b|.  A grouped call applies the same choice
 *                  problem by problem (one persistent launch per kind).
 *   G3_BF16        A, B bfloat16 (raw 16-bit patterns); C float32.
 *   G3_FP8_E4M3    A, B OCP E4M3 bytes with per-tensor scales (g3_gemm_ex);
 *                  C float32 = alpha*scale_a*scale_b*(Aq Bq) + beta*C.
 *   G3_INT8        A, B int8; C int32; alpha must be 1 and beta 0 or 1; exact
 *                  (k <= 131072 so that no int32 overflow is possible).
 *                  Single-CTA tiles read the int8 operands as they are (an
 *                  aligned copy only for rows that are not 16-byte
 *                  multiples) and convert them in the kernel, k split so
 *                  that each split sums at most 1024 products; CTA pairs
 *                  convert them in a pre-pass.
 *   G3_FP16        A, B IEEE binary16 (raw 16-bit patterns); C float32.
 *   G3_TF32        A, B, C float32; A and B rounded to TF32 (10 fraction
 *                  bits, nearest even) by a pre-pass, products on kind::tf32
 *                  with FP32 accumulation.
 *   G3_F32_3XTF32  A, B, C float32; a second FP32-accurate mode: each operand
 *                  split into hi + lo TF32 parts (hi = tf32(x), lo =
 *                  tf32(x - hi): 22 significant bits), C += Ahi*Bhi + Ahi*Blo
 *                  + Alo*Bhi on kind::tf32 with FP32 accumulation (lo*lo is
 *                  dropped; at most 3*2^-22 of |a||b| per product).  Twice
 *                  the tensor time of G3_F32_3XBF16; single GEMMs only (the
 *                  grouped calls take G3_BF16 and G3_F32_3XBF16).
 *   G3_F64         A, B, C float64; FP64 FMA on the CUDA cores (the binary64
 *                  entry of the datatype study); alpha and beta are used in
 *                  binary64.  Single GEMMs only.
 *   G3_INT16       A, B int16; C int64; alpha must be 1 and beta 0 or 1;
 *                  exact (products widened to 64 bits on the CUDA cores).
 *                  Single GEMMs only.
 * The CUDA-core dtypes (G3_F32, G3_F64, G3_INT16) take m up to 65535 row
 * blocks (8 388 480 rows for G3_F32, 4 194 240 for the others) when they
 * compute a product; beyond that a call returns G3_ERR_UNSUPPORTED.        */
typedef enum {
  G3_F32 = 0,
  G3_F32_3XBF16 = 1,
  G3_BF16 = 2,
  G3_FP8_E4M3 = 3,
  G3_INT8 = 4,
  G3_FP16 = 5,
  G3_TF32 = 6,
  G3_F32_3XTF32 = 7,
  G3_F64 = 8,
  G3_INT16 = 9
} g3_dtype;

/* g3_gemm_args.split_k value that asks for a stream-K tail (see there).    */
#define G3_SPLIT_STREAM_K (-1)

typedef enum {
  G3_OK = 0,
  G3_ERR_ARG = -1,          /* generic invalid argument (positional: -(100+i)) */
  G3_ERR_UNSUPPORTED = -2,  /* valid but not supported (e.g. INT8 with alpha != 1) */
  G3_ERR_CUDA = -3,         /* a CUDA runtime call failed */
  G3_ERR_NOMEM = -4,        /* workspace could not be allocated */
  G3_ERR_TIMEOUT = -5,      /* a device-side bounded wait expired */
  G3_ERR_NOT_INIT = -6      /* no usable CUDA device */
} g3_status;

/* C := beta*C + alpha*A*B on the current stream (Section 3.1).
 * `dtype` is a g3_dtype; alpha and beta are converted to float (kept in
 * binary64 for G3_F64).  For
 * G3_FP8_E4M3 the scales are 1; use g3_gemm_ex to pass scales.  May allocate
 * library workspace on first use of a size class (3xBF16 operand planes,
 * split-K partials, re-packed operands).                                   */
G3_API int g3_gemm(int64_t m, int64_t n, int64_t k, double alpha, const void* A, int64_t lda, const void* B,
            int64_t ldb, double beta, void* C, int64_t ldc, int dtype);

/* g3_gemm with A, B and C in HOST memory (row-major, leading dimensions in
 * elements; C is read when beta != 0 and overwritten with the result).  The
 * call copies B to the device, then streams row blocks of A (and C) up while
 * earlier blocks compute and finished blocks of C come back, on two
 * library-owned copy streams ordered against `cuda_stream` (NULL = the
 * current stream).  It returns before the work is done: the host buffers must
 * stay valid and untouched until `cuda_stream` has completed.  Page-locked
 * host memory is needed for the copies to overlap.  The device copies, and
 * the scratch of the row blocks' GEMMs, live in a library buffer of the
 * calling stream (grown on first use of a size), so calls on different
 * streams may overlap: with requests alternating between two streams, one
 * call's uploads run while the other computes.  Up to four streams keep
 * buffers of their own; a fifth takes over the least recently used stream's
 * buffer, after that stream's last call (ordered on the device, no host
 * wait).  Calls on one stream from several host threads at once are not
 * supported.  FP8 runs with unit scales.  Errors as g3_gemm; G3_ERR_NOMEM
 * when the device copies do not fit.                                         */
G3_API int g3_gemm_host(int64_t m, int64_t n, int64_t k, double alpha, const void* A, int64_t lda, const void* B,
                        int64_t ldb, double beta, void* C, int64_t ldc, int dtype, void* cuda_stream);

/* Convolution as an implicit GEMM (the convolution layers the paper casts to
 * GEMM, Section 8.1 / Table 1), without a materialised im2col matrix:
 *   y[n][p][q][k] := beta*y + alpha * sum over r, s, c of
 *       x[n][p*stride_h - pad_h + r*dil_h][q*stride_w - pad_w + s*dil_w][c] * w[r][s][c][k]
 * x: device N x H x W x C (NHWC), w: device R x S x C x K, both BF16 or FP16
 * (dtype G3_BF16 / G3_FP16, raw 16-bit patterns; x 16-byte aligned); y:
 * device float32 N x P x Q x K with P = (H + 2 pad_h - dil_h (R-1) - 1) /
 * stride_h + 1 (Q likewise).  Input positions outside the image count as
 * zero.  It is the GEMM m = N P Q, n = K, k = R S C with A read through a TMA
 * im2col tensor map.  Requires C a multiple of 64, strides 1..8, paddings
 * 0..128; otherwise G3_ERR_UNSUPPORTED.  -101 / -105: bad sizes.          */
G3_API int g3_conv2d(int64_t N, int64_t H, int64_t W, int64_t C, int64_t K, int64_t R, int64_t S, int64_t stride_h,
                     int64_t stride_w, int64_t pad_h, int64_t pad_w, int64_t dil_h, int64_t dil_w, double alpha,
                     const void* x, const void* w, double beta, float* y, int dtype, void* cuda_stream);

/* Set the stream later calls without an explicit stream use (a cudaStream_t;
 * NULL = legacy default stream).  The setting is per process.             */
G3_API int g3_set_stream(void* cuda_stream);

/* Extended arguments.  Fields beyond the g3_gemm signature:
 *   scale_a, scale_b   device pointers to one float each (FP8 per-tensor
 *                      scales; NULL means 1); ignored for other dtypes.
 *   workspace, workspace_bytes   optional caller-owned device scratch; when
 *                      non-NULL and large enough (g3_gemm_workspace_size) the
 *                      call allocates nothing; too small -> G3_ERR_ARG.
 *   config             -1: the planner's choice; otherwise the index of a
 *                      member of the generated kernel family (g3_family_*).
 *                      G3_F32 (the SIMT kernel): the blocking -- 0: 128 x 128
 *                      blocks of C, 1: 64 x 64 blocks, 2 / 3: 128 x 256
 *                      blocks with k-blocks of 8 / 16 (all give the same
 *                      result bit for bit; split_k applies to 64 x 64).
 *   split_k            0: the planner's choice; >= 1 forces that many splits
 *                      (k cut into equal ranges, partial planes of m x n
 *                      reduced by a second kernel); G3_SPLIT_STREAM_K (-1)
 *                      forces a stream-K tail: the tiles that do not fill the
 *                      last wave of the persistent grid are cut along k into
 *                      one equal piece per CTA (segments of bm x bn partial
 *                      tiles added by a fix-up kernel in a fixed order, so
 *                      results are deterministic); where the tiles fill whole
 *                      waves it computes without a split.  The planner
 *                      takes a stream-K tail only on request (or from an
 *                      autotuner record): measured on GB300 it seldom pays.
 *                      FP8 with device scales takes no split-K (a forced
 *                      split is ignored) but may take the stream-K tail.
 *                      G3_F32 (the SIMT kernel): split_k >= 2 (at most 8
 *                      used) cuts k over a thread-block cluster of that many
 *                      CTAs per 64 x 64 block of C, the partial blocks summed
 *                      through distributed shared memory in a fixed order (no
 *                      workspace); 1 forbids it; 0 lets the planner take it
 *                      when fewer 64 x 64 blocks than SMs would run.
 *   raster             0: the planner's choice (8 tile rows; for a claimed
 *                      walk 2-8, as many as keep the band's panels of A
 *                      within 80 MiB of L2); >= 1 the band width (in tiles)
 *                      of the tile walk.  Launches of at least 16 waves of
 *                      tiles claim their tiles in walk order from a counter
 *                      (one int in the workspace, zeroed by a memset before
 *                      the call's first launch) rather than each CTA taking
 *                      every grid-th tile, so that the tiles running at one
 *                      time stay neighbours in the walk and share their
 *                      operand panels in L2; a caller workspace without the
 *                      256 bytes for it (g3_gemm_workspace_size counts them)
 *                      keeps the static walk, as does G3_STATIC_WALK=1 in
 *                      the environment.  Results are the same bit for bit.
 *   trans_a, trans_b   0: A is m x k (lda >= k), B is k x n (ldb >= n);
 *                      1: the operand is stored transposed -- A as k x m
 *                      (lda >= m), B as n x k (ldb >= k) -- and C := beta*C
 *                      + alpha * op(A) op(B) (BLAS transa/transb).
 *                      G3_BF16, G3_FP16 and G3_FP8_E4M3 read a transposed
 *                      operand in place when its base address and row stride
 *                      are 16-byte aligned (and, for A, unless the planner
 *                      takes an FP8 member with 64 rows of A per CTA).  Every
 *                      other case first copies the operand into the
 *                      row-major layout in a library-owned buffer (grown on
 *                      first use, even when `workspace` is given).          */
typedef struct g3_gemm_args {
  int64_t m, n, k;
  double alpha, beta;
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  void* C;
  int64_t ldc;
  int dtype;
  const float* scale_a;
  const float* scale_b;
  void* workspace;
  size_t workspace_bytes;
  int config;
  int split_k;
  int raster;
  int trans_a;
  int trans_b;
} g3_gemm_args;

/* Initialise the optional fields of `args` to their defaults (config = -1,
 * everything else 0/NULL).                                                  */
G3_API void g3_gemm_args_init(g3_gemm_args* args);

/* g3_gemm with the extended arguments on an explicit stream (NULL = the
 * current stream).                                                          */
G3_API int g3_gemm_ex(const g3_gemm_args* args, void* cuda_stream);

/* Bytes of device scratch g3_gemm_ex needs for these arguments with the
 * planner's (or the forced) configuration; 0 when none.  Returns 0 and sets
 * *bytes on success.                                                         */
G3_API int g3_gemm_workspace_size(const g3_gemm_args* args, size_t* bytes);

/* --- Operand preparation (the packing step of Section 5.3) ----------------
 * x: device float32 rows x cols, leading dimension ldx.  Outputs are device
 * buffers owned by the caller with leading dimension ldy (elements).        */

/* y = bfloat16(x), round to nearest even (raw 16-bit patterns).             */
G3_API int g3_convert_bf16(const float* x, int64_t rows, int64_t cols, int64_t ldx, void* y, int64_t ldy,
                    void* cuda_stream);

/* y = x rounded to TF32 (10 fraction bits, nearest even; overflow to +-Inf,
 * NaN to 0x7FC00000), stored as float32: the pre-pass of G3_TF32.          */
G3_API int g3_convert_tf32(const float* x, int64_t rows, int64_t cols, int64_t ldx, float* y, int64_t ldy,
                           void* cuda_stream);

/* hi = bf16(x), lo = bf16(x - hi): the split of the FP32-accurate mode.     */
G3_API int g3_split_bf16(const float* x, int64_t rows, int64_t cols, int64_t ldx, void* hi, void* lo, int64_t ldy,
                  void* cuda_stream);

/* hi = tf32(x), lo = tf32(x - hi) (nearest even on the TF32 grid, stored as
 * float32; the difference is exact): the split of G3_F32_3XTF32.  Errors as
 * g3_split_bf16.                                                            */
G3_API int g3_split_tf32(const float* x, int64_t rows, int64_t cols, int64_t ldx, float* hi, float* lo, int64_t ldy,
                         void* cuda_stream);

/* hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid): the three-part
 * split the FP32-accurate mode uses for k <= 512 (both differences are exact
 * in FP32).  Errors as g3_split_bf16; -106 / -107: mid / lo is null.        */
G3_API int g3_split3_bf16(const float* x, int64_t rows, int64_t cols, int64_t ldx, void* hi, void* mid, void* lo,
                          int64_t ldy, void* cuda_stream);

/* Per-tensor E4M3 quantisation: scale = amax|x| / 448 (1 when x == 0),
 * q = e4m3_satfinite(x / scale) with the quotient rounded in float32.
 * `scale` is a device float written by the call; q has leading dimension ldq. */
G3_API int g3_quantize_fp8(const float* x, int64_t rows, int64_t cols, int64_t ldx, uint8_t* q, int64_t ldq,
                    float* scale, void* cuda_stream);

/* --- Grouped GEMM: many independent problems in one persistent launch ------
 * One descriptor per problem, same conventions as g3_gemm; all problems of a
 * call share one dtype: G3_BF16, G3_F32_3XBF16 or G3_FP8_E4M3 (C float32).
 * scale_a, scale_b: the per-tensor scales of a G3_FP8_E4M3 problem (host
 * values, finite and > 0: C := beta*C + alpha*scale_a*scale_b*A*B over the
 * decoded E4M3 codes); ignored by the other dtypes.                          */
typedef struct g3_gemm_desc {
  int64_t m, n, k;
  int64_t lda, ldb, ldc;
  double alpha, beta;
  const void* A;
  const void* B;
  void* C;
  float scale_a, scale_b;
} g3_gemm_desc;

typedef struct g3_grouped_plan g3_grouped_plan;

/* Validate the descriptors, bucket the shapes, encode the per-problem tensor
 * maps into a device table and allocate the plan's workspace.  Synchronous.
 * The caller must keep A, B, C of every problem alive until the plan is
 * destroyed.  Descriptor i with an invalid field (including, for
 * G3_FP8_E4M3, a scale that is not finite and > 0) returns -(100 + i)
 * clipped to G3_ERR_ARG for i >= 900.                                       */
G3_API int g3_grouped_plan_create(int count, const g3_gemm_desc* descs, int dtype, g3_grouped_plan** plan);

/* g3_grouped_plan_create with options.  flags = 0 (the same plan) or
 * G3_GROUPED_SPLIT_IN_KERNEL: a G3_F32_3XBF16 plan splits inside the grouped
 * kernels -- warps of the kernel read each tile's FP32 A and B (row-major,
 * any alignment) and write their bfloat16 parts (the two-part split for
 * k > 512, the three-part split for k <= 512, the pre-pass's arithmetic)
 * into shared memory, on tiles of 64 rows -- so the plan holds no operand
 * planes and runs no split pass (the paper's packing, Section 5.3, done in
 * the kernel).  Results equal the default plan's bit for bit where both take
 * 64-row tiles.  The default plan is faster on GB300 (the split-in-kernel
 * warps cannot keep enough loads in flight within their registers); the
 * option serves memory budgets that cannot hold the planes.  Other dtypes
 * ignore the flag; other flag bits: G3_ERR_ARG.                             */
#define G3_GROUPED_SPLIT_IN_KERNEL 1
G3_API int g3_grouped_plan_create_ex(int count, const g3_gemm_desc* descs, int dtype, int flags,
                                     g3_grouped_plan** plan);

/* Run every problem of the plan: pre-passes (if any) and one persistent
 * kernel launch per kernel kind (BF16, FP8: one; FP32-accurate: one for the
 * problems with k > 512 and one for those with k <= 512).  A plan with two
 * kinds that both have split jobs runs the first kind (its jobs and launch)
 * on a stream of its own, forked from `cuda_stream` by an event and joined
 * back into it before the call returns, beside the second kind's; all of the
 * plan's work is ordered on `cuda_stream`.  No
 * host synchronisation and no allocation, so the call can be captured into
 * a CUDA graph.                                                             */
G3_API int g3_grouped_plan_execute(g3_grouped_plan* plan, void* cuda_stream);

G3_API int g3_grouped_plan_destroy(g3_grouped_plan* plan);

/* Introspection: the tile height (64 or 128 rows) and kernel kind (0: the
 * plan's first launch -- BF16, FP8 or the FP32-accurate two-part split; 1:
 * the three-part split) of problem `index`; both -1 for a problem without
 * products.  -101: plan is NULL; -102: index out of range.                  */
G3_API int g3_grouped_plan_describe(const g3_grouped_plan* plan, int index, int* bm, int* kind);

/* Per-bucket selection for grouped plans (the paper's Section 8.4 search,
 * applied to the grouped kernel): times a plan of problems of shape
 * m x n x k (dtype as g3_grouped_plan_create) with every problem on tiles of
 * 64 and of 128 rows -- each a CUDA graph of back-to-back executions over
 * scratch operands the call allocates and frees -- and records the faster
 * height for the size bucket (dtype, ceil(log2) of m, n, k).  Plans created
 * later take that height for every problem in the bucket instead of the
 * fixed rule (64 rows for m <= 64, 128 above).  The records live in the
 * tuning cache (saved, loaded and cleared with the g3_tune_cache_* calls).
 * Outputs (any may be NULL): the height, its time per execution in ms.
 * Synchronous; allocates.  -101..-104: bad m, n, k, dtype.                  */
G3_API int g3_autotune_grouped(int64_t m, int64_t n, int64_t k, int dtype, int* best_bm, double* best_ms);

/* Convenience: create, execute, destroy (synchronises on destroy).          */
G3_API int g3_gemm_grouped(int count, const g3_gemm_desc* descs, int dtype, void* cuda_stream);

/* --- Status, introspection, timing ----------------------------------------*/

/* Synchronise the device, return G3_ERR_TIMEOUT if any kernel since the last
 * call reported an expired wait (G3_OK otherwise) and clear the word.  The
 * raw device code is stored in *code when code != NULL: 0x101-0x105 name the
 * wait that expired (producer, MMA stage, MMA accumulator, epilogue, drain);
 * 0x106: the two CTAs of a CTA-pair member were given different TMEM
 * addresses, and the kernel did no work; 0x107: the wait for a claimed tile
 * number (or for a free entry of the queue that passes it on).              */
G3_API int g3_get_last_device_status(int* code);

G3_API const char* g3_status_string(int status);

/* Number of members of the generated tensor-core kernel family, and a
 * one-line description ("mode=bf16 bm=256 bn=128 stages=4 smem=197888 bufs=2
 * cg=1"; cg = 2: a CTA-pair member with 256-column tiles) of member `index`
 * written to buf (NUL-terminated, truncated to len).                        */
G3_API int g3_family_size(void);
G3_API int g3_family_describe(int index, char* buf, size_t len);

/* Which configuration the planner picks for a problem (index into the family,
 * split count -- G3_SPLIT_STREAM_K when it takes a stream-K tail --, raster
 * band); -1 in *config for the CUDA-core kernels (G3_F32, G3_F64,
 * G3_INT16), with *split_k the FP32 SIMT kernel's cluster split (1: none).  */
G3_API int g3_plan_query(int64_t m, int64_t n, int64_t k, int dtype, int* config, int* split_k, int* raster);

/* --- Autotuner: the per-shape search of the paper's Section 8.4 -------------
 * g3_autotune times every member of the generated family that applies to
 * `dtype`, each with split-K in {1, stream-K, 2, 3, 4, 6, 8, 12, 16} (bounded by the
 * k-blocks), on scratch operands of shape m x n x k it allocates and frees,
 * and records the fastest (member, split) for the shape's size bucket: dtype
 * and ceil(log2) of each of m, n, k.  Later g3_gemm calls in that bucket use
 * the record instead of the planner's model.  Each candidate is timed as
 * calls run inside a captured network: a CUDA graph of back-to-back calls
 * over copies of the operands that together exceed four times the L2 cache,
 * replayed; the time per call is reported.  Synchronous; allocates.
 * Outputs (any may be NULL): the member index, the split count, its time in
 * ms.  The CUDA-core dtypes (G3_F32, G3_F64, G3_INT16) are not timed:
 * *best_config = -1, *best_split = the planner's choice (for G3_F32 the SIMT
 * kernel's cluster split, as g3_plan_query reports), *best_ms = 0.
 * g3_tune_cache_save / load write and read the records as text ("dtype
 * log2(m) log2(n) log2(k) member split ms" per line); the environment variable
 * G3_TUNE_CACHE names a file loaded on first planning.  clear forgets all.   */
G3_API int g3_autotune(int64_t m, int64_t n, int64_t k, int dtype, int* best_config, int* best_split,
                       double* best_ms);
G3_API int g3_tune_cache_save(const char* path);
G3_API int g3_tune_cache_load(const char* path);
G3_API int g3_tune_cache_clear(void);

/* Kernel launches issued by the library since the process started.         */
G3_API uint64_t g3_launch_count(void);

/* Memory-traffic yardstick (no counterpart in the paper): one streaming
 * kernel that reads in_bytes from `in` and writes out_bytes to `out` (device
 * buffers, 16-byte aligned, sizes multiples of 16 and at most 32 GiB), the two streams
 * interleaved in their own proportion, on `cuda_stream` (NULL = the current
 * stream).  Timing it gives the rate HBM sustains for a given read/write mix
 * -- the floor of a memory-bound GEMM with the same mix (on GB300 a stream
 * with twice as many bytes written as read moves fewer bytes per second than
 * either alone).  The data written are filler; `in` is only read.
 * -101..-104: bad in, in_bytes, out, out_bytes.                             */
G3_API int g3_stream_traffic(const void* in, int64_t in_bytes, void* out, int64_t out_bytes, void* cuda_stream);

/* Device allocations (cudaMalloc calls that succeeded) the library has made
 * since the process started, on all devices: workspace growth, transpose and
 * host-entry buffers, grouped plans and the autotuner's scratch operands.
 * Lets a caller (or a test) confirm that a sequence of calls allocated
 * nothing, e.g. g3_gemm_3xbf16_noalloc.                                      */
G3_API int64_t g3_debug_device_allocations(void);

/* When enabled, the library brackets its main GEMM kernel launch with CUDA
 * events on the launching stream; g3_kernel_time_ms returns (after
 * synchronising) the summed device time of those kernels since the last
 * reset and the number of launches timed.                                   */
G3_API int g3_kernel_timing(int enable);
G3_API int g3_kernel_time_ms(double* total_ms, int* launches, int reset);

/* Failure-detection test hook.  The next tensor-core GEMM launch withholds
 * the producer's arrive on its first k-block, so the MMA thread's bounded
 * wait expires after timeout_ms (1..10000): the kernel records the watchdog
 * code, every role leaves its loop, in-flight copies and MMAs are drained and
 * TMEM is freed; nothing hangs or faults.  That call's C is left undefined and
 * g3_get_last_device_status() then returns G3_ERR_TIMEOUT.                   */
G3_API int g3_debug_withhold_next(int64_t timeout_ms);

/* --- Allocation-free FP32-accurate GEMM -------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that may not allocate device memory themselves or through the library:
 * applications whose framework owns all device memory and hands it out from
 * its own pool, processes held to a fixed memory budget, and code that must
 * not risk the device-wide synchronisation a cudaMalloc or cudaFree can cause.
 *
 * Computes the same C := beta*C + alpha*A*B as g3_gemm(..., G3_F32_3XBF16)
 * (float32 A, B, C on the device, same layout rules, same argument errors),
 * without split-K, on `cuda_stream` (NULL = the current stream).  The hi/lo
 * bfloat16 copies of A and B are kept in a 64 MiB array built into the library
 * instead of allocated workspace; the call issues no cudaMalloc, cudaFree or
 * other allocating routine.  Limit: the bfloat16 planes of A and B, each
 * plane rounded up to 256 bytes, must fit in 64 MiB; that is
 *   4 * (m * ceil8(k) + k * ceil8(n)) bytes for k > 512 (hi and lo planes,
 *       e.g. m = n = k = 2800), and
 *   6 * (m * ceil8(k) + k * ceil8(n)) bytes for k <= 512 (the three-part
 *       split the FP32-accurate mode takes there: hi, mid and lo planes),
 * and k <= 32768 (beyond it g3_gemm splits k to keep the FP32 accumulation
 * within 2e-6, which needs workspace); other problems return
 * G3_ERR_UNSUPPORTED before anything is launched.
 *
 * - The first call on a device looks up that device's copy of the array; make
 *   that first call before any stream capture.
 * - Every call, on every stream, uses the same array, and the array keeps the
 *   previous call's contents.  Nothing in it has to start at zero: each call
 *   writes every byte it later reads.  Two calls whose work overlaps on the
 *   GPU (e.g. on two streams without ordering between them) race on the
 *   array and corrupt each other's results.
 * - Every GPU that loads the library holds the 64 MiB until the process exits. */
G3_API int g3_gemm_3xbf16_noalloc(int64_t m, int64_t n, int64_t k, double alpha, const float* A, int64_t lda,
                                  const float* B, int64_t ldb, double beta, float* C, int64_t ldc,
                                  void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* G3GEMM_H */
