/*
 * oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow CPU reference for the blocked general matrix multiplication of
 * "Automatic Generators for a Family of Matrix Multiplication Routines with
 * Apache TVM" (Alaejos et al.), used to check the GPU library and nothing else.
 * Only tests/, the smoke check and the benchmark's CPU-baseline arm may load it;
 * the GPU library never links, includes or calls it, and it includes nothing
 * from the GPU library.
 *
 * Conventions: all matrices are row-major with explicit leading dimensions,
 * element (i, p) of A at A[i*lda + p], (p, j) of B at B[p*ldb + j], (i, j) of C at
 * C[i*ldc + j].  Sizes are int64_t.  Floating point is IEEE binary64 unless the
 * function name says otherwise.  The library is built with -ffp-contract=off so
 * that x86-64 and aarch64 hosts produce identical bits.
 */
#ifndef G3_ORACLE_H
#define G3_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* --- Definition of the operation (Section 3.1, generalised with alpha/beta;
 *     Section 5.1, the three-loop basic realisation) ---------------------------
 *
 * C_out[r][j] = beta * C_in[i][j] + alpha * sum_{p<k} A[i][p] * B[p][j]
 *
 * for every i in rows[0..nrows) (r is the position of i in rows; rows == NULL
 * means rows = 0..nrows-1) and j < n.  The sum runs over p in increasing order,
 * in binary64.  beta == 0 never reads C_in (NaN there is overwritten);
 * alpha == 0 or k == 0 never reads A or B.  C_out must not alias C_in.
 * nthreads <= 0 uses every OpenMP thread; threads split whole rows only, so the
 * result does not depend on the thread count.                               */
void oracle_gemm_rows_f64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                          double alpha, const double* A, int64_t lda,
                          const double* B, int64_t ldb, double beta,
                          const double* C_in, int64_t ldc_in,
                          double* C_out, int64_t ldc_out, int nthreads);

/* One entry (i, j) computed as a dot product in the same order as above. */
double oracle_entry_f64(int64_t k, double alpha, const double* A_row,
                        const double* B, int64_t ldb, int64_t j,
                        double beta, double c_in);

/* Error-metric denominator D[r][j] = |alpha| * sum_p |A[i][p]| * |B[p][j]|. */
void oracle_absprod_rows_f64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                             double alpha, const double* A, int64_t lda,
                             const double* B, int64_t ldb,
                             double* D, int64_t ldd, int nthreads);

/* Integer definition for 8-bit integer inputs, exact in int64:
 * C_out[r][j] = beta * C_in[i][j] + alpha * sum_p A[i][p] * B[p][j].
 * beta == 0 never reads C_in.                                               */
void oracle_gemm_rows_i8_i64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                             int64_t alpha, const int8_t* A, int64_t lda,
                             const int8_t* B, int64_t ldb, int64_t beta,
                             const int32_t* C_in, int64_t ldc_in,
                             int64_t* C_out, int64_t ldc_out, int nthreads);

/* The same for 16-bit integer inputs and a 64-bit C (the INT16 entry of the
 * datatype study, Section 8.6), exact in int64 for k < 2^33.               */
void oracle_gemm_rows_i16_i64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                              int64_t alpha, const int16_t* A, int64_t lda,
                              const int16_t* B, int64_t ldb, int64_t beta,
                              const int64_t* C_in, int64_t ldc_in,
                              int64_t* C_out, int64_t ldc_out, int nthreads);

/* --- Convolution --------------------------------------------------------------
 * y := beta*y + alpha*conv(x, w), the convolution layers the paper casts to
 * GEMM (Section 8.1, Table 1), by its definition: x is N x H x W x C (NHWC),
 * w is R x S x C x K, y is N x P x Q x K with P = (H + 2*pad_h - dil_h*(R-1)
 * - 1) / str_h + 1 (Q likewise) and
 *   y[n][p][q][k] = sum over r, s, c of x[n][p*str_h - pad_h + r*dil_h]
 *                                      [q*str_w - pad_w + s*dil_w][c] * w[r][s][c][k],
 * input positions outside the image contributing zero.  Sums in binary64 in
 * the order r, s, c.  Threads over (n, p).                                   */
void oracle_conv2d_nhwc_f64(int64_t N, int64_t H, int64_t W, int64_t C, int64_t K, int64_t R, int64_t S,
                            int64_t str_h, int64_t str_w, int64_t pad_h, int64_t pad_w, int64_t dil_h,
                            int64_t dil_w, double alpha, const double* x, const double* w, double beta,
                            const double* y_in, double* y_out, int nthreads);

/* --- Number formats ---------------------------------------------------------
 * bfloat16: 1 sign, 8 exponent, 7 fraction bits (the top half of a binary32).
 * Round to nearest, ties to even; overflow gives +-Inf; NaN gives the quiet
 * NaN 0x7FC0 with the input's sign dropped.  Returned as the binary32 value. */
float oracle_round_bf16(float x);
void  oracle_round_bf16_array(const float* x, float* y, int64_t count);

/* TF32: binary32's sign and 8-bit exponent with 10 fraction bits.  Round to
 * nearest, ties to even, on the TF32 grid: spacing 2^(E-10) at a normal x of
 * unbiased exponent E, 2^-136 among subnormals; beyond the largest finite
 * TF32 value the result overflows to +-Inf; NaN gives 0x7FC00000.  Returned
 * as the binary32 value. */
float oracle_round_tf32(float x);
void  oracle_round_tf32_array(const float* x, float* y, int64_t count);

/* --- A second FP32-accurate split on TF32 (a further datatype of Section 8.6's
 *     study): x_hi = tf32(x), x_lo = tf32(x - x_hi), both rounded to nearest
 *     even on the TF32 grid (the difference is exact in binary32: x_hi is x
 *     rounded to 11 significant bits).  |x - x_hi - x_lo| <= 2^-22 |x| for
 *     normal x.                                                              */
void oracle_split_tf32(float x, float* hi, float* lo);

/* The 3-product method on the TF32 split, step by step, in binary64:
 * S = sum_p (Ahi*Bhi + Ahi*Blo + Alo*Bhi), the Alo*Blo term dropped;
 * C_out = beta*C_in + alpha*S, for the rows given (as oracle_gemm_rows_f64). */
void oracle_gemm_rows_3xtf32_f64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                                 double alpha, const float* A, int64_t lda,
                                 const float* B, int64_t ldb, double beta,
                                 const double* C_in, int64_t ldc_in,
                                 double* C_out, int64_t ldc_out, int nthreads);

/* OCP FP8 E4M3 ("fn"): 1 sign, 4 exponent (bias 7), 3 fraction bits, no
 * infinities, NaN = S.1111.111, largest finite 448.  Decoding is the format
 * definition; encoding picks the nearest finite value with ties to the even
 * code, and saturates beyond 448 to +-448 ("satfinite").  NaN encodes 0x7F. */
float   oracle_e4m3_decode(uint8_t code);
uint8_t oracle_e4m3_encode(float x);

/* Per-tensor FP8 scaling: amax = max |x|; scale = amax / 448 in binary32
 * (1 when amax == 0); code = e4m3(x / scale) with the quotient in binary32.
 * Rows are `rows` x `cols` with leading dimension ld; q is packed (ld = cols).
 * Returns the scale.                                                         */
float oracle_fp8_quantize(const float* x, int64_t rows, int64_t cols, int64_t ld,
                          uint8_t* q);

/* --- The FP32-accurate split (compensated 3-product bfloat16 split) ----------
 * x_hi = bf16(x), x_lo = bf16(x - x_hi) (the difference is exact in binary32). */
void oracle_split_bf16(float x, float* hi, float* lo);

/* The 3-product method, step by step, in binary64:
 * S = sum_p (Ahi*Bhi + Ahi*Blo + Alo*Bhi), the Alo*Blo term dropped;
 * C_out = beta*C_in + alpha*S.  A and B are the binary32 operands.          */
void oracle_gemm_rows_3xbf16_f64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                                 double alpha, const float* A, int64_t lda,
                                 const float* B, int64_t ldb, double beta,
                                 const double* C_in, int64_t ldc_in,
                                 double* C_out, int64_t ldc_out, int nthreads);

/* Three-part split: hi = bf16(x), mid = bf16(x - hi), lo = bf16((x - hi) - mid),
 * every difference exact in binary32, so that x = hi + mid + lo for normal x. */
void oracle_split3_bf16(float x, float* hi, float* mid, float* lo);

/* The 6-product method on the three-part split, step by step, in binary64:
 * S = sum_p (Ah*Bh + Ah*Bm + Am*Bh + Ah*Bl + Al*Bh + Am*Bm); the products
 * Am*Bl, Al*Bm and Al*Bl (relative size <= 2^-23) are dropped;
 * C_out = beta*C_in + alpha*S.                                               */
void oracle_gemm_rows_6xbf16_f64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                                 double alpha, const float* A, int64_t lda,
                                 const float* B, int64_t ldb, double beta,
                                 const double* C_in, int64_t ldc_in,
                                 double* C_out, int64_t ldc_out, int nthreads);

/* Number of OpenMP threads a call with nthreads <= 0 would use. */
int oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
