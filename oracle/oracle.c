/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Everything here is written from the definitions it cites, with no blocking,
 * packing or reordering: the paper's point is that every member of its family
 * of blocked algorithms computes the same product as the three-loop basic
 * realisation of Section 5.1, differing only in rounding order.  This file is
 * that basic realisation (in binary64, or int64 for integer inputs) plus the
 * number-format conversions the GPU path's precision modes need.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * (closed forms, brute force, a library routine, exhaustive format tables).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int threads_for(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(void) { return threads_for(0); }

static int64_t row_index(const int64_t* rows, int64_t r) { return rows ? rows[r] : r; }

/* Section 3.1 (C = C + AB, A m x k, B k x n) with the alpha/beta scaling of the
 * general routine; Section 5.1 gives the loop nest i -> j -> p.  Here the p loop
 * is hoisted above j so that a row of B is streamed, but every C(i,j) still
 * accumulates its own products in increasing p: the same sum, bit for bit, as
 * oracle_entry_f64 below (tests check that they agree exactly).              */
void oracle_gemm_rows_f64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                          double alpha, const double* A, int64_t lda,
                          const double* B, int64_t ldb, double beta,
                          const double* C_in, int64_t ldc_in,
                          double* C_out, int64_t ldc_out, int nthreads) {
    if (nrows <= 0 || n <= 0) return;
    int nt = threads_for(nthreads);
#pragma omp parallel num_threads(nt)
    {
        double* acc = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = row_index(rows, r);
            for (int64_t j = 0; j < n; ++j) acc[j] = 0.0;
            if (alpha != 0.0) {
                for (int64_t p = 0; p < k; ++p) {
                    double a = A[i * lda + p];
                    const double* brow = B + p * ldb;
                    for (int64_t j = 0; j < n; ++j) acc[j] += a * brow[j];
                }
            }
            double* crow = C_out + r * ldc_out;
            for (int64_t j = 0; j < n; ++j) {
                double ab = (alpha != 0.0) ? alpha * acc[j] : 0.0;
                double bc = (beta != 0.0) ? beta * C_in[i * ldc_in + j] : 0.0;
                crow[j] = bc + ab;
            }
        }
        free(acc);
    }
}

double oracle_entry_f64(int64_t k, double alpha, const double* A_row,
                        const double* B, int64_t ldb, int64_t j,
                        double beta, double c_in) {
    double s = 0.0;
    if (alpha != 0.0)
        for (int64_t p = 0; p < k; ++p) s += A_row[p] * B[p * ldb + j];
    double ab = (alpha != 0.0) ? alpha * s : 0.0;
    double bc = (beta != 0.0) ? beta * c_in : 0.0;
    return bc + ab;
}

/* Denominator of the error metric max |C - C_ref| / (|alpha| |A| |B|). */
void oracle_absprod_rows_f64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                             double alpha, const double* A, int64_t lda,
                             const double* B, int64_t ldb,
                             double* D, int64_t ldd, int nthreads) {
    if (nrows <= 0 || n <= 0) return;
    int nt = threads_for(nthreads);
    double aa = fabs(alpha);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = row_index(rows, r);
        double* drow = D + r * ldd;
        for (int64_t j = 0; j < n; ++j) drow[j] = 0.0;
        for (int64_t p = 0; p < k; ++p) {
            double a = fabs(A[i * lda + p]);
            const double* brow = B + p * ldb;
            for (int64_t j = 0; j < n; ++j) drow[j] += a * fabs(brow[j]);
        }
        for (int64_t j = 0; j < n; ++j) drow[j] *= aa;
    }
}

/* Integer form of the same definition; exact because |A B| <= 2^14 and
 * k <= 2^40 keeps every partial sum far inside int64.                        */
void oracle_gemm_rows_i8_i64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                             int64_t alpha, const int8_t* A, int64_t lda,
                             const int8_t* B, int64_t ldb, int64_t beta,
                             const int32_t* C_in, int64_t ldc_in,
                             int64_t* C_out, int64_t ldc_out, int nthreads) {
    if (nrows <= 0 || n <= 0) return;
    int nt = threads_for(nthreads);
#pragma omp parallel num_threads(nt)
    {
        int64_t* acc = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = row_index(rows, r);
            for (int64_t j = 0; j < n; ++j) acc[j] = 0;
            for (int64_t p = 0; p < k; ++p) {
                int64_t a = A[i * lda + p];
                const int8_t* brow = B + p * ldb;
                for (int64_t j = 0; j < n; ++j) acc[j] += a * (int64_t)brow[j];
            }
            int64_t* crow = C_out + r * ldc_out;
            for (int64_t j = 0; j < n; ++j) {
                int64_t bc = (beta != 0) ? beta * (int64_t)C_in[i * ldc_in + j] : 0;
                crow[j] = bc + alpha * acc[j];
            }
        }
        free(acc);
    }
}

void oracle_gemm_rows_i16_i64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                              int64_t alpha, const int16_t* A, int64_t lda,
                              const int16_t* B, int64_t ldb, int64_t beta,
                              const int64_t* C_in, int64_t ldc_in,
                              int64_t* C_out, int64_t ldc_out, int nthreads) {
    if (nrows <= 0 || n <= 0) return;
    int nt = threads_for(nthreads);
#pragma omp parallel num_threads(nt)
    {
        int64_t* acc = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = row_index(rows, r);
            for (int64_t j = 0; j < n; ++j) acc[j] = 0;
            for (int64_t p = 0; p < k; ++p) {
                int64_t a = A[i * lda + p];
                const int16_t* brow = B + p * ldb;
                for (int64_t j = 0; j < n; ++j) acc[j] += a * (int64_t)brow[j];
            }
            int64_t* crow = C_out + r * ldc_out;
            for (int64_t j = 0; j < n; ++j) {
                int64_t bc = (beta != 0) ? beta * C_in[i * ldc_in + j] : 0;
                crow[j] = bc + alpha * acc[j];
            }
        }
        free(acc);
    }
}

/* ---------------------------------------------------------------------------
 * Number formats, written from their bit-level definitions.                   */

static uint32_t f32_bits(float x) { uint32_t u; memcpy(&u, &x, 4); return u; }
static float f32_from(uint32_t u) { float x; memcpy(&x, &u, 4); return x; }

/* bfloat16 keeps the top 16 bits of a binary32.  The bit patterns of binary32
 * magnitudes are ordered like the magnitudes, so rounding the magnitude to a
 * multiple of 0x10000 is rounding the value: the truncated pattern is the
 * neighbour towards zero, the truncated pattern + 0x10000 the neighbour away
 * from zero (0x7F7F0000 + 0x10000 is +Inf: overflow).  Pick the nearer one,
 * and on an exact tie the one whose last kept bit is 0 (even).               */
float oracle_round_bf16(float x) {
    if (isnan(x)) return f32_from(0x7FC00000u);
    uint32_t u = f32_bits(x);
    uint32_t kept = u & 0xFFFF0000u;
    uint32_t dropped = u & 0x0000FFFFu;
    int away = dropped > 0x8000u || (dropped == 0x8000u && (kept & 0x10000u));
    if (away) kept += 0x10000u;
    return f32_from(kept);
}

void oracle_round_bf16_array(const float* x, float* y, int64_t count) {
    for (int64_t i = 0; i < count; ++i) y[i] = oracle_round_bf16(x[i]);
}

void oracle_conv2d_nhwc_f64(int64_t N, int64_t H, int64_t W, int64_t C, int64_t K, int64_t R, int64_t S,
                            int64_t str_h, int64_t str_w, int64_t pad_h, int64_t pad_w, int64_t dil_h,
                            int64_t dil_w, double alpha, const double* x, const double* w, double beta,
                            const double* y_in, double* y_out, int nthreads) {
    const int64_t P = (H + 2 * pad_h - dil_h * (R - 1) - 1) / str_h + 1;
    const int64_t Q = (W + 2 * pad_w - dil_w * (S - 1) - 1) / str_w + 1;
    const int nt = threads_for(nthreads);
#pragma omp parallel for num_threads(nt) collapse(2) schedule(dynamic)
    for (int64_t n = 0; n < N; ++n) {
        for (int64_t p = 0; p < P; ++p) {
            for (int64_t q = 0; q < Q; ++q) {
                double* out = y_out + ((n * P + p) * Q + q) * K;
                for (int64_t k = 0; k < K; ++k) out[k] = 0.0;
                for (int64_t r = 0; r < R; ++r) {
                    const int64_t h = p * str_h - pad_h + r * dil_h;
                    if (h < 0 || h >= H) continue;
                    for (int64_t s = 0; s < S; ++s) {
                        const int64_t v = q * str_w - pad_w + s * dil_w;
                        if (v < 0 || v >= W) continue;
                        const double* xp = x + ((n * H + h) * W + v) * C;
                        const double* wp = w + (r * S + s) * C * K;
                        for (int64_t c = 0; c < C; ++c)
                            for (int64_t k = 0; k < K; ++k) out[k] += xp[c] * wp[c * K + k];
                    }
                }
                const double* yin = y_in ? y_in + ((n * P + p) * Q + q) * K : NULL;
                for (int64_t k = 0; k < K; ++k)
                    out[k] = alpha * out[k] + (yin && beta != 0.0 ? beta * yin[k] : 0.0);
            }
        }
    }
}

/* TF32 rounding written from the number grid: q = x / spacing rounded to the
 * nearest integer (rint: ties to even in the default rounding mode), then
 * q * spacing; both steps are exact in binary64. */
float oracle_round_tf32(float x) {
    if (isnan(x)) return f32_from(0x7FC00000u);
    if (isinf(x) || x == 0.0f) return x;
    int e;
    frexp((double)x, &e);              /* |x| = f * 2^e with f in [0.5, 1) */
    int E = e - 1;                     /* unbiased exponent of x */
    if (E < -126) E = -126;            /* subnormals share the smallest spacing */
    const double spacing = ldexp(1.0, E - 10);
    const double r = rint((double)x / spacing) * spacing;
    if (fabs(r) >= ldexp(1.0, 128)) return x > 0 ? f32_from(0x7F800000u) : f32_from(0xFF800000u);
    return (float)r;
}

void oracle_round_tf32_array(const float* x, float* y, int64_t count) {
    for (int64_t i = 0; i < count; ++i) y[i] = oracle_round_tf32(x[i]);
}

/* OCP 8-bit floating point, E4M3: exponent bias 7, subnormals m * 2^-9,
 * S.1111.111 is NaN (there is no infinity).                                  */
float oracle_e4m3_decode(uint8_t code) {
    int sign = code >> 7;
    int e = (code >> 3) & 0xF;
    int f = code & 0x7;
    double v;
    if (e == 0xF && f == 0x7) return f32_from(0x7FC00000u);
    if (e == 0) v = ldexp((double)f, -9);
    else v = ldexp(1.0 + f / 8.0, e - 7);
    return (float)(sign ? -v : v);
}

/* Nearest finite E4M3 value by search over the 127 non-negative finite codes
 * (0x00 .. 0x7E, whose values increase with the code); ties go to the even
 * code, i.e. the one with fraction LSB 0.  Anything at or beyond 448 gives
 * 448 (the "satfinite" rule).                                                */
uint8_t oracle_e4m3_encode(float x) {
    if (isnan(x)) return 0x7F;
    uint8_t sign = signbit(x) ? 0x80 : 0x00;
    double a = fabs((double)x);
    if (a >= 448.0) return (uint8_t)(sign | 0x7E);
    /* largest code c with value(c) <= a; values are exact in binary64 */
    int lo = 0;
    for (int c = 1; c <= 0x7E; ++c)
        if ((double)oracle_e4m3_decode((uint8_t)c) <= a) lo = c;
        else break;
    if (lo == 0x7E) return (uint8_t)(sign | 0x7E);
    double vlo = oracle_e4m3_decode((uint8_t)lo);
    double vhi = oracle_e4m3_decode((uint8_t)(lo + 1));
    double dlo = a - vlo, dhi = vhi - a;
    int pick;
    if (dlo < dhi) pick = lo;
    else if (dhi < dlo) pick = lo + 1;
    else pick = (lo % 2 == 0) ? lo : lo + 1;
    return (uint8_t)(sign | pick);
}

float oracle_fp8_quantize(const float* x, int64_t rows, int64_t cols, int64_t ld,
                          uint8_t* q) {
    float amax = 0.0f;
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) {
            float a = fabsf(x[i * ld + j]);
            if (a > amax) amax = a;
        }
    float scale = (amax > 0.0f) ? amax / 448.0f : 1.0f;
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) {
            float t = x[i * ld + j] / scale;   /* binary32 quotient */
            q[i * cols + j] = oracle_e4m3_encode(t);
        }
    return scale;
}

void oracle_split_bf16(float x, float* hi, float* lo) {
    float h = oracle_round_bf16(x);
    float d = x - h;   /* exact in binary32: h is x rounded to 8 significant bits */
    *hi = h;
    *lo = oracle_round_bf16(d);
}

void oracle_split3_bf16(float x, float* hi, float* mid, float* lo) {
    float h = oracle_round_bf16(x);
    float d = x - h;              /* exact: h is x rounded to 8 significant bits */
    float m = oracle_round_bf16(d);
    float e = d - m;              /* exact: m is d rounded to 8 significant bits */
    *hi = h;
    *mid = m;
    *lo = oracle_round_bf16(e);
}

/* The 6-product method: 1) split both operands in three, 2) form the six
 * kept products per term, 3) sum over p.  Products are exact in binary64.    */
void oracle_gemm_rows_6xbf16_f64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                                 double alpha, const float* A, int64_t lda,
                                 const float* B, int64_t ldb, double beta,
                                 const double* C_in, int64_t ldc_in,
                                 double* C_out, int64_t ldc_out, int nthreads) {
    if (nrows <= 0 || n <= 0) return;
    int nt = threads_for(nthreads);
    size_t kn = (size_t)(k > 0 ? k : 1) * (size_t)n;
    double* Bh = (double*)malloc(sizeof(double) * kn);
    double* Bm = (double*)malloc(sizeof(double) * kn);
    double* Bl = (double*)malloc(sizeof(double) * kn);
    for (int64_t p = 0; p < k; ++p)
        for (int64_t j = 0; j < n; ++j) {
            float h, m, l;
            oracle_split3_bf16(B[p * ldb + j], &h, &m, &l);
            Bh[p * n + j] = h;
            Bm[p * n + j] = m;
            Bl[p * n + j] = l;
        }
#pragma omp parallel num_threads(nt)
    {
        double* acc = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = row_index(rows, r);
            for (int64_t j = 0; j < n; ++j) acc[j] = 0.0;
            if (alpha != 0.0) {
                for (int64_t p = 0; p < k; ++p) {
                    float h, m, l;
                    oracle_split3_bf16(A[i * lda + p], &h, &m, &l);
                    double ah = h, am = m, al = l;
                    const double* bh = Bh + p * n;
                    const double* bm = Bm + p * n;
                    const double* bl = Bl + p * n;
                    for (int64_t j = 0; j < n; ++j)
                        acc[j] += ah * bh[j] + ah * bm[j] + am * bh[j] + ah * bl[j] + al * bh[j] + am * bm[j];
                }
            }
            double* crow = C_out + r * ldc_out;
            for (int64_t j = 0; j < n; ++j) {
                double ab = (alpha != 0.0) ? alpha * acc[j] : 0.0;
                double bc = (beta != 0.0) ? beta * C_in[i * ldc_in + j] : 0.0;
                crow[j] = bc + ab;
            }
        }
        free(acc);
    }
    free(Bh);
    free(Bm);
    free(Bl);
}

/* The compensated 3-product split, in the order the method takes it:
 * 1) split both operands, 2) form the three products per term, 3) sum over p.
 * Each product of two bfloat16 values is exact in binary64, so S differs from
 * the exact 3-product sum only by binary64 additions.                        */
void oracle_gemm_rows_3xbf16_f64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                                 double alpha, const float* A, int64_t lda,
                                 const float* B, int64_t ldb, double beta,
                                 const double* C_in, int64_t ldc_in,
                                 double* C_out, int64_t ldc_out, int nthreads) {
    if (nrows <= 0 || n <= 0) return;
    int nt = threads_for(nthreads);
    /* split B once: k x n hi and lo planes */
    double* Bh = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1) * (size_t)n);
    double* Bl = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1) * (size_t)n);
    for (int64_t p = 0; p < k; ++p)
        for (int64_t j = 0; j < n; ++j) {
            float h, l;
            oracle_split_bf16(B[p * ldb + j], &h, &l);
            Bh[p * n + j] = h;
            Bl[p * n + j] = l;
        }
#pragma omp parallel num_threads(nt)
    {
        double* acc = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = row_index(rows, r);
            for (int64_t j = 0; j < n; ++j) acc[j] = 0.0;
            if (alpha != 0.0) {
                for (int64_t p = 0; p < k; ++p) {
                    float ah_f, al_f;
                    oracle_split_bf16(A[i * lda + p], &ah_f, &al_f);
                    double ah = ah_f, al = al_f;
                    const double* bh = Bh + p * n;
                    const double* bl = Bl + p * n;
                    for (int64_t j = 0; j < n; ++j)
                        acc[j] += ah * bh[j] + ah * bl[j] + al * bh[j];
                }
            }
            double* crow = C_out + r * ldc_out;
            for (int64_t j = 0; j < n; ++j) {
                double ab = (alpha != 0.0) ? alpha * acc[j] : 0.0;
                double bc = (beta != 0.0) ? beta * C_in[i * ldc_in + j] : 0.0;
                crow[j] = bc + ab;
            }
        }
        free(acc);
    }
    free(Bh);
    free(Bl);
}

void oracle_split_tf32(float x, float* hi, float* lo) {
    float h = oracle_round_tf32(x);
    float d = x - h;   /* exact in binary32: h is x rounded to 11 significant bits */
    *hi = h;
    *lo = oracle_round_tf32(d);
}

/* The 3-product method on the TF32 split: 1) split both operands in two,
 * 2) form the three kept products per term, 3) sum over p in binary64.       */
void oracle_gemm_rows_3xtf32_f64(int64_t nrows, const int64_t* rows, int64_t n, int64_t k,
                                 double alpha, const float* A, int64_t lda,
                                 const float* B, int64_t ldb, double beta,
                                 const double* C_in, int64_t ldc_in,
                                 double* C_out, int64_t ldc_out, int nthreads) {
    if (nrows <= 0 || n <= 0) return;
    int nt = threads_for(nthreads);
    size_t kn = (size_t)(k > 0 ? k : 1) * (size_t)n;
    double* Bh = (double*)malloc(sizeof(double) * kn);
    double* Bl = (double*)malloc(sizeof(double) * kn);
    for (int64_t p = 0; p < k; ++p)
        for (int64_t j = 0; j < n; ++j) {
            float h, l;
            oracle_split_tf32(B[p * ldb + j], &h, &l);
            Bh[p * n + j] = h;
            Bl[p * n + j] = l;
        }
#pragma omp parallel num_threads(nt)
    {
        double* acc = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = row_index(rows, r);
            for (int64_t j = 0; j < n; ++j) acc[j] = 0.0;
            if (alpha != 0.0) {
                for (int64_t p = 0; p < k; ++p) {
                    float ah_f, al_f;
                    oracle_split_tf32(A[i * lda + p], &ah_f, &al_f);
                    double ah = ah_f, al = al_f;
                    const double* bh = Bh + p * n;
                    const double* bl = Bl + p * n;
                    for (int64_t j = 0; j < n; ++j)
                        acc[j] += ah * bh[j] + ah * bl[j] + al * bh[j];
                }
            }
            double* crow = C_out + r * ldc_out;
            for (int64_t j = 0; j < n; ++j) {
                double ab = (alpha != 0.0) ? alpha * acc[j] : 0.0;
                double bc = (beta != 0.0) ? beta * C_in[i * ldc_in + j] : 0.0;
                crow[j] = bc + ab;
            }
        }
        free(acc);
    }
    free(Bh);
    free(Bl);
}
