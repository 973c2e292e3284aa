// simt_dgemm.cuh -- FP64 GEMM on the CUDA cores (the binary64 entry of the
// paper's datatype study, Section 8.6).
//
// The same blocked structure as the FP32 "plain method" (simt_sgemm.cuh),
// sized for doubles: a 64 x 64 block of C per CTA, k-blocks of 16 staged
// through double-buffered shared memory (A stored k-major, the packed Ac of
// Section 4.1), and a 4 x 4 micro-tile Cr of doubles per thread updated by one
// outer product per k (16 DFMAs per 8 shared loads).  Thread (tx, ty) of the
// 16 x 16 block owns rows 4ty..4ty+3 and columns 4tx..4tx+3.  FP64 arithmetic
// throughout, one FMA per product, so the result differs from an exact
// binary64 sum only by rounding order.
#pragma once
#include <cstdint>

namespace g3 {

struct SimtParams64 {
  int m, n, k;
  double alpha, beta;
  const double* A;
  long long lda;
  const double* B;
  long long ldb;
  double* C;
  long long ldc;
};

// Four consecutive doubles of row `row` starting at column `col`, zero outside
// rows x cols; 16-byte loads when VEC (rows 16-byte aligned).
template <bool VEC>
__device__ __forceinline__ void load4d_guarded(const double* base, long long row, int rows, int col, int cols,
                                               long long ld, double (&v)[4]) {
  v[0] = v[1] = v[2] = v[3] = 0.0;
  if (row >= rows) return;
  const double* p = base + row * ld + col;
  if (VEC && col + 3 < cols) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (col + i < cols) v[i] = __ldg(p + i);
  }
}

template <bool VEC>
__global__ void __launch_bounds__(256, 2) simt_dgemm_kernel(const SimtParams64 p) {
  constexpr int BM = 64, BN = 64, BK = 16, PAD = 2;
  __shared__ __align__(16) double As[2][BK][BM + PAD];
  __shared__ __align__(16) double Bs[2][BK][BN];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int a_row = tid >> 2, a_col = (tid & 3) * 4;   // A: 64 rows x 16 k
  const int b_row = tid >> 4, b_col = (tid & 15) * 4;  // B: 16 k x 64 cols

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  double ra[4], rb[4];
  load4d_guarded<VEC>(p.A, m0 + a_row, p.m, a_col, p.k, p.lda, ra);
  load4d_guarded<VEC>(p.B, b_row, p.k, n0 + b_col, p.n, p.ldb, rb);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    As[0][a_col + i][a_row] = ra[i];
    Bs[0][b_row][b_col + i] = rb[i];
  }
  __syncthreads();

  int buf = 0;
  for (int k0 = 0; k0 < p.k; k0 += BK) {
    const bool more = k0 + BK < p.k;
    if (more) {
      load4d_guarded<VEC>(p.A, m0 + a_row, p.m, k0 + BK + a_col, p.k, p.lda, ra);
      load4d_guarded<VEC>(p.B, k0 + BK + b_row, p.k, n0 + b_col, p.n, p.ldb, rb);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const double2 a0 = *reinterpret_cast<const double2*>(&As[buf][kk][ty * 4]);
      const double2 a1 = *reinterpret_cast<const double2*>(&As[buf][kk][ty * 4 + 2]);
      const double2 b0 = *reinterpret_cast<const double2*>(&Bs[buf][kk][tx * 4]);
      const double2 b1 = *reinterpret_cast<const double2*>(&Bs[buf][kk][tx * 4 + 2]);
      const double a[4] = {a0.x, a0.y, a1.x, a1.y};
      const double b[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) {
      const int nb = buf ^ 1;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        As[nb][a_col + i][a_row] = ra[i];
        Bs[nb][b_row][b_col + i] = rb[i];
      }
    }
    __syncthreads();
    buf ^= 1;
  }

  // epilogue: C = alpha * acc + beta * C (C not read when beta == 0)
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = m0 + ty * 4 + i;
    if (row >= p.m) continue;
    double* crow = p.C + (long long)row * p.ldc;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = n0 + tx * 4 + j;
      if (col < p.n) crow[col] = (p.beta != 0.0) ? fma(p.beta, crow[col], p.alpha * acc[i][j]) : p.alpha * acc[i][j];
    }
  }
}

}  // namespace g3
