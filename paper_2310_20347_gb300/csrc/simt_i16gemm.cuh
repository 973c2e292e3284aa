// simt_i16gemm.cuh -- INT16 GEMM on the CUDA cores (the 16-bit integer entry of
// the paper's datatype study, Section 8.6): C := (beta ? C : 0) + A*B exactly,
// int16 A and B, int64 C.
//
// A product of two int16 values needs 31 bits, so two of them can already
// overflow int32: every product is widened and accumulated in int64 (a
// 32 x 32 -> 64-bit multiply-add per product), which keeps the result exact
// for any k this library accepts.  The blocking is the FP64 kernel's: a 64 x 64
// block of C per CTA, k-blocks of 16 double-buffered in shared memory (A stored
// k-major; the int16 values widened to int32 on the way in), and a 4 x 4
// micro-tile of int64 sums per thread.
#pragma once
#include <cstdint>

namespace g3 {

struct SimtParamsI16 {
  int m, n, k;
  int beta;   // 0 or 1
  const int16_t* A;
  long long lda;
  const int16_t* B;
  long long ldb;
  int64_t* C;
  long long ldc;
};

// Four consecutive int16 values of row `row` from column `col`, widened to
// int32, zero outside rows x cols.
__device__ __forceinline__ void load4s_guarded(const int16_t* base, long long row, int rows, int col, int cols,
                                               long long ld, int (&v)[4]) {
  v[0] = v[1] = v[2] = v[3] = 0;
  if (row >= rows) return;
  const int16_t* p = base + row * ld + col;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (col + i < cols) v[i] = __ldg(p + i);
}

// BK: k per shared-memory block (16).
template <int BK>
__global__ void __launch_bounds__(256, 2) simt_i16gemm_kernel(const SimtParamsI16 p) {
  static_assert(BK == 16, "the load mapping covers 16 k per block");
  constexpr int BM = 64, BN = 64, PAD = 4;
  __shared__ __align__(16) int As[2][BK][BM + PAD];
  __shared__ __align__(16) int Bs[2][BK][BN];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int a_row = tid >> 2, a_col = (tid & 3) * 4;   // A: 64 rows x 16 k
  const int b_row = tid >> 4, b_col = (tid & 15) * 4;  // B: 16 k x 64 cols

  long long acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;

  int ra[4], rb[4];
  load4s_guarded(p.A, m0 + a_row, p.m, a_col, p.k, p.lda, ra);
  load4s_guarded(p.B, b_row, p.k, n0 + b_col, p.n, p.ldb, rb);
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
      load4s_guarded(p.A, m0 + a_row, p.m, k0 + BK + a_col, p.k, p.lda, ra);
      load4s_guarded(p.B, k0 + BK + b_row, p.k, n0 + b_col, p.n, p.ldb, rb);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const int4 a = *reinterpret_cast<const int4*>(&As[buf][kk][ty * 4]);
      const int4 b = *reinterpret_cast<const int4*>(&Bs[buf][kk][tx * 4]);
      const int av[4] = {a.x, a.y, a.z, a.w};
      const int bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += (long long)av[i] * (long long)bv[j];
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

  // epilogue: C = A*B (+ C when beta == 1; C not read when beta == 0)
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = m0 + ty * 4 + i;
    if (row >= p.m) continue;
    int64_t* crow = p.C + (long long)row * p.ldc;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = n0 + tx * 4 + j;
      if (col < p.n) crow[col] = p.beta ? crow[col] + acc[i][j] : acc[i][j];
    }
  }
}

}  // namespace g3
