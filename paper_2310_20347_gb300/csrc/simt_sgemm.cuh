// simt_sgemm.cuh -- the "plain method": FP32 GEMM on the CUDA cores.
//
// This is the paper's baseline algorithm with the C-resident micro-kernel of
// Section 4.1 transplanted to a GPU thread block:
//   * a 128 x 128 block of C per CTA (the ic/jc loops become the CTA grid),
//   * k-blocks of 8 (loop pc) staged through double-buffered shared memory, A
//     stored k-major ("packed" so that one column of the A micro-panel is
//     contiguous, as Section 4.1 asks of Ac),
//   * every thread keeps an 8 x 8 micro-tile Cr in registers (mr = nr = 8) and,
//     per k (loop L6), performs one outer product of an 8-vector of A and an
//     8-vector of B: 64 FFMAs per 4 vector loads from shared memory.
// The 16 x 16 threads of a CTA take rows {4ty..4ty+3, 64+4ty..64+4ty+3} and the
// same split of columns, so a warp's 128-bit shared loads are conflict-free.
#pragma once
#include <cstdint>

namespace g3 {

struct SimtParams {
  int m, n, k;
  float alpha, beta;
  const float* A;
  long long lda;
  const float* B;
  long long ldb;
  float* C;
  long long ldc;
};

template <bool VEC>
__device__ __forceinline__ float4 load4_guarded(const float* base, long long row, int rows, int col, int cols,
                                                long long ld) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (row >= rows) return v;
  const float* p = base + row * ld + col;
  if (VEC && col + 3 < cols) {
    v = __ldg(reinterpret_cast<const float4*>(p));
  } else {
    if (col + 0 < cols) v.x = __ldg(p + 0);
    if (col + 1 < cols) v.y = __ldg(p + 1);
    if (col + 2 < cols) v.z = __ldg(p + 2);
    if (col + 3 < cols) v.w = __ldg(p + 3);
  }
  return v;
}

// VEC: A, B and C rows are 16-byte aligned (pointers and leading dimensions
// multiples of 4 floats), so full 4-wide groups move as float4.
template <bool VEC>
__global__ void __launch_bounds__(256, 2) simt_sgemm_kernel(const SimtParams p) {
  constexpr int BM = 128, BN = 128, BK = 8, PAD = 4;
  __shared__ __align__(16) float As[2][BK][BM + PAD];
  __shared__ __align__(16) float Bs[2][BK][BN];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  // global -> register mapping of one k-block
  const int a_row = tid >> 1, a_col = (tid & 1) * 4;    // A: 128 rows x 8 k
  const int b_row = tid >> 5, b_col = (tid & 31) * 4;   // B: 8 k x 128 cols

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float4 ra = load4_guarded<VEC>(p.A, m0 + a_row, p.m, a_col, p.k, p.lda);
  float4 rb = load4_guarded<VEC>(p.B, b_row, p.k, n0 + b_col, p.n, p.ldb);
  As[0][a_col + 0][a_row] = ra.x;
  As[0][a_col + 1][a_row] = ra.y;
  As[0][a_col + 2][a_row] = ra.z;
  As[0][a_col + 3][a_row] = ra.w;
  *reinterpret_cast<float4*>(&Bs[0][b_row][b_col]) = rb;
  __syncthreads();

  int buf = 0;
  for (int k0 = 0; k0 < p.k; k0 += BK) {
    const bool more = k0 + BK < p.k;
    if (more) {
      ra = load4_guarded<VEC>(p.A, m0 + a_row, p.m, k0 + BK + a_col, p.k, p.lda);
      rb = load4_guarded<VEC>(p.B, k0 + BK + b_row, p.k, n0 + b_col, p.n, p.ldb);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      const int nb = buf ^ 1;
      As[nb][a_col + 0][a_row] = ra.x;
      As[nb][a_col + 1][a_row] = ra.y;
      As[nb][a_col + 2][a_row] = ra.z;
      As[nb][a_col + 3][a_row] = ra.w;
      *reinterpret_cast<float4*>(&Bs[nb][b_row][b_col]) = rb;
    }
    __syncthreads();
    buf ^= 1;
  }

  // epilogue: C = alpha * acc + beta * C  (C not read when beta == 0)
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = m0 + ((i < 4) ? (ty * 4 + i) : (64 + ty * 4 + i - 4));
    if (row >= p.m) continue;
    float* crow = p.C + (long long)row * p.ldc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = n0 + h * 64 + tx * 4;
      float v[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) v[jj] = p.alpha * acc[i][h * 4 + jj];
      if (VEC && col + 3 < p.n) {
        float4* cp = reinterpret_cast<float4*>(crow + col);
        if (p.beta != 0.f) {
          const float4 o = *cp;
          v[0] = fmaf(p.beta, o.x, v[0]);
          v[1] = fmaf(p.beta, o.y, v[1]);
          v[2] = fmaf(p.beta, o.z, v[2]);
          v[3] = fmaf(p.beta, o.w, v[3]);
        }
        *cp = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          if (col + jj < p.n)
            crow[col + jj] = (p.beta != 0.f) ? fmaf(p.beta, crow[col + jj], v[jj]) : v[jj];
        }
      }
    }
  }
}

}  // namespace g3
