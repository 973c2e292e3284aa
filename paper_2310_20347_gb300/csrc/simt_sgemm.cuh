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

// Four floats at shared::cluster address `caddr` (16-byte aligned), which may
// lie in another CTA of the cluster.
__device__ __forceinline__ float4 ld_cluster_f4(uint32_t caddr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(caddr)
               : "memory");
  return v;
}

__device__ __forceinline__ void simt_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The same without the release fence: for a barrier that only has to keep
// this CTA's shared memory alive until the other CTAs have finished reading
// it (their loads have returned before they arrive).
__device__ __forceinline__ void simt_cluster_sync_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// Epilogue of one row of four: C = alpha * v + beta * C (C not read when
// beta == 0), float4 when the row is 16-byte aligned and whole.
template <bool VEC>
__device__ __forceinline__ void store4_epilogue(const SimtParams& p, int row, int col, const float (&acc)[4]) {
  if (row >= p.m) return;
  float* crow = p.C + (long long)row * p.ldc;
  float v[4];
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) v[jj] = p.alpha * acc[jj];
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
    for (int jj = 0; jj < 4; ++jj)
      if (col + jj < p.n) crow[col + jj] = (p.beta != 0.f) ? fmaf(p.beta, crow[col + jj], v[jj]) : v[jj];
  }
}

// The same method on 128 x 256 blocks of C for large problems: every thread
// keeps an 8 x 16 micro-tile (mr = 8, nr = 16: 128 FFMAs per six 128-bit
// shared loads, against 64 per four on 128 x 128 blocks) and the register
// fragments of the next k are loaded while the current k's outer product
// runs.  Thread (tx, ty) owns rows {4ty..4ty+3, 64+4ty..64+4ty+3} and columns
// {64q + 4tx .. 64q + 4tx + 3 : q = 0..3}.  k-blocks of BK (8 or 16) staged
// through double-buffered shared memory with A transposed k-major on the way
// in, one k-block of register prefetch; one CTA per SM (the micro-tile and
// fragments take ~210 registers).  Each element's products are still added in
// k order with one FMA each, so the result equals the other blockings' bit for
// bit.
template <bool VEC, int BK>
__global__ void __launch_bounds__(256, 1) simt_sgemm_wide_kernel(const SimtParams p) {
  constexpr int BM = 128, BN = 256, PAD = 4;
  constexpr int A_V4 = BK / 8;                 // float4s of A per thread per k-block
  constexpr int B_TPR = 256 / BK;              // threads per row of B's k-block
  constexpr int B_V4 = BK / 4;                 // float4s of B per thread per k-block
  extern __shared__ __align__(16) float wsmem[];
  float (*As)[BK][BM + PAD] = reinterpret_cast<float (*)[BK][BM + PAD]>(wsmem);                 // [2][BK][BM+PAD]
  float (*Bs)[BK][BN] = reinterpret_cast<float (*)[BK][BN]>(wsmem + 2 * BK * (BM + PAD));      // [2][BK][BN]

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int a_row = tid >> 1, a_k = (tid & 1) * (BK / 2);
  const int b_row = tid / B_TPR, b_col = (tid % B_TPR) * 4;

  float acc[8][16];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[i][j] = 0.f;

  float4 ra[A_V4], rb[B_V4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int v = 0; v < A_V4; ++v) ra[v] = load4_guarded<VEC>(p.A, m0 + a_row, p.m, k0 + a_k + 4 * v, p.k, p.lda);
#pragma unroll
    for (int v = 0; v < B_V4; ++v)
      rb[v] = load4_guarded<VEC>(p.B, k0 + b_row, p.k, n0 + b_col + v * (B_TPR * 4), p.n, p.ldb);
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int v = 0; v < A_V4; ++v) {
      As[buf][a_k + 4 * v + 0][a_row] = ra[v].x;
      As[buf][a_k + 4 * v + 1][a_row] = ra[v].y;
      As[buf][a_k + 4 * v + 2][a_row] = ra[v].z;
      As[buf][a_k + 4 * v + 3][a_row] = ra[v].w;
    }
#pragma unroll
    for (int v = 0; v < B_V4; ++v) *reinterpret_cast<float4*>(&Bs[buf][b_row][b_col + v * (B_TPR * 4)]) = rb[v];
  };

  fetch(0);
  stash(0);
  __syncthreads();

  int buf = 0;
  for (int k0 = 0; k0 < p.k; k0 += BK) {
    const bool more = k0 + BK < p.k;
    if (more) fetch(k0 + BK);
    float fa[2][8], fb[2][16];
    auto frag = [&](int kk, int f) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      fa[f][0] = a0.x; fa[f][1] = a0.y; fa[f][2] = a0.z; fa[f][3] = a0.w;
      fa[f][4] = a1.x; fa[f][5] = a1.y; fa[f][6] = a1.z; fa[f][7] = a1.w;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][kk][q * 64 + tx * 4]);
        fb[f][4 * q + 0] = b.x; fb[f][4 * q + 1] = b.y; fb[f][4 * q + 2] = b.z; fb[f][4 * q + 3] = b.w;
      }
    };
    frag(0, 0);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      if (kk + 1 < BK) frag(kk + 1, (kk + 1) & 1);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[i][j] = fmaf(fa[kk & 1][i], fb[kk & 1][j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = m0 + ((i < 4) ? (ty * 4 + i) : (64 + ty * 4 + i - 4));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float v[4] = {acc[i][4 * q], acc[i][4 * q + 1], acc[i][4 * q + 2], acc[i][4 * q + 3]};
      store4_epilogue<VEC>(p, row, n0 + q * 64 + tx * 4, v);
    }
  }
}

template <int BK>
constexpr int simt_wide_smem_bytes() {
  return (2 * BK * (128 + 4) + 2 * BK * 256) * 4;
}

// Asynchronous copies global -> shared (cp.async): `bytes` of 4 or 16, of
// which the first `src_bytes` are read and the rest zero-filled (src_bytes 0
// reads nothing).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The same method on 64 x 64 blocks of C with a 4 x 4 micro-tile per thread
// and k-blocks of 16, for problems whose 128 x 128 grid would leave SMs idle
// (four times the CTAs).  Thread (tx, ty) owns rows 4ty..4ty+3 and columns
// 4tx..4tx+3.
//
// Small problems run few k-blocks per CTA, so the copies run STAGES - 1
// k-blocks ahead of the arithmetic through a ring of shared-memory stages
// filled by cp.async in 16-byte pieces (zero-filled past the edges), which
// hides the DRAM latency that one block of register prefetch cannot.  A stays
// row-major in shared memory; per four k a thread reads four 4-vectors of A
// (its rows) and four of B, i.e. 64 FFMAs per 8 vector loads.
//
// SPLIT: the grid's z dimension is one thread-block cluster of S = gridDim.z
// CTAs per block of C, CTA z taking the k-range [z kc, (z+1) kc) with kc =
// ceil(k / S) rounded up to 16 (the loop pc of Section 4.1 shared out over
// the cluster).  Each CTA leaves its 64 x 64 partial block in shared memory;
// after a cluster barrier CTA z sums rows [64 z / S, 64 (z+1) / S) of the S
// partials through distributed shared memory, always in the order 0..S-1
// (deterministic), applies alpha and beta and stores them.  A second cluster
// barrier keeps every partial readable until all sums are taken.
template <bool VEC, bool SPLIT>
__global__ void __launch_bounds__(256, SPLIT ? 2 : 4) simt_sgemm64_kernel(const SimtParams p) {
  constexpr int BM = 64, BN = 64, BK = 16, APAD = 4, STAGES = 4;
  constexpr int LDA_S = BK + APAD;   // 20 floats: rows 4 apart fall 16 banks apart
  constexpr int A_STAGE = BM * LDA_S, B_STAGE = BK * BN;
  static_assert(BM * BN <= STAGES * (A_STAGE + B_STAGE), "the partial block reuses the stage ring");
  __shared__ __align__(16) float smem[STAGES * (A_STAGE + B_STAGE)];
  float* const As = smem;                     // [STAGES][BM][LDA_S], row-major
  float* const Bs = smem + STAGES * A_STAGE;  // [STAGES][BK][BN]

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int a_row = tid >> 2, a_col = (tid & 3) * 4;   // A: 64 rows x 16 k
  const int b_row = tid >> 4, b_col = (tid & 15) * 4;  // B: 16 k x 64 cols
  int kbeg = 0, kend = p.k;
  if (SPLIT) {
    const int kc = ((p.k + (int)gridDim.z - 1) / (int)gridDim.z + BK - 1) / BK * BK;
    kbeg = min(p.k, (int)blockIdx.z * kc);
    kend = min(p.k, kbeg + kc);
  }
  const int nkb = (kend - kbeg + BK - 1) / BK;

  // copies of k-block kb into stage st (zero outside m x [kbeg, kend) x n)
  const bool a_in = m0 + a_row < p.m;
  const float* const a_src = p.A + (a_in ? (long long)(m0 + a_row) * p.lda : 0);
  auto issue = [&](int kb, int st) {
    const int k0 = kbeg + kb * BK;
    float* as = As + st * A_STAGE + a_row * LDA_S + a_col;
    const int ka = k0 + a_col;
    const int a_left = a_in ? kend - ka : 0;   // valid elements from ka on
    const int kr = k0 + b_row, col = n0 + b_col;
    float* bs = Bs + st * B_STAGE + b_row * BN + b_col;
    const float* b_src = p.B + (long long)kr * p.ldb + col;
    const int b_left = kr < kend ? p.n - col : 0;
    if (VEC) {
      cp_async16(as, a_left > 0 ? a_src + ka : p.A, 4 * max(0, min(4, a_left)));
      cp_async16(bs, b_left > 0 ? b_src : p.B, 4 * max(0, min(4, b_left)));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        cp_async4(as + j, j < a_left ? a_src + ka + j : p.A, j < a_left ? 4 : 0);
        cp_async4(bs + j, j < b_left ? b_src + j : p.B, j < b_left ? 4 : 0);
      }
    }
  };

  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

#pragma unroll
  for (int st = 0; st < STAGES - 1; ++st) {
    if (st < nkb) issue(st, st);
    cp_async_commit();
  }
  for (int kb = 0; kb < nkb; ++kb) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();   // stage kb landed for every thread; stage kb - 1 is free
    if (kb + STAGES - 1 < nkb) issue(kb + STAGES - 1, (kb + STAGES - 1) % STAGES);
    cp_async_commit();
    const float* as = As + (kb % STAGES) * A_STAGE + ty * 4 * LDA_S;
    const float* bs = Bs + (kb % STAGES) * B_STAGE + tx * 4;
    if constexpr (SPLIT) {
      // At most two CTAs per SM leave few warps to hide shared-memory
      // latency: the fragments of step k4 + 4 are loaded while step k4's
      // outer products run (same products, same order per element).
      float a[2][4][4], b[2][4][4];   // a[.][i][u]: row 4ty + i, k = k4 + u; b[.][u][j]: k4 + u, column 4tx + j
      auto load = [&](int buf, int k4) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 v = *reinterpret_cast<const float4*>(as + i * LDA_S + k4);
          a[buf][i][0] = v.x;
          a[buf][i][1] = v.y;
          a[buf][i][2] = v.z;
          a[buf][i][3] = v.w;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 v = *reinterpret_cast<const float4*>(bs + (k4 + u) * BN);
          b[buf][u][0] = v.x;
          b[buf][u][1] = v.y;
          b[buf][u][2] = v.z;
          b[buf][u][3] = v.w;
        }
      };
      load(0, 0);
#pragma unroll
      for (int s4 = 0; s4 < BK / 4; ++s4) {
        const int cur = s4 & 1;
        if (s4 + 1 < BK / 4) load(cur ^ 1, (s4 + 1) * 4);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[cur][i][u], b[cur][u][j], acc[i][j]);
      }
      continue;
    }
#pragma unroll
    for (int k4 = 0; k4 < BK; k4 += 4) {
      float a[4][4];   // a[i][u]: row 4ty + i, k = k4 + u
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 v = *reinterpret_cast<const float4*>(as + i * LDA_S + k4);
        a[i][0] = v.x;
        a[i][1] = v.y;
        a[i][2] = v.z;
        a[i][3] = v.w;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 b4 = *reinterpret_cast<const float4*>(bs + (k4 + u) * BN);
        const float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i][u], b[j], acc[i][j]);
      }
    }
  }
  cp_async_wait<0>();

  if constexpr (!SPLIT) {
#pragma unroll
    for (int i = 0; i < 4; ++i) store4_epilogue<VEC>(p, m0 + ty * 4 + i, n0 + tx * 4, acc[i]);
  } else {
    __syncthreads();   // every thread is done with the stage ring
    float* const part = smem;   // [BM][BN]
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<float4*>(part + (ty * 4 + i) * BN + tx * 4) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    simt_cluster_sync();
    const int S = (int)gridDim.z, z = (int)blockIdx.z;
    const int r0 = z * BM / S, r1 = (z + 1) * BM / S;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(part);
    for (int idx = tid; idx < (r1 - r0) * (BN / 4); idx += 256) {
      const int r = r0 + idx / (BN / 4), c = (idx % (BN / 4)) * 4;
      const uint32_t off = base + (uint32_t)((r * BN + c) * 4);
      float sum[4] = {0.f, 0.f, 0.f, 0.f};
      for (int q = 0; q < S; ++q) {
        uint32_t caddr;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(caddr) : "r"(off), "r"(q));
        const float4 v = ld_cluster_f4(caddr);
        sum[0] += v.x;
        sum[1] += v.y;
        sum[2] += v.z;
        sum[3] += v.w;
      }
      store4_epilogue<VEC>(p, m0 + r, n0 + c, sum);
    }
    simt_cluster_sync_relaxed();
  }
}

}  // namespace g3
