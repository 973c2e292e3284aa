// kernels.cu -- launchers of the CUDA-core kernels: the FP32 SIMT GEMM and the
// memory-bound pre-/post-passes (see simt_sgemm.cuh and prepass.cuh).
#include <algorithm>
#include <atomic>

#include "internal.h"
#include "prepass.cuh"

namespace g3 {

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// Rows on grid.y (capped; kernels grid-stride), 4 columns per thread on grid.x.
static dim3 rows_grid(int rows, long long cols, int per_thread) {
  long long xblocks = (cols + 256LL * per_thread - 1) / (256LL * per_thread);
  xblocks = std::max(1LL, std::min(xblocks, 1024LL));
  int yblocks = std::max(1, std::min(rows, 32768));
  return dim3((unsigned)xblocks, (unsigned)yblocks, 1);
}

template <int BK>
static cudaError_t launch_simt_wide(const SimtParams& p, bool vec, cudaStream_t s) {
  constexpr int smem = simt_wide_smem_bytes<BK>();
  auto kern = vec ? simt_sgemm_wide_kernel<true, BK> : simt_sgemm_wide_kernel<false, BK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((p.n + 255) / 256, (p.m + 127) / 128, 1);
  kern<<<grid, 256, smem, s>>>(p);
  return cudaSuccess;
}

// kind 0: 128 x 128 blocks; kind 1: 64 x 64 blocks, cut along k over a
// cluster of `splits` CTAs when splits > 1 (1 <= splits <= 8); kind 2 / 3:
// 128 x 256 blocks with k-blocks of 8 / 16 through double-buffered shared
// memory.
cudaError_t launch_simt(const SimtParams& p, bool vec, int kind, int splits, cudaStream_t s) {
  if (kind == 2 || kind == 3) {
    const cudaError_t e = kind == 2 ? launch_simt_wide<8>(p, vec, s) : launch_simt_wide<16>(p, vec, s);
    if (e != cudaSuccess) return e;
  } else if (kind == 0) {
    dim3 grid((p.n + 127) / 128, (p.m + 127) / 128, 1);
    if (vec) simt_sgemm_kernel<true><<<grid, 256, 0, s>>>(p);
    else simt_sgemm_kernel<false><<<grid, 256, 0, s>>>(p);
  } else if (splits <= 1) {
    dim3 grid((p.n + 63) / 64, (p.m + 63) / 64, 1);
    if (vec) simt_sgemm64_kernel<true, false><<<grid, 256, 0, s>>>(p);
    else simt_sgemm64_kernel<false, false><<<grid, 256, 0, s>>>(p);
  } else {
    if (splits > 8) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.n + 63) / 64, (p.m + 63) / 64, splits);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = splits;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = vec ? cudaLaunchKernelEx(&cfg, simt_sgemm64_kernel<true, true>, p)
                              : cudaLaunchKernelEx(&cfg, simt_sgemm64_kernel<false, true>, p);
    if (e != cudaSuccess) return e;
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_split_bf16(const float* x, int rows, int cols, long long ldx, uint16_t* hi, uint16_t* lo,
                              long long ldy, cudaStream_t s) {
  const bool vec = reinterpret_cast<uintptr_t>(x) % 16 == 0 && ldx % 4 == 0 && reinterpret_cast<uintptr_t>(hi) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(lo) % 16 == 0 && ldy % 8 == 0;
  if (vec) {
    split_bf16_vec8_kernel<<<rows_grid(rows, cols, 8), 256, 0, s>>>(x, rows, cols, ldx, hi, lo, ldy);
    count_launch();
    return cudaGetLastError();
  }
  split_bf16_kernel<<<rows_grid(rows, cols, 4), 256, 0, s>>>(x, rows, cols, ldx, hi, lo, ldy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_split_bf16_pair(const float* xa, int rows_a, int cols_a, long long lda, uint16_t* ahi, uint16_t* alo,
                                   long long lda_p, const float* xb, int rows_b, int cols_b, long long ldb,
                                   uint16_t* bhi, uint16_t* blo, long long ldb_p, cudaStream_t s) {
  auto vec = [](const float* x, long long ldx, const uint16_t* hi, const uint16_t* lo, long long ldy) {
    return reinterpret_cast<uintptr_t>(x) % 16 == 0 && ldx % 4 == 0 && reinterpret_cast<uintptr_t>(hi) % 16 == 0 &&
           reinterpret_cast<uintptr_t>(lo) % 16 == 0 && ldy % 8 == 0;
  };
  if (!vec(xa, lda, ahi, alo, lda_p) || !vec(xb, ldb, bhi, blo, ldb_p)) {
    cudaError_t e = launch_split_bf16(xa, rows_a, cols_a, lda, ahi, alo, lda_p, s);
    return e != cudaSuccess ? e : launch_split_bf16(xb, rows_b, cols_b, ldb, bhi, blo, ldb_p, s);
  }
  const dim3 ga = rows_grid(rows_a, cols_a, 8), gb = rows_grid(rows_b, cols_b, 8);
  const dim3 grid(std::max(ga.x, gb.x), std::max(ga.y, gb.y), 2);
  split_bf16_vec8_pair_kernel<<<grid, 256, 0, s>>>(SplitJob{xa, rows_a, cols_a, lda, ahi, alo, lda_p},
                                                   SplitJob{xb, rows_b, cols_b, ldb, bhi, blo, ldb_p});
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_split3_bf16_pair(const float* xa, int rows_a, int cols_a, long long lda, uint16_t* ahi,
                                    uint16_t* amid, uint16_t* alo, long long lda_p, const float* xb, int rows_b,
                                    int cols_b, long long ldb, uint16_t* bhi, uint16_t* bmid, uint16_t* blo,
                                    long long ldb_p, cudaStream_t s) {
  const dim3 ga = rows_grid(rows_a, cols_a, 1), gb = rows_grid(rows_b, cols_b, 1);
  const dim3 grid(std::max(ga.x, gb.x), std::max(ga.y, gb.y), 2);
  split3_bf16_pair_kernel<<<grid, 256, 0, s>>>(Split3Job{xa, rows_a, cols_a, lda, ahi, amid, alo, lda_p},
                                               Split3Job{xb, rows_b, cols_b, ldb, bhi, bmid, blo, ldb_p});
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_int8_to_bf16_pair(const int8_t* xa, int rows_a, int cols_a, long long lda, uint16_t* ya,
                                     long long lda_p, const int8_t* xb, int rows_b, int cols_b, long long ldb,
                                     uint16_t* yb, long long ldb_p, cudaStream_t s) {
  auto vec = [](const int8_t* x, long long ldx, const uint16_t* y, long long ldy) {
    return reinterpret_cast<uintptr_t>(x) % 16 == 0 && ldx % 16 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0 &&
           ldy % 8 == 0;
  };
  if (!vec(xa, lda, ya, lda_p) || !vec(xb, ldb, yb, ldb_p)) {
    cudaError_t e = launch_int8_to_bf16(xa, rows_a, cols_a, lda, ya, lda_p, s);
    return e != cudaSuccess ? e : launch_int8_to_bf16(xb, rows_b, cols_b, ldb, yb, ldb_p, s);
  }
  const dim3 ga = rows_grid(rows_a, cols_a, 16), gb = rows_grid(rows_b, cols_b, 16);
  const dim3 grid(std::max(ga.x, gb.x), std::max(ga.y, gb.y), 2);
  int8_to_bf16_vec16_pair_kernel<<<grid, 256, 0, s>>>(I8Job{xa, rows_a, cols_a, lda, ya, lda_p},
                                                      I8Job{xb, rows_b, cols_b, ldb, yb, ldb_p});
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_split3_bf16(const float* x, int rows, int cols, long long ldx, uint16_t* hi, uint16_t* mid,
                               uint16_t* lo, long long ldy, cudaStream_t s) {
  split3_bf16_kernel<<<rows_grid(rows, cols, 1), 256, 0, s>>>(x, rows, cols, ldx, hi, mid, lo, ldy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_convert_tf32(const float* x, int rows, int cols, long long ldx, float* y, long long ldy,
                                cudaStream_t s) {
  const bool vec = reinterpret_cast<uintptr_t>(x) % 16 == 0 && ldx % 4 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0 &&
                   ldy % 4 == 0;
  if (vec) convert_tf32_kernel<true><<<rows_grid(rows, cols, 4), 256, 0, s>>>(x, rows, cols, ldx, y, ldy);
  else convert_tf32_kernel<false><<<rows_grid(rows, cols, 1), 256, 0, s>>>(x, rows, cols, ldx, y, ldy);
  count_launch();
  return cudaGetLastError();
}

// 64 x 64 tiles, up to eight resident blocks per SM
static int transpose64_grid(int rows, int cols) {
  const long long tiles = (long long)((rows + 63) / 64) * ((cols + 63) / 64);
  return (int)std::max<long long>(1, std::min<long long>(tiles, 152LL * 8));
}

cudaError_t launch_convert_tf32_t(const float* x, int rows, int cols, long long ldx, float* y, long long ldy,
                                  cudaStream_t s) {
  transpose64_kernel<kTransposeTf32><<<transpose64_grid(rows, cols), dim3(32, 8, 1), 0, s>>>(
      reinterpret_cast<const uint32_t*>(x), rows, cols, ldx, reinterpret_cast<uint32_t*>(y), nullptr, ldy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_simt64(const SimtParams64& p, bool vec, cudaStream_t s) {
  dim3 grid((p.n + 63) / 64, (p.m + 63) / 64, 1);
  if (vec) simt_dgemm_kernel<true><<<grid, 256, 0, s>>>(p);
  else simt_dgemm_kernel<false><<<grid, 256, 0, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_simt_i16(const SimtParamsI16& p, cudaStream_t s) {
  dim3 grid((p.n + 63) / 64, (p.m + 63) / 64, 1);
  simt_i16gemm_kernel<16><<<grid, 256, 0, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

__global__ void scale_c_f64_kernel(double* __restrict__ C, int rows, int cols, long long ldc, double beta) {
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    double* cr = C + r * ldc;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x)
      cr[c] = (beta == 0.0) ? 0.0 : beta * cr[c];
  }
}

cudaError_t launch_scale_c_f64(double* C, int rows, int cols, long long ldc, double beta, cudaStream_t s) {
  scale_c_f64_kernel<<<rows_grid(rows, cols, 1), 256, 0, s>>>(C, rows, cols, ldc, beta);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_split_tf32(const float* x, int rows, int cols, long long ldx, float* hi, float* lo,
                             long long ldy, cudaStream_t s) {
  const bool vec = reinterpret_cast<uintptr_t>(x) % 16 == 0 && ldx % 4 == 0 && reinterpret_cast<uintptr_t>(hi) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(lo) % 16 == 0 && ldy % 4 == 0;
  if (vec) split_tf32_kernel<true><<<rows_grid(rows, cols, 4), 256, 0, s>>>(x, rows, cols, ldx, hi, lo, ldy);
  else split_tf32_kernel<false><<<rows_grid(rows, cols, 1), 256, 0, s>>>(x, rows, cols, ldx, hi, lo, ldy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_split_tf32_t(const float* x, int rows, int cols, long long ldx, float* hi, float* lo,
                               long long ldy, cudaStream_t s) {
  transpose64_kernel<kTransposeSplitTf32><<<transpose64_grid(rows, cols), dim3(32, 8, 1), 0, s>>>(
      reinterpret_cast<const uint32_t*>(x), rows, cols, ldx, reinterpret_cast<uint32_t*>(hi),
      reinterpret_cast<uint32_t*>(lo), ldy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_convert_bf16(const float* x, int rows, int cols, long long ldx, uint16_t* y, long long ldy,
                                cudaStream_t s) {
  convert_bf16_kernel<<<rows_grid(rows, cols, 4), 256, 0, s>>>(x, rows, cols, ldx, y, ldy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_int8_to_bf16(const int8_t* x, int rows, int cols, long long ldx, uint16_t* y, long long ldy,
                                cudaStream_t s) {
  const bool vec = reinterpret_cast<uintptr_t>(x) % 16 == 0 && ldx % 16 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0 &&
                   ldy % 8 == 0;
  if (vec) {
    int8_to_bf16_vec16_kernel<<<rows_grid(rows, cols, 16), 256, 0, s>>>(x, rows, cols, ldx, y, ldy);
    count_launch();
    return cudaGetLastError();
  }
  int8_to_bf16_kernel<<<rows_grid(rows, cols, 4), 256, 0, s>>>(x, rows, cols, ldx, y, ldy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_transpose(const void* x, int rows, int cols, long long ldx, void* y, long long ldy, int esize,
                             cudaStream_t s) {
  const long long tiles = (long long)((rows + 31) / 32) * ((cols + 31) / 32);
  const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, 152LL * 16));
  const dim3 block(32, 8, 1);
  if (esize == 8)
    transpose_kernel<uint64_t><<<grid, block, 0, s>>>(static_cast<const uint64_t*>(x), rows, cols, ldx,
                                                       static_cast<uint64_t*>(y), ldy);
  else if (esize == 4)
    transpose64_kernel<kTransposeCopy><<<transpose64_grid(rows, cols), block, 0, s>>>(
        static_cast<const uint32_t*>(x), rows, cols, ldx, static_cast<uint32_t*>(y), nullptr, ldy);
  else if (esize == 2)
    transpose_kernel<uint16_t><<<grid, block, 0, s>>>(static_cast<const uint16_t*>(x), rows, cols, ldx,
                                                       static_cast<uint16_t*>(y), ldy);
  else
    transpose_kernel<uint8_t><<<grid, block, 0, s>>>(static_cast<const uint8_t*>(x), rows, cols, ldx,
                                                      static_cast<uint8_t*>(y), ldy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pack_rows(const void* x, int rows, long long row_bytes, long long ldx_bytes, void* y,
                             long long ldy_bytes, cudaStream_t s) {
  pack_rows_kernel<<<rows_grid(rows, row_bytes, 1), 256, 0, s>>>(static_cast<const uint8_t*>(x), rows, row_bytes,
                                                                 ldx_bytes, static_cast<uint8_t*>(y), ldy_bytes);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_quantize_e4m3(const float* x, int rows, int cols, long long ldx, unsigned int* amax_bits,
                                 uint8_t* q, long long ldq, float* scale, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(amax_bits, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  absmax_kernel<<<rows_grid(rows, cols, 1), 256, 0, s>>>(x, rows, cols, ldx, amax_bits);
  quantize_e4m3_kernel<<<rows_grid(rows, cols, 1), 256, 0, s>>>(x, rows, cols, ldx, amax_bits, q, ldq, scale);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_scale_c(void* C, bool is_int, int rows, int cols, long long ldc, float beta, cudaStream_t s) {
  if (is_int) scale_c_kernel<int><<<rows_grid(rows, cols, 1), 256, 0, s>>>(static_cast<int*>(C), rows, cols, ldc, beta);
  else scale_c_kernel<float><<<rows_grid(rows, cols, 1), 256, 0, s>>>(static_cast<float*>(C), rows, cols, ldc, beta);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_splitk_reduce(const float* P, int splits, int rows, int cols, long long ldp, float alpha,
                                 float beta, void* C, long long ldc, bool is_int, cudaStream_t s) {
  // 16-byte accesses of C when its rows allow (the partial planes always do)
  const bool vec = reinterpret_cast<uintptr_t>(C) % 16 == 0 && ldc % 4 == 0 && ldp % 4 == 0 &&
                   reinterpret_cast<uintptr_t>(P) % 16 == 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = rows_grid(rows, cols, 4);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // a dependent of the GEMM
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void (*kern)(const float*, int, int, int, long long, float, float, void*, long long) =
      is_int ? (vec ? splitk_reduce_kernel<true, true> : splitk_reduce_kernel<true, false>)
             : (vec ? splitk_reduce_kernel<false, true> : splitk_reduce_kernel<false, false>);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, P, splits, rows, cols, ldp, alpha, beta, C, ldc);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Stream-K fix-up (sched.cuh).  Block (t, y) covers a strip of 256 x 4
// consecutive elements of tail tile t: each thread adds the four columns it
// owns over the tile's partial results -- the slots of the streams whose
// pieces overlap the tile's k-blocks, in stream order (deterministic, as in
// the split-K reduce) -- and writes C.  One 16-byte vector per thread and slot
// keeps many independent loads in flight (partial tiles are bm x bn,
// row-major, bn a multiple of 4).
constexpr int kFixupMaxStreams = 1024;
constexpr int kFixupThreads = 256;

template <bool INT>
__global__ void __launch_bounds__(kFixupThreads) streamk_fixup_kernel(const SkFixup f) {
  __shared__ int slot_of[kFixupMaxStreams];   // per stream c0 + i: its slot, or -1 (no segment)
  __shared__ int nslot;
  const int t = blockIdx.x;
  const StreamK sk{(long long)f.tail * f.num_kb, f.streams, f.num_kb};
  const int c0 = sk.stream_of((long long)t * f.num_kb);
  const int c1 = sk.stream_of((long long)(t + 1) * f.num_kb - 1);
  if (threadIdx.x == 0) {   // the tile's slots, compacted, in stream order
    int ns = 0;
    for (int c = c0; c <= c1; ++c) {
      const int j = t - sk.first_tile(c);
      int tt, kb0, kb1;
      if (j >= 0 && sk.segment(c, j, tt, kb0, kb1)) slot_of[ns++] = c * f.segs + j;
    }
    nslot = ns;
  }
  int tm, tn;
  raster_tile(f.dp + t, f.tiles_m, f.tiles_n, f.raster, tm, tn);
  const int row0 = tm * f.bm, col0 = tn * f.bn;
  const int rows = min(f.bm, f.m - row0), cols = min(f.bn, f.n - col0);
  const int vec_per_row = f.bn / 4;
  const int v = blockIdx.y * kFixupThreads + threadIdx.x;   // this thread's vector of the tile
  const int r = v / vec_per_row;
  const int c4 = (v - r * vec_per_row) * 4;
  // launched as a programmatic dependent of the GEMM: wait for its grid (and
  // its memory) before reading any partial tile
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  if (r >= rows || c4 >= cols) return;
  const long long tile_elems = (long long)f.bm * f.bn;
  const long long off = (long long)r * f.bn + c4;
  const int ns = nslot;
  const int nq = min(4, cols - c4);
  if (INT) {
    int acc[4] = {0, 0, 0, 0};
    for (int i0 = 0; i0 < ns; i0 += 4) {
      int4 x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u < ns) x[u] = __ldcs(reinterpret_cast<const int4*>(f.partial + slot_of[i0 + u] * tile_elems + off));
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u < ns) {
          acc[0] += x[u].x;
          acc[1] += x[u].y;
          acc[2] += x[u].z;
          acc[3] += x[u].w;
        }
    }
    int* cp = static_cast<int*>(f.C) + (long long)(row0 + r) * f.ldc + col0 + c4;
    if (f.beta != 0.f) {
      int cv[4];
      for (int q = 0; q < nq; ++q) cv[q] = cp[q];
      for (int q = 0; q < nq; ++q) cp[q] = cv[q] + acc[q];
    } else {
      for (int q = 0; q < nq; ++q) cp[q] = acc[q];
    }
  } else {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i0 = 0; i0 < ns; i0 += 4) {
      float4 x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u < ns) x[u] = __ldcs(reinterpret_cast<const float4*>(f.partial + slot_of[i0 + u] * tile_elems + off));
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u < ns) {
          acc[0] += x[u].x;
          acc[1] += x[u].y;
          acc[2] += x[u].z;
          acc[3] += x[u].w;
        }
    }
    float scale = f.alpha;
    if (f.scale_a) scale *= *f.scale_a;
    if (f.scale_b) scale *= *f.scale_b;
    float* cp = static_cast<float*>(f.C) + (long long)(row0 + r) * f.ldc + col0 + c4;
    if (f.beta != 0.f) {
      float cv[4];
      for (int q = 0; q < nq; ++q) cv[q] = cp[q];
      for (int q = 0; q < nq; ++q) cp[q] = fmaf(scale, acc[q], f.beta * cv[q]);
    } else {
      for (int q = 0; q < nq; ++q) cp[q] = scale * acc[q];
    }
  }
}

// Memory-traffic yardstick: reads nin and writes nout 16-byte units.  The
// traffic is cut into chunks of 2048 units (32 KB); chunk c of the C = cin +
// cout chunks is a read chunk when floor((c + 1) cin / C) steps past
// floor(c cin / C), else a write chunk, so every block's grid-stride walk (and
// the memory system at any moment) sees reads and writes in their overall
// proportion.  A thread moves 8 units of a chunk (8 independent 16-byte
// accesses in flight) with streaming cache hints; writes carry filler
// (chunk + 1, thread + 1, 0, 0) and wait for no load; the loads are folded
// into a value that reaches memory only in the (never expected) case that it
// equals a fixed constant, so that none of them can be dropped.  Measured on
// GB300: 6.3 TB/s for a 1:1 mix (a device-to-device copy: 6.8), 6.0-6.4 for
// 1:2 and 1:8, 7.0 for reads or writes alone.
constexpr int kStreamUnits = 8;
constexpr int kStreamChunk = 256 * kStreamUnits;
__device__ unsigned int g_stream_sink;

__global__ void __launch_bounds__(256) stream_traffic_kernel(const uint4* __restrict__ in, long long nin,
                                                             uint4* __restrict__ out, long long nout) {
  const long long cin = (nin + kStreamChunk - 1) / kStreamChunk, cout = (nout + kStreamChunk - 1) / kStreamChunk;
  const long long C = cin + cout;
  unsigned int acc = 0;
  for (long long c = blockIdx.x; c < C; c += gridDim.x) {
    const long long r0 = c * cin / C, r1 = (c + 1) * cin / C;
    if (r1 > r0) {
      uint4 v[kStreamUnits];
#pragma unroll
      for (int u = 0; u < kStreamUnits; ++u) {
        const long long i = r0 * kStreamChunk + u * 256 + threadIdx.x;
        v[u] = i < nin ? __ldcs(in + i) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < kStreamUnits; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    } else {
      const long long w = c - r0;   // write chunks before this one
      const uint4 f = make_uint4((unsigned)c + 1u, threadIdx.x + 1u, 0u, 0u);   // never all zero
#pragma unroll
      for (int u = 0; u < kStreamUnits; ++u) {
        const long long i = w * kStreamChunk + u * 256 + threadIdx.x;
        if (i < nout) __stcs(out + i, f);
      }
    }
  }
  if (acc == 0x9E3779B9u) g_stream_sink = acc;
}

cudaError_t launch_stream_traffic(const void* in, long long in_units, void* out, long long out_units, int sms,
                                  cudaStream_t s) {
  const long long chunks = (in_units + kStreamChunk - 1) / kStreamChunk + (out_units + kStreamChunk - 1) / kStreamChunk;
  if (chunks == 0) return cudaSuccess;
  const long long blocks = std::min<long long>(chunks, (long long)sms * 16);
  stream_traffic_kernel<<<(unsigned)blocks, 256, 0, s>>>(static_cast<const uint4*>(in), in_units,
                                                          static_cast<uint4*>(out), out_units);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_streamk_fixup(const SkFixup& f, cudaStream_t s) {
  if (f.tail <= 0) return cudaSuccess;
  if (f.streams > kFixupMaxStreams || f.bn % 4 != 0) return cudaErrorInvalidValue;
  // programmatic stream serialisation: the fix-up's launch overlaps the tail
  // of the GEMM kernel, which signals its dependents early
  const int vecs = f.bm * (f.bn / 4);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)f.tail, (unsigned)((vecs + kFixupThreads - 1) / kFixupThreads), 1);
  cfg.blockDim = dim3(kFixupThreads, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = f.is_int ? cudaLaunchKernelEx(&cfg, streamk_fixup_kernel<true>, f)
                                 : cudaLaunchKernelEx(&cfg, streamk_fixup_kernel<false>, f);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace g3
