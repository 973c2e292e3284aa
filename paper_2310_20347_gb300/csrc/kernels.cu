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

cudaError_t launch_simt(const SimtParams& p, bool vec, cudaStream_t s) {
  dim3 grid((p.n + 127) / 128, (p.m + 127) / 128, 1);
  if (vec) simt_sgemm_kernel<true><<<grid, 256, 0, s>>>(p);
  else simt_sgemm_kernel<false><<<grid, 256, 0, s>>>(p);
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

cudaError_t launch_convert_tf32_t(const float* x, int rows, int cols, long long ldx, float* y, long long ldy,
                                  cudaStream_t s) {
  const long long tiles = (long long)((rows + 31) / 32) * ((cols + 31) / 32);
  const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, 152LL * 16));
  transpose_kernel<uint32_t, true><<<grid, dim3(32, 8, 1), 0, s>>>(reinterpret_cast<const uint32_t*>(x), rows, cols,
                                                                    ldx, reinterpret_cast<uint32_t*>(y), ldy);
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
  if (esize == 4)
    transpose_kernel<uint32_t><<<grid, block, 0, s>>>(static_cast<const uint32_t*>(x), rows, cols, ldx,
                                                       static_cast<uint32_t*>(y), ldy);
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

cudaError_t launch_splitk_reduce(const float* P, int splits, int rows, int cols, float alpha, float beta, void* C,
                                 long long ldc, bool is_int, cudaStream_t s) {
  if (is_int)
    splitk_reduce_kernel<true><<<rows_grid(rows, cols, 1), 256, 0, s>>>(P, splits, rows, cols, alpha, beta, C, ldc);
  else
    splitk_reduce_kernel<false><<<rows_grid(rows, cols, 1), 256, 0, s>>>(P, splits, rows, cols, alpha, beta, C, ldc);
  count_launch();
  return cudaGetLastError();
}

}  // namespace g3
