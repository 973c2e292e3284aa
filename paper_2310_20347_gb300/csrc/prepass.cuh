// prepass.cuh -- memory-bound operand preparation and epilogue-only kernels.
//
// These are the GPU form of the paper's packing step (Section 5.3): copies that
// put an operand in the layout and number format the blocked kernel consumes,
// paid once per operand so that the O(mnk) work reads a friendly layout.
//   split_bf16      FP32 -> (hi, lo) bfloat16 planes for the FP32-accurate mode
//   convert_bf16    FP32 -> bfloat16 (round to nearest even)
//   int8_to_bf16    int8 -> bfloat16 (exact)
//   pack_rows       byte copy of a strided matrix into a 16-byte-aligned one
//   absmax / quantize_e4m3   per-tensor FP8 scaling
//   scale_c         C := beta*C (the k == 0 / alpha == 0 cases)
//   splitk_reduce   C := alpha * sum_s P[s] + beta*C in a fixed split order
// Rows go to blockIdx.y (grid-stride) and columns to threads, 4 per thread, so
// that every warp reads and writes contiguous runs of a row.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cstdint>

#include "bf16.cuh"

namespace g3 {

// hi = bf16(x), lo = bf16(x - hi); x - hi is exact in FP32.
__global__ void split_bf16_kernel(const float* __restrict__ x, int rows, int cols, long long ldx,
                                  uint16_t* __restrict__ hi, uint16_t* __restrict__ lo, long long ldy) {
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const float* xr = x + r * ldx;
    uint16_t* hr = hi + r * ldy;
    uint16_t* lr = lo + r * ldy;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) * 4; c < cols; c += gridDim.x * blockDim.x * 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (c + u < cols) {
          const float v = xr[c + u];
          const uint16_t h = bf16_bits(v);
          hr[c + u] = h;
          lr[c + u] = bf16_bits(v - bf16_value(h));
        }
      }
    }
  }
}

__device__ __forceinline__ uint32_t pack_bf16x2(uint16_t lo_elem, uint16_t hi_elem) {
  return static_cast<uint32_t>(lo_elem) | (static_cast<uint32_t>(hi_elem) << 16);
}

// The same split, 8 elements per thread step: two 16-byte loads of x, one
// 16-byte store per plane.  Requires 16-byte-aligned rows of x (ldx % 4 == 0)
// and of the planes (ldy % 8 == 0); the last cols % 8 elements of a row are
// done one by one.
__device__ __forceinline__ void split_bf16_vec8_rows(const float* __restrict__ x, int rows, int cols, long long ldx,
                                                    uint16_t* __restrict__ hi, uint16_t* __restrict__ lo,
                                                    long long ldy) {
  const int cols8 = cols >> 3;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const float* xr = x + r * ldx;
    uint16_t* hr = hi + r * ldy;
    uint16_t* lr = lo + r * ldy;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols8; c += gridDim.x * blockDim.x) {
      const float4 a = __ldcs(reinterpret_cast<const float4*>(xr) + 2 * c);
      const float4 b = __ldcs(reinterpret_cast<const float4*>(xr) + 2 * c + 1);
      const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      uint16_t h[8], l[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        h[u] = bf16_bits(v[u]);
        l[u] = bf16_bits(v[u] - bf16_value(h[u]));
      }
      reinterpret_cast<uint4*>(hr)[c] =
          make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]), pack_bf16x2(h[4], h[5]), pack_bf16x2(h[6], h[7]));
      reinterpret_cast<uint4*>(lr)[c] =
          make_uint4(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]), pack_bf16x2(l[4], l[5]), pack_bf16x2(l[6], l[7]));
    }
    if (blockIdx.x == 0) {
      for (int c = (cols8 << 3) + threadIdx.x; c < cols; c += blockDim.x) {
        const float v = xr[c];
        const uint16_t h = bf16_bits(v);
        hr[c] = h;
        lr[c] = bf16_bits(v - bf16_value(h));
      }
    }
  }
}

__global__ void split_bf16_vec8_kernel(const float* __restrict__ x, int rows, int cols, long long ldx,
                                       uint16_t* __restrict__ hi, uint16_t* __restrict__ lo, long long ldy) {
  split_bf16_vec8_rows(x, rows, cols, ldx, hi, lo, ldy);
}

// Both operands of one call in a single launch: blockIdx.z selects the job
// (0: A, 1: B), which saves a launch and its gap on small problems.
struct SplitJob {
  const float* x;
  int rows, cols;
  long long ldx;
  uint16_t* hi;
  uint16_t* lo;
  long long ldy;
};

__global__ void split_bf16_vec8_pair_kernel(const SplitJob j0, const SplitJob j1) {
  const SplitJob& J = blockIdx.z == 0 ? j0 : j1;
  split_bf16_vec8_rows(J.x, J.rows, J.cols, J.ldx, J.hi, J.lo, J.ldy);
}

// Three-part split for the small-k FP32-accurate mode: hi = bf16(x),
// mid = bf16(x - hi), lo = bf16((x - hi) - mid); both differences are exact.
__device__ __forceinline__ void split3(float v, uint16_t& h, uint16_t& m, uint16_t& l) {
  h = bf16_bits(v);
  const float d = v - bf16_value(h);
  m = bf16_bits(d);
  l = bf16_bits(d - bf16_value(m));
}

__device__ __forceinline__ void split3_bf16_rows(const float* __restrict__ x, int rows, int cols, long long ldx,
                                                 uint16_t* __restrict__ hi, uint16_t* __restrict__ mid,
                                                 uint16_t* __restrict__ lo, long long ldy) {
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const float* xr = x + r * ldx;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
      uint16_t h, m, l;
      split3(xr[c], h, m, l);
      hi[r * ldy + c] = h;
      mid[r * ldy + c] = m;
      lo[r * ldy + c] = l;
    }
  }
}

__global__ void split3_bf16_kernel(const float* __restrict__ x, int rows, int cols, long long ldx,
                                   uint16_t* __restrict__ hi, uint16_t* __restrict__ mid, uint16_t* __restrict__ lo,
                                   long long ldy) {
  split3_bf16_rows(x, rows, cols, ldx, hi, mid, lo, ldy);
}

// Both operands of one call in a single launch (blockIdx.z: 0 = A, 1 = B).
struct Split3Job {
  const float* x;
  int rows, cols;
  long long ldx;
  uint16_t *hi, *mid, *lo;
  long long ldy;
};

__global__ void split3_bf16_pair_kernel(const Split3Job j0, const Split3Job j1) {
  const Split3Job& J = blockIdx.z == 0 ? j0 : j1;
  split3_bf16_rows(J.x, J.rows, J.cols, J.ldx, J.hi, J.mid, J.lo, J.ldy);
}

// TF32 round to nearest even on the encoding: add half an ulp of the 10-bit
// fraction (plus one when the kept last bit is odd) and clear the 13 dropped
// bits; a carry into the exponent rounds up to the next binade or to infinity.
__device__ __forceinline__ float tf32_rne(float v) {
  uint32_t u = __float_as_uint(v);
  if ((u & 0x7F800000u) == 0x7F800000u) return __uint_as_float((u & 0x007FFFFFu) ? 0x7FC00000u : u);
  u += 0x0FFFu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xFFFFE000u);
}

// y = tf32(x); 4 elements per thread step with 16-byte accesses when both
// matrices' rows are 16-byte aligned (vec), else one by one.
template <bool VEC>
__global__ void convert_tf32_kernel(const float* __restrict__ x, int rows, int cols, long long ldx,
                                    float* __restrict__ y, long long ldy) {
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const float* xr = x + r * ldx;
    float* yr = y + r * ldy;
    if (VEC) {
      const int cols4 = cols >> 2;
      for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols4; c += gridDim.x * blockDim.x) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(xr) + c);
        reinterpret_cast<float4*>(yr)[c] = make_float4(tf32_rne(a.x), tf32_rne(a.y), tf32_rne(a.z), tf32_rne(a.w));
      }
      if (blockIdx.x == 0)
        for (int c = (cols4 << 2) + threadIdx.x; c < cols; c += blockDim.x) yr[c] = tf32_rne(xr[c]);
    } else {
      for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) yr[c] = tf32_rne(xr[c]);
    }
  }
}

// The two-part TF32 split: hi = tf32(x), lo = tf32(x - hi) (the difference is
// exact in binary32); 4 elements per thread step with 16-byte accesses when
// all rows are 16-byte aligned (vec), else one by one.
__device__ __forceinline__ void split_tf32(float v, float& h, float& l) {
  h = tf32_rne(v);
  l = tf32_rne(__fsub_rn(v, h));
}

template <bool VEC>
__global__ void split_tf32_kernel(const float* __restrict__ x, int rows, int cols, long long ldx,
                                  float* __restrict__ hi, float* __restrict__ lo, long long ldy) {
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const float* xr = x + r * ldx;
    float* hr = hi + r * ldy;
    float* lr = lo + r * ldy;
    if (VEC) {
      const int cols4 = cols >> 2;
      for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols4; c += gridDim.x * blockDim.x) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(xr) + c);
        float4 h, l;
        split_tf32(a.x, h.x, l.x);
        split_tf32(a.y, h.y, l.y);
        split_tf32(a.z, h.z, l.z);
        split_tf32(a.w, h.w, l.w);
        reinterpret_cast<float4*>(hr)[c] = h;
        reinterpret_cast<float4*>(lr)[c] = l;
      }
      if (blockIdx.x == 0)
        for (int c = (cols4 << 2) + threadIdx.x; c < cols; c += blockDim.x) split_tf32(xr[c], hr[c], lr[c]);
    } else {
      for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x)
        split_tf32(xr[c], hr[c], lr[c]);
    }
  }
}

__global__ void convert_bf16_kernel(const float* __restrict__ x, int rows, int cols, long long ldx,
                                    uint16_t* __restrict__ y, long long ldy) {
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const float* xr = x + r * ldx;
    uint16_t* yr = y + r * ldy;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) * 4; c < cols; c += gridDim.x * blockDim.x * 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c + u < cols) yr[c + u] = bf16_bits(xr[c + u]);
    }
  }
}

__global__ void int8_to_bf16_kernel(const int8_t* __restrict__ x, int rows, int cols, long long ldx,
                                    uint16_t* __restrict__ y, long long ldy) {
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const int8_t* xr = x + r * ldx;
    uint16_t* yr = y + r * ldy;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) * 4; c < cols; c += gridDim.x * blockDim.x * 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c + u < cols) yr[c + u] = bf16_bits(static_cast<float>(xr[c + u]));
    }
  }
}

// The same, 16 elements per thread step: one 16-byte load of x, two 16-byte
// stores of y.  Requires 16-byte-aligned rows of x (ldx % 16 == 0) and of y
// (ldy % 8 == 0); the last cols % 16 elements of a row are done one by one.
__device__ __forceinline__ void int8_to_bf16_vec16_rows(const int8_t* __restrict__ x, int rows, int cols,
                                                        long long ldx, uint16_t* __restrict__ y, long long ldy) {
  const int cols16 = cols >> 4;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const int8_t* xr = x + r * ldx;
    uint16_t* yr = y + r * ldy;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols16; c += gridDim.x * blockDim.x) {
      const uint4 q = __ldcs(reinterpret_cast<const uint4*>(xr) + c);
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
      uint32_t o[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int8_t b0 = static_cast<int8_t>(w[i] & 0xFF), b1 = static_cast<int8_t>((w[i] >> 8) & 0xFF);
        const int8_t b2 = static_cast<int8_t>((w[i] >> 16) & 0xFF), b3 = static_cast<int8_t>(w[i] >> 24);
        o[2 * i] = pack_bf16x2(bf16_bits(static_cast<float>(b0)), bf16_bits(static_cast<float>(b1)));
        o[2 * i + 1] = pack_bf16x2(bf16_bits(static_cast<float>(b2)), bf16_bits(static_cast<float>(b3)));
      }
      reinterpret_cast<uint4*>(yr)[2 * c] = make_uint4(o[0], o[1], o[2], o[3]);
      reinterpret_cast<uint4*>(yr)[2 * c + 1] = make_uint4(o[4], o[5], o[6], o[7]);
    }
    if (blockIdx.x == 0)
      for (int c = (cols16 << 4) + threadIdx.x; c < cols; c += blockDim.x) yr[c] = bf16_bits(static_cast<float>(xr[c]));
  }
}

__global__ void int8_to_bf16_vec16_kernel(const int8_t* __restrict__ x, int rows, int cols, long long ldx,
                                          uint16_t* __restrict__ y, long long ldy) {
  int8_to_bf16_vec16_rows(x, rows, cols, ldx, y, ldy);
}

// Both int8 operands of one call in a single launch (blockIdx.z: 0 = A, 1 = B).
struct I8Job {
  const int8_t* x;
  int rows, cols;
  long long ldx;
  uint16_t* y;
  long long ldy;
};

__global__ void int8_to_bf16_vec16_pair_kernel(const I8Job j0, const I8Job j1) {
  const I8Job& J = blockIdx.z == 0 ? j0 : j1;
  int8_to_bf16_vec16_rows(J.x, J.rows, J.cols, J.ldx, J.y, J.ldy);
}

// Copy `cols` elements of `esize` bytes per row from a strided source into a
// destination whose rows start on 16-byte boundaries.
__global__ void pack_rows_kernel(const uint8_t* __restrict__ x, int rows, long long row_bytes, long long ldx_bytes,
                                 uint8_t* __restrict__ y, long long ldy_bytes) {
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const uint8_t* xr = x + r * ldx_bytes;
    uint8_t* yr = y + r * ldy_bytes;
    for (long long c = blockIdx.x * blockDim.x + threadIdx.x; c < row_bytes; c += (long long)gridDim.x * blockDim.x)
      yr[c] = xr[c];
  }
}

// y (cols x rows, leading dimension ldy) := transpose of x (rows x cols,
// leading dimension ldx), elements of type T, through a 32 x 33 shared tile so
// that both the reads and the writes are coalesced.  Block (32, 8).
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ x, int rows, int cols, long long ldx, T* __restrict__ y,
                                 long long ldy) {
  __shared__ T tile[32][33];
  const int tr = (rows + 31) / 32, tc = (cols + 31) / 32;
  for (long long t = blockIdx.x; t < (long long)tr * tc; t += gridDim.x) {
    const int r0 = (int)(t / tc) * 32, c0 = (int)(t % tc) * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
      const int r = r0 + i, c = c0 + threadIdx.x;
      if (r < rows && c < cols) tile[i][threadIdx.x] = x[(long long)r * ldx + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
      const int c = c0 + i, r = r0 + threadIdx.x;   // output row c, column r
      if (c < cols && r < rows) y[(long long)c * ldy + r] = tile[threadIdx.x][i];
    }
    __syncthreads();
  }
}

// Transpose of 4-byte elements through 64 x 64 tiles (block (32, 8), 16
// elements per thread each way): every warp access covers 256 consecutive
// bytes of a row, twice the 32 x 32 tile's segments, which keeps DRAM pages
// open longer on both the read and the write side.  OP maps one input value
// to the output value(s): kTransposeCopy, kTransposeTf32 (round), or
// kTransposeSplitTf32 (hi -> y, lo -> y2).
enum TransposeOp : int { kTransposeCopy = 0, kTransposeTf32 = 1, kTransposeSplitTf32 = 2 };

template <int OP>
__global__ void __launch_bounds__(256) transpose64_kernel(const uint32_t* __restrict__ x, int rows, int cols,
                                                          long long ldx, uint32_t* __restrict__ y,
                                                          uint32_t* __restrict__ y2, long long ldy) {
  __shared__ uint32_t tile[64][65];
  const int tr = (rows + 63) / 64, tc = (cols + 63) / 64;
  for (long long t = blockIdx.x; t < (long long)tr * tc; t += gridDim.x) {
    const int r0 = (int)(t / tc) * 64, c0 = (int)(t % tc) * 64;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = r0 + threadIdx.y + 8 * i;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = c0 + h * 32 + threadIdx.x;
        if (r < rows && c < cols) tile[threadIdx.y + 8 * i][h * 32 + threadIdx.x] = __ldcs(x + (long long)r * ldx + c);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = c0 + threadIdx.y + 8 * i;   // output row
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = r0 + h * 32 + threadIdx.x;   // output column
        if (c < cols && r < rows) {
          const uint32_t v = tile[h * 32 + threadIdx.x][threadIdx.y + 8 * i];
          if constexpr (OP == kTransposeCopy) {
            y[(long long)c * ldy + r] = v;
          } else if constexpr (OP == kTransposeTf32) {
            y[(long long)c * ldy + r] = __float_as_uint(tf32_rne(__uint_as_float(v)));
          } else {
            const float f = __uint_as_float(v);
            const float hi = tf32_rne(f);
            y[(long long)c * ldy + r] = __float_as_uint(hi);
            y2[(long long)c * ldy + r] = __float_as_uint(tf32_rne(__fsub_rn(f, hi)));
          }
        }
      }
    }
    __syncthreads();
  }
}

// amax of |x| as the bit pattern of a non-negative float (monotone as unsigned).
__global__ void absmax_kernel(const float* __restrict__ x, int rows, int cols, long long ldx,
                              unsigned int* __restrict__ amax_bits) {
  float m = 0.f;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const float* xr = x + r * ldx;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
      const float a = fabsf(xr[c]);
      m = (a > m) ? a : m;   // NaN never wins the comparison
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  __shared__ float wmax[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) wmax[w] = m;
  __syncthreads();
  if (w == 0) {
    m = (l < (int)(blockDim.x >> 5)) ? wmax[l] : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (l == 0) atomicMax(amax_bits, __float_as_uint(m));
  }
}

// scale = amax / 448 (1 when amax == 0); code = e4m3_satfinite(x / scale).
__global__ void quantize_e4m3_kernel(const float* __restrict__ x, int rows, int cols, long long ldx,
                                     const unsigned int* __restrict__ amax_bits, uint8_t* __restrict__ q,
                                     long long ldq, float* __restrict__ scale_out) {
  const float amax = __uint_as_float(*amax_bits);
  const float scale = (amax > 0.f) ? __fdiv_rn(amax, 448.0f) : 1.0f;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && scale_out) *scale_out = scale;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const float* xr = x + r * ldx;
    uint8_t* qr = q + r * ldq;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x)
      qr[c] = static_cast<uint8_t>(__nv_cvt_float_to_fp8(__fdiv_rn(xr[c], scale), __NV_SATFINITE, __NV_E4M3));
  }
}

template <typename TC>
__global__ void scale_c_kernel(TC* __restrict__ C, int rows, int cols, long long ldc, float beta) {
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    TC* cr = C + r * ldc;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
      if (beta == 0.f) cr[c] = TC(0);
      else cr[c] = static_cast<TC>(beta * static_cast<float>(cr[c]));
    }
  }
}

// Deterministic split-K reduction: partial sums are added in split order 0..S-1.
// INT: the partial planes hold int32 values (the exact-integer kernel writes
// them as such); they are summed in int32, then C (beta in {0, 1}) is added.
// Plane s holds rows of ldp elements (whole 128-byte lines).  Each thread
// takes 4 consecutive columns of a row; VEC: 16-byte loads of the partials
// and 16-byte accesses of C (columns beyond the last full group of 4 one by
// one).  Launched as a programmatic dependent of the GEMM that writes the
// partials: its blocks are placed while that grid drains and wait for it (and
// its memory) before the first read; the next kernel may place its own
// blocks once these have started.
template <bool INT, bool VEC>
__global__ void splitk_reduce_kernel(const float* __restrict__ P, int splits, int rows, int cols, long long ldp,
                                     float alpha, float beta, void* C, long long ldc) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const long long plane = (long long)rows * ldp;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) * 4; c < cols; c += gridDim.x * blockDim.x * 4) {
      const long long off = (long long)r * ldp + c;
      if (VEC && c + 4 <= cols) {
        if (INT) {
          int4 acc = make_int4(0, 0, 0, 0);
          for (int s = 0; s < splits; ++s) {
            const int4 v = *reinterpret_cast<const int4*>(reinterpret_cast<const int*>(P) + s * plane + off);
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
          }
          int4* cp = reinterpret_cast<int4*>(static_cast<int*>(C) + r * ldc + c);
          if (beta != 0.f) {
            const int4 o = *cp;
            acc.x += o.x; acc.y += o.y; acc.z += o.z; acc.w += o.w;
          }
          *cp = acc;
        } else {
          float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int s = 0; s < splits; ++s) {
            const float4 v = *reinterpret_cast<const float4*>(P + s * plane + off);
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
          }
          float4* cp = reinterpret_cast<float4*>(static_cast<float*>(C) + r * ldc + c);
          if (beta != 0.f) {
            const float4 o = *cp;
            acc = make_float4(fmaf(alpha, acc.x, beta * o.x), fmaf(alpha, acc.y, beta * o.y),
                              fmaf(alpha, acc.z, beta * o.z), fmaf(alpha, acc.w, beta * o.w));
          } else {
            acc = make_float4(alpha * acc.x, alpha * acc.y, alpha * acc.z, alpha * acc.w);
          }
          *cp = acc;
        }
        continue;
      }
      for (int u = c; u < c + 4 && u < cols; ++u) {
        const long long o = (long long)r * ldp + u;
        if (INT) {
          int s32 = 0;
          const int* Pi = reinterpret_cast<const int*>(P);
          for (int s = 0; s < splits; ++s) s32 += Pi[s * plane + o];
          int* cp = static_cast<int*>(C) + r * ldc + u;
          *cp = (beta != 0.f) ? (*cp + s32) : s32;
        } else {
          float sum = 0.f;
          for (int s = 0; s < splits; ++s) sum += P[s * plane + o];
          float* cp = static_cast<float*>(C) + r * ldc + u;
          *cp = (beta != 0.f) ? fmaf(alpha, sum, beta * *cp) : alpha * sum;
        }
      }
    }
  }
}

}  // namespace g3
