// bf16.cuh -- bfloat16 bit-pattern helpers (round to nearest even via the CUDA intrinsic).
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace g3 {

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_value(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

}  // namespace g3
