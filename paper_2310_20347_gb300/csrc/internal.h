// internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <mutex>

#include "simt_dgemm.cuh"
#include "simt_i16gemm.cuh"
#include "simt_sgemm.cuh"
#include "tc_gemm.cuh"

namespace g3 {

// maps: A, B of operand planes 0, 1, 2, then C (used only when p.c_tma); the
// launcher sizes the persistent grid from the tile count and `sms`.
using TcLaunchFn = cudaError_t (*)(const CUtensorMap* maps, const TcParams& p, int sms, cudaStream_t s);

// One member of the generated tensor-core kernel family.
struct FamilyEntry {
  int index;
  int mode;     // TcMode
  int bm;       // output rows per tile (= MMA N)
  int stages;   // shared-memory ring depth
  int smem;     // dynamic shared memory bytes
  int bufs;     // TMEM accumulator sets (2: the epilogue overlaps the next tile)
  int cg;       // CTAs per MMA: 1, or 2 (a CTA pair; tiles are 256 columns wide)
  TcLaunchFn launch;
  int (*slots)(int sms);   // CTAs (pairs) that can be resident at once; 0 on error
  bool stream_k;           // takes a stream-K tail (TcParams::sk_*)
  bool raw8;               // INT8 member reading the int8 operands as they are (converted in the kernel)
};

void register_family_bf16(FamilyEntry* table);
void register_family_3xbf16(FamilyEntry* table);
void register_family_fp8(FamilyEntry* table);
void register_family_int8emu(FamilyEntry* table);
void register_family_6xbf16(FamilyEntry* table);
void register_family_f16(FamilyEntry* table);
void register_family_tf32(FamilyEntry* table);
void register_family_3xtf32(FamilyEntry* table);

using GroupedLaunchFn = cudaError_t (*)(const GroupedParams& p, int grid, cudaStream_t s);

// One persistent grouped kernel (tiles of at most bm_max rows).  fused = 1:
// the FP32-accurate split inside the kernel (FP32 A and B read through the
// problem table, no preparation jobs for them).
struct GroupedEntry {
  int index;
  int mode;
  int bm_max;
  int stages;
  int smem;
  GroupedLaunchFn launch;
  int fused;
};

void register_grouped_bf16(GroupedEntry* table);
void register_grouped_3xbf16(GroupedEntry* table);
void register_grouped_fp8(GroupedEntry* table);
void register_grouped_int8emu(GroupedEntry* table);
void register_grouped_6xbf16(GroupedEntry* table);
void register_grouped_f16(GroupedEntry* table);
void register_grouped_tf32(GroupedEntry* table);
void register_grouped_3xtf32(GroupedEntry* table);

// kernels.cu: launchers of the non-tensor-core kernels.  Each returns the
// launch's cudaError_t; sizes are validated by the caller.
cudaError_t launch_simt(const SimtParams& p, bool vec, int kind, int splits, cudaStream_t s);
cudaError_t launch_simt64(const SimtParams64& p, bool vec, cudaStream_t s);
cudaError_t launch_simt_i16(const SimtParamsI16& p, cudaStream_t s);
// C := beta * C in binary64 (beta == 0 writes zeros without reading C).
cudaError_t launch_scale_c_f64(double* C, int rows, int cols, long long ldc, double beta, cudaStream_t s);
cudaError_t launch_split_bf16(const float* x, int rows, int cols, long long ldx, uint16_t* hi, uint16_t* lo,
                              long long ldy, cudaStream_t s);
// The split of both operands of a call in one launch (two launches when a
// matrix's rows are not 16-byte aligned).
cudaError_t launch_split_bf16_pair(const float* xa, int rows_a, int cols_a, long long lda, uint16_t* ahi, uint16_t* alo,
                                   long long lda_p, const float* xb, int rows_b, int cols_b, long long ldb,
                                   uint16_t* bhi, uint16_t* blo, long long ldb_p, cudaStream_t s);
cudaError_t launch_split3_bf16_pair(const float* xa, int rows_a, int cols_a, long long lda, uint16_t* ahi,
                                    uint16_t* amid, uint16_t* alo, long long lda_p, const float* xb, int rows_b,
                                    int cols_b, long long ldb, uint16_t* bhi, uint16_t* bmid, uint16_t* blo,
                                    long long ldb_p, cudaStream_t s);
cudaError_t launch_int8_to_bf16_pair(const int8_t* xa, int rows_a, int cols_a, long long lda, uint16_t* ya,
                                     long long lda_p, const int8_t* xb, int rows_b, int cols_b, long long ldb,
                                     uint16_t* yb, long long ldb_p, cudaStream_t s);
cudaError_t launch_split3_bf16(const float* x, int rows, int cols, long long ldx, uint16_t* hi, uint16_t* mid,
                               uint16_t* lo, long long ldy, cudaStream_t s);
// y = x rounded to TF32 (nearest, ties to even), kept as binary32.
cudaError_t launch_convert_tf32(const float* x, int rows, int cols, long long ldx, float* y, long long ldy,
                                cudaStream_t s);
// y (cols x rows) = transpose of x rounded to TF32: B of the TF32 mode, K-major.
cudaError_t launch_convert_tf32_t(const float* x, int rows, int cols, long long ldx, float* y, long long ldy,
                                  cudaStream_t s);
cudaError_t launch_convert_bf16(const float* x, int rows, int cols, long long ldx, uint16_t* y, long long ldy,
                                cudaStream_t s);
// hi = tf32(x), lo = tf32(x - hi); the _t form writes both transposed (cols x rows).
cudaError_t launch_split_tf32(const float* x, int rows, int cols, long long ldx, float* hi, float* lo,
                             long long ldy, cudaStream_t s);
cudaError_t launch_split_tf32_t(const float* x, int rows, int cols, long long ldx, float* hi, float* lo,
                               long long ldy, cudaStream_t s);
cudaError_t launch_int8_to_bf16(const int8_t* x, int rows, int cols, long long ldx, uint16_t* y, long long ldy,
                                cudaStream_t s);
// y (cols x rows) := transpose of x (rows x cols), elements of esize bytes (1, 2 or 4).
cudaError_t launch_transpose(const void* x, int rows, int cols, long long ldx, void* y, long long ldy, int esize,
                             cudaStream_t s);
cudaError_t launch_pack_rows(const void* x, int rows, long long row_bytes, long long ldx_bytes, void* y,
                             long long ldy_bytes, cudaStream_t s);
cudaError_t launch_quantize_e4m3(const float* x, int rows, int cols, long long ldx, unsigned int* amax_bits,
                                 uint8_t* q, long long ldq, float* scale, cudaStream_t s);
cudaError_t launch_scale_c(void* C, bool is_int, int rows, int cols, long long ldc, float beta, cudaStream_t s);
cudaError_t launch_splitk_reduce(const float* P, int splits, int rows, int cols, long long ldp, float alpha,
                                 float beta, void* C, long long ldc, bool is_int, cudaStream_t s);

// Stream-K fix-up: for each of the `tail` last tiles of the walk (sched.cuh),
// the sum of its segments' partial tiles in stream order, then
// C := alpha * scale_a * scale_b * sum + beta * C (int32: C := sum (+ C)).
struct SkFixup {
  const float* partial;   // [streams * segs][bm][bn] FP32 (int32 bits when is_int)
  int streams, segs, dp, tail, num_kb;
  int tiles_m, tiles_n, raster, bm, bn;
  int m, n;
  float alpha, beta;
  const float* scale_a;   // device scalars (FP8), or null = 1
  const float* scale_b;
  void* C;
  long long ldc;
  bool is_int;
};
cudaError_t launch_streamk_fixup(const SkFixup& f, cudaStream_t s);
cudaError_t launch_stream_traffic(const void* in, long long in_units, void* out, long long out_units, int sms,
                                  cudaStream_t s);

// Number of kernel launches the library has issued (all translation units).
void count_launch(int n = 1);

// api.cu services.  Callers of the functions below hold api_mutex().
struct DeviceInfo {
  int device;
  int sms;
  int* status;   // device status word of the watchdog
};
std::mutex& api_mutex();
int current_device_info(DeviceInfo* out);
int encode_tensor_2d(CUtensorMap* map, const void* base, int esize, uint64_t inner, uint64_t outer, uint64_t ld,
                     uint32_t box_inner, uint32_t box_outer);
unsigned long long watchdog_timeout_ns();
bool kernel_timing_enabled();
void kernel_timing_push(cudaEvent_t e0, cudaEvent_t e1);
bool take_withhold(unsigned long long* timeout_ns);   // one-shot failure-detection test hook
// Tile height (64 or 128) g3_autotune_grouped recorded for the size bucket of
// (m, n, k) and dtype, 0 if none; store one.
int tuned_grouped_bm(int64_t m, int64_t n, int64_t k, int dtype);
void store_grouped_tuning(int64_t m, int64_t n, int64_t k, int dtype, int bm, double ms);

// Every device allocation the library makes goes through device_alloc, which
// counts the successful ones (g3_debug_device_allocations reads the count).
cudaError_t device_alloc(void** p, size_t bytes);

}  // namespace g3
