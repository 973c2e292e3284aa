// api.cu -- the C ABI of include/g3gemm.h: argument validation, the planner
// (per-shape choice of a member of the generated kernel family, split-K and
// raster), library workspace, TMA descriptor encoding and dispatch.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "g3gemm.h"
#include "family_gen.inc"
#include "internal.h"

namespace g3 {

__device__ int g_device_status;   // first watchdog code raised since the last query
uint64_t launch_count();

namespace {
std::atomic<long long> g_device_allocs{0};
}

cudaError_t device_alloc(void** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_device_allocs.fetch_add(1, std::memory_order_relaxed);
  return e;
}

namespace {

constexpr int kMaxDevices = 64;

constexpr int kHostMaxBlocks = 8;   // row blocks of a g3_gemm_host pipeline
constexpr int kHostMaxSlabs = 4;    // k-slabs in which g3_gemm_host sends B up (FP32-accurate)
constexpr int kHostPipes = 4;       // caller streams with g3_gemm_host device copies of their own

// g3_gemm_host state of one caller stream: device copies of A, B, C (and
// B's prepared planes), scratch for the block GEMMs, two copy streams and
// the pipeline's events.  free_ev, recorded on the caller's stream after a
// call's last download, orders the next call that takes these buffers.
struct HostPipe {
  bool used = false;
  cudaStream_t owner = nullptr;
  uint64_t last_use = 0;
  void* buf = nullptr;
  size_t bytes = 0;
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t ev[2 * kHostMaxBlocks + kHostMaxSlabs + 3] = {};
  cudaEvent_t free_ev = nullptr;
  bool free_recorded = false;
};

struct DevState {
  bool init = false;
  int sms = 0;
  int* status = nullptr;   // device address of g_device_status
  void* ws = nullptr;      // library-owned workspace
  size_t ws_bytes = 0;
  // row-major copies of transposed operands (trans_a / trans_b)
  void* tbuf = nullptr;
  size_t tbuf_bytes = 0;
  // g3_gemm_host: per caller stream (the least recently used one is taken
  // over by a new stream)
  HostPipe pipes[kHostPipes];
  uint64_t pipe_tick = 0;
};

std::mutex g_mu;
DevState g_dev[kMaxDevices];
cudaStream_t g_stream = nullptr;
FamilyEntry g_family[G3_FAMILY_SIZE];
bool g_family_ready = false;
bool g_timing = false;
bool g_withhold_next = false;              // failure-detection test hook
unsigned long long g_withhold_timeout_ns = 0;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_events;

unsigned long long watchdog_ns() {
  static unsigned long long ns = [] {
    const char* e = std::getenv("G3_WATCHDOG_MS");
    long long ms = e ? std::atoll(e) : 2000;
    if (ms <= 0) ms = 2000;
    return (unsigned long long)ms * 1000000ULL;
  }();
  return ns;
}

void family_init() {
  if (g_family_ready) return;
  std::memset(g_family, 0, sizeof(g_family));
  register_family_bf16(g_family);
  register_family_3xbf16(g_family);
  register_family_fp8(g_family);
  register_family_int8emu(g_family);
  register_family_6xbf16(g_family);
  register_family_f16(g_family);
  register_family_tf32(g_family);
  register_family_3xtf32(g_family);
  g_family_ready = true;
}

int ensure_device(DevState** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return G3_ERR_NOT_INIT;
  }
  DevState& d = g_dev[dev];
  if (!d.init) {
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return G3_ERR_NOT_INIT;
    }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) {
      cudaGetLastError();
      return G3_ERR_CUDA;
    }
    d.status = static_cast<int*>(p);
    d.init = true;
  }
  family_init();
  *out = &d;
  return G3_OK;
}

// ---------------------------------------------------------------- TMA descriptors
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

using EncodeIm2colFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const int*, const int*, cuuint32_t, cuuint32_t,
                                    const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeIm2colFn encode_im2col_fn() {
  static EncodeIm2colFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeIm2col", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeIm2colFn) nullptr;
    }
    return reinterpret_cast<EncodeIm2colFn>(p);
  }();
  return fn;
}

// Geometry of an implicit-GEMM convolution (g3_conv2d).
struct ConvDesc {
  int64_t N, H, W, C, K, R, S, sh, sw, ph, pw, dh, dw, P, Q;
};

// The NHWC activation tensor as a 4-D im2col tensor map (dims C, W, H, N): a
// load walks `pixels` output positions -- base positions from (-pad) in steps
// of the stride, inside the box that ends where the last filter tap still
// overlaps the padded image -- and reads 64 channels of each.
int encode_im2col(CUtensorMap* map, const void* x, int esize, const ConvDesc& c, uint32_t pixels) {
  EncodeIm2colFn fn = encode_im2col_fn();
  if (!fn) return G3_ERR_CUDA;
  cuuint64_t dims[4] = {(cuuint64_t)c.C, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)c.N};
  cuuint64_t strides[3] = {(cuuint64_t)(c.C * esize), (cuuint64_t)(c.W * c.C * esize),
                           (cuuint64_t)(c.H * c.W * c.C * esize)};
  int lower[2] = {(int)-c.pw, (int)-c.ph};
  int upper[2] = {(int)(c.pw - (c.S - 1) * c.dw), (int)(c.ph - (c.R - 1) * c.dh)};
  cuuint32_t estr[4] = {1, (cuuint32_t)c.sw, (cuuint32_t)c.sh, 1};
  const CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;   // 2-byte elements; the bytes are copied as is
  CUresult r = fn(map, dt, 4, const_cast<void*>(x), dims, strides, lower, upper, 64, pixels, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? G3_OK : G3_ERR_CUDA;
}

// A row-major matrix of `outer` rows x `inner` elements (leading dimension ld
// elements) as a 2-D tensor, loaded in boxes of box_inner x box_outer with the
// 128-byte swizzle; out-of-range elements of a box read as zero.
int encode_2d(CUtensorMap* map, const void* base, int esize, uint64_t inner, uint64_t outer, uint64_t ld,
              uint32_t box_inner, uint32_t box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return G3_ERR_CUDA;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {ld * (uint64_t)esize};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                : (esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8);
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? G3_OK : G3_ERR_CUDA;
}

// A row-major int8 matrix (outer rows x inner bytes, leading dimension ld
// bytes) in unswizzled boxes of box_inner x box_outer: the raw tiles of the
// RAW8 members; out-of-range bytes read as zero.
int encode_raw8_2d(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_inner,
                   uint32_t box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return G3_ERR_CUDA;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {ld};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? G3_OK : G3_ERR_CUDA;
}

// C (m rows x n columns of 4-byte elements, leading dimension ldc) for TMA
// stores of 32-row x 128-column boxes, no swizzle (row-major staging tile).
int encode_c_2d(CUtensorMap* map, void* base, bool is_int, uint64_t n, uint64_t m, uint64_t ldc) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return G3_ERR_CUDA;
  cuuint64_t dims[2] = {n, m};
  cuuint64_t strides[1] = {ldc * 4};
  cuuint32_t box[2] = {128, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, is_int ? CU_TENSOR_MAP_DATA_TYPE_INT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? G3_OK : G3_ERR_CUDA;
}

// The split-K partial planes (splits x m rows x n columns of 4-byte elements,
// row stride ldp, plane stride m * ldp) for TMA stores of 32-row x
// 128-column boxes into plane z; a box is clipped at its plane's edges.
int encode_partial_3d(CUtensorMap* map, void* base, bool is_int, uint64_t n, uint64_t m, uint64_t splits,
                      uint64_t ldp) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return G3_ERR_CUDA;
  cuuint64_t dims[3] = {n, m, splits};
  cuuint64_t strides[2] = {ldp * 4, m * ldp * 4};
  cuuint32_t box[3] = {128, 32, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, is_int ? CU_TENSOR_MAP_DATA_TYPE_INT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? G3_OK : G3_ERR_CUDA;
}

bool tma_ok(const void* p, int64_t ld, int esize) {
  return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && ((ld * esize) % 16 == 0);
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ---------------------------------------------------------------- planner
// FP32-accurate GEMMs with k <= 512 take the three-part split (6 products):
// at small k the two-part split's dropped terms exceed 2e-6 of sum |a||b|.
// 512 is a power of two, so one tuning-cache k bucket never mixes the modes.
constexpr int64_t kSixProductMaxK = 512;

int tc_mode_of(int dtype, int64_t k) {
  switch (dtype) {
    case G3_BF16: return TC_BF16;
    case G3_FP16: return TC_F16;
    case G3_TF32: return TC_TF32;
    case G3_F32_3XTF32: return TC_3XTF32;
    case G3_F32_3XBF16: return k <= kSixProductMaxK ? TC_6XBF16 : TC_3XBF16;
    case G3_FP8_E4M3: return TC_FP8;
    case G3_INT8: return TC_I8EMU;  // exact emulation: int8 values are exact in bfloat16
    default: return -1;
  }
}

// k per k-block: one 128-byte row of the swizzled tile
int kblock_of(int mode) { return mode == TC_FP8 ? 128 : ((mode == TC_TF32 || mode == TC_3XTF32) ? 32 : 64); }

struct Plan {
  int member = -1;
  int splits = 1;
  int kb_per_split = 1;
  int num_kb = 1;
  int tiles_m = 1, tiles_n = 1;
  int raster = 8;
  int sk_streams = 0, sk_dp = 0, sk_tail = 0, sk_segs = 0;   // stream-K tail (sched.cuh); 0 streams = none
};

// Clocks one k-block of a tile costs a member, measured on GB300: the MMA
// time (73 clocks per MMA of 128 x 128 x 16, x 2 for N = 256, times the
// products per k-step), the shared-memory fill (about 64 bytes per clock per
// SM), or the load latency the ring must cover (about 3000 clocks for one
// CTA, 4400 for a CTA pair, whose stages complete only when both CTAs' loads
// have landed) spread over its stages -- whichever is largest; a two-stage
// ring exposes part of every refill.
double kblock_clocks(const FamilyEntry& f) {
  const int products = (f.mode == TC_3XBF16 || f.mode == TC_3XTF32) ? 3 : (f.mode == TC_6XBF16 ? 6 : 1);
  const double mma = 4.0 * products * 73.0 * f.bm / 128.0;
  const double stage_bytes = (double)(f.smem - 1024 - 2 * 32 * 128 * 4 - 256) / f.stages;
  const double fill = stage_bytes / 64.0;
  const double lat = (f.cg > 1 ? 4400.0 : 3000.0) / f.stages;
  double t = std::max(mma, std::max(fill, lat));
  if (f.stages <= 2) t *= 1.07;
  return t;
}

// Time one CTA (or pair) spends on one output tile, in ns: the main loop
// (k-blocks at kblock_clocks, 1.9 GHz) and the epilogue, which writes the
// CTA's bm x 128 block of C at about 22 bytes per ns per SM (the rate C leaves
// at when every SM writes, ~3.4 TB/s in all) plus ~1.5 us of TMEM, barrier and
// store latency (0.6 us more for a pair's cluster hand-offs) -- fitted to the
// im2col layers, where tiles of 1 to 8 k-blocks spend longer in the epilogue
// than in the main loop.  With two or more accumulator sets the epilogue of
// one tile overlaps the main loop of the next, so the slower of the two sets
// the pace; with one set they add up.
double tile_time_ns(const FamilyEntry& f, int num_kb) {
  const double t_main = num_kb * kblock_clocks(f) / 1.9;
  const double t_epi = f.bm * 128.0 * 4.0 / 22.0 + 1500.0 + (f.cg > 1 ? 600.0 : 0.0);
  return f.bufs >= 2 ? std::max(t_main, t_epi) : t_main + t_epi;
}


// ---------------------------------------------------------------- tuning cache
// Results of g3_autotune, keyed by dtype and the power-of-two bucket of each of
// m, n, k (the smallest b with 2^b >= x); the planner prefers them to its model.
struct TuneKey {
  int dtype, bm, bn, bk;
  bool operator<(const TuneKey& o) const {
    return std::tie(dtype, bm, bn, bk) < std::tie(o.dtype, o.bm, o.bn, o.bk);
  }
};
struct TuneVal {
  int member, split;
  double ms;
};
std::map<TuneKey, TuneVal> g_tune;
// Records of g3_autotune_grouped share the table under dtype + kGroupedTuneTag;
// their "member" is the tile height (64 or 128 rows) of a grouped problem.
constexpr int kGroupedTuneTag = 100;
bool g_tune_env_loaded = false;

int size_bucket(int64_t x) {
  int b = 0;
  while ((int64_t(1) << b) < x && b < 62) ++b;
  return b;
}
TuneKey tune_key(int64_t m, int64_t n, int64_t k, int dtype) {
  return TuneKey{dtype, size_bucket(m), size_bucket(n), size_bucket(k)};
}

int tune_load_locked(const char* path) {
  FILE* f = std::fopen(path, "r");
  if (!f) return -101;
  char line[256];
  int loaded = 0;
  while (std::fgets(line, sizeof line, f)) {
    TuneKey key;
    TuneVal val;
    if (line[0] == '#') continue;
    if (std::sscanf(line, "%d %d %d %d %d %d %lf", &key.dtype, &key.bm, &key.bn, &key.bk, &val.member, &val.split,
                    &val.ms) != 7)
      continue;
    const bool grouped = key.dtype >= kGroupedTuneTag;   // grouped record: member = tile height
    if (grouped ? ((val.member == 64 || val.member == 128) && val.split == 1)
                : (val.member >= 0 && val.member < G3_FAMILY_SIZE && (val.split >= 1 || val.split == G3_SPLIT_STREAM_K))) {
      g_tune[key] = val;
      ++loaded;
    }
  }
  std::fclose(f);
  return loaded;
}

void tune_env_once() {
  if (g_tune_env_loaded) return;
  g_tune_env_loaded = true;
  if (const char* p = std::getenv("G3_TUNE_CACHE")) tune_load_locked(p);
}

Plan make_plan(int64_t m, int64_t n, int64_t k, int dtype, int sms, int force_member, int force_split,
               int force_raster, bool allow_splitk = true) {
  Plan pl;
  bool automatic = force_member < 0;   // the member is the planner's own choice
  if (force_member < 0 && force_split == 0) {
    tune_env_once();
    auto it = g_tune.find(tune_key(m, n, k, dtype));
    if (it != g_tune.end()) {
      force_member = it->second.member;
      force_split = it->second.split;
      automatic = false;
    }
  }
  const int mode = tc_mode_of(dtype, k);
  const int bk = kblock_of(mode);
  pl.num_kb = (int)((k + bk - 1) / bk);
  // Modelled time of a member with s splits of k: waves of tiles (the
  // member's resident CTAs or pairs, as the device reports them, else the SM
  // count over the cluster size) x the time of one tile of ceil(num_kb / s)
  // k-blocks, plus, when split, the reduce kernel: ~2 us of launch and
  // dependency latency in a stream of calls, and s partial planes plus C at
  // ~6 TB/s (partial tiles leave through TMA stores; the reduce reads 16 bytes
  // per access).
  const bool search_split = force_split == 0 && allow_splitk;
  auto cost_of = [&](const FamilyEntry& f, int s) {
    const long long tiles = ((m + f.bm - 1) / f.bm) * ((n + 128LL * f.cg - 1) / (128LL * f.cg));
    const int resident = f.slots ? f.slots(sms) : 0;
    const long long slots = resident > 0 ? resident : std::max(1, sms / f.cg);
    const long long waves = (tiles * s + slots - 1) / slots;
    const int kb = (pl.num_kb + s - 1) / s;
    double t = (double)waves * tile_time_ns(f, kb);
    if (s > 1) t += 2000.0 + (double)(s + 1) * (double)m * (double)n * 4.0 / 6000.0;
    return t;
  };
  auto splits_for = [&](const FamilyEntry& f, auto&& visit) {
    visit(1);
    if (!search_split) return;
    const long long tiles = ((m + f.bm - 1) / f.bm) * ((n + 128LL * f.cg - 1) / (128LL * f.cg));
    const long long slots = std::max(1, sms / f.cg);
    for (int s : {2, 3, 4, 6, 8, 12, 16})   // pieces of at least two k-blocks, at most ~2 waves of them
      if (2 * s <= pl.num_kb && tiles * s <= 2 * slots) visit(s);
  };
  int best_split = 1;
  if (force_member >= 0 && force_member < G3_FAMILY_SIZE && g_family[force_member].mode == mode &&
      g_family[force_member].launch) {
    pl.member = force_member;
    double best = 1e300;
    splits_for(g_family[force_member], [&](int s) {
      const double c = cost_of(g_family[force_member], s);
      if (c < best * 0.999) { best = c; best_split = s; }
    });
  } else {
    double best = 1e300;
    for (int i = 0; i < G3_FAMILY_SIZE; ++i) {
      const FamilyEntry& f = g_family[i];
      if (!f.launch || f.mode != mode || f.raw8) continue;
      // first (deepest) variant per (bm, cg)
      if (pl.member >= 0 && g_family[pl.member].bm == f.bm && g_family[pl.member].cg == f.cg) continue;
      splits_for(f, [&](int s) {
        const double c = cost_of(f, s);
        if (c < best * 0.999) { best = c; pl.member = i; best_split = s; }
      });
    }
  }
  if (pl.member < 0) return pl;
  // INT8 on one CTA: a twin that reads the int8 operands as they are
  // replaces the int8 -> bf16 conversion pass (CTA pairs keep it).  RAW8
  // members split k so that every split is one exact accumulation chunk (16
  // k-blocks, 1024 products); past one chunk the 128-row twin, whose tiles
  // convert fewer blocks of B per output (measured on the deep im2col layers:
  // 256 x 3136 x 2304 15.8 us against 18.9 with 64 rows and 20.3 with the
  // pass; 512 x 784 x 4608 16.5 against 25.5).
  if (automatic && mode == TC_I8EMU && g_family[pl.member].cg == 1 && !g_family[pl.member].raw8) {
    const int want = pl.num_kb > 16 ? 128 : std::min(g_family[pl.member].bm, 128);
    for (int i = 0; i < G3_FAMILY_SIZE; ++i)
      if (g_family[i].launch && g_family[i].raw8 && g_family[i].bm == want) {
        pl.member = i;
        break;
      }
  }
  const int bm = g_family[pl.member].bm;
  const int cg = g_family[pl.member].cg;
  pl.tiles_n = (int)((n + 128LL * cg - 1) / (128LL * cg));
  pl.tiles_m = (int)((m + bm - 1) / bm);
  const long long tiles = (long long)pl.tiles_m * pl.tiles_n;
  (void)tiles;
  int splits = 1;
  if (force_split > 0) splits = force_split;
  else if (force_split == 0) splits = best_split;
  if (!allow_splitk) splits = 1;
  // FP32-accurate modes: a bounded k per FP32 accumulator.  The tensor core
  // adds each k-step's products to its FP32 accumulator with truncation, so the
  // error grows as sqrt(k) / (k-step depth) * 2^-23 of sum |a||b| -- measured
  // 1.04e-6 for 3xBF16 (16-deep steps) and 1.9e-6 for 3xTF32 (8-deep) at
  // k = 16384, against the 2e-6 these modes promise; s partial sums added in
  // round-to-nearest cut it by s.  At most 32768 of k (3xBF16) or 8192
  // (3xTF32) per accumulator; split-K beyond.
  if (force_split == 0 && mode == TC_3XTF32) splits = std::max(splits, (pl.num_kb + 255) / 256);
  if (force_split == 0 && mode == TC_3XBF16) splits = std::max(splits, (pl.num_kb + 511) / 512);
  // RAW8 members: every split within one exact FP32 chunk of 16 k-blocks
  if (g_family[pl.member].raw8) splits = std::max(splits, (pl.num_kb + 15) / 16);
  splits = std::min(splits, pl.num_kb);
  pl.kb_per_split = (pl.num_kb + splits - 1) / splits;
  pl.splits = (pl.num_kb + pl.kb_per_split - 1) / pl.kb_per_split;
  pl.raster = force_raster > 0 ? force_raster : 8;
  pl.raster = std::max(1, std::min(pl.raster, pl.tiles_m));
  // Stream-K tail (sched.cuh), by request only (split_k = G3_SPLIT_STREAM_K,
  // or a tuning record of g3_autotune, which times it among the candidates).
  // The planner does not choose it by itself: measured on GB300 (FP32-accurate
  // 2048^3, BF16 4096^3, INT8 8192^3) the last, partly idle wave of whole
  // tiles runs nearly in proportion to its tile count -- fewer busy SMs share
  // L2 and HBM -- so cutting it into segments saved at most 3% of the GEMM
  // kernel (and cost 7% with the 256 x 256 pair tiles, whose segments each
  // write a 128 KB partial per CTA) while the fix-up pass took 12-14 us.
  const FamilyEntry& f = g_family[pl.member];
  if (pl.splits == 1 && force_split == G3_SPLIT_STREAM_K && f.slots && f.stream_k) {
    const int slots = f.slots(sms);
    if (slots > 0 && slots <= 1024) {
      const long long waves = tiles / slots, tail = tiles - waves * slots;
      if (tail > 0) {
        const StreamK sk{tail * pl.num_kb, slots, pl.num_kb};
        int segs = 0;
        for (int c = 0; c < slots; ++c) segs = std::max(segs, sk.segments(c));
        pl.sk_streams = slots;
        pl.sk_dp = (int)(waves * slots);
        pl.sk_tail = (int)tail;
        pl.sk_segs = segs;
      }
    }
  }
  return pl;
}

// ---------------------------------------------------------------- workspace layout
struct Layout {
  bool pack_a = false, pack_b = false;
  int64_t lda_p = 0, ldb_p = 0;   // leading dimensions of re-packed / converted operands
  size_t a_hi = 0, a_lo = 0, b_hi = 0, b_lo = 0, partial = 0, amax = 0;
  size_t a_mid = 0, b_mid = 0;    // middle planes of the three-part split
  size_t total = 0;
};

// B of the FP32-accurate mode already split into bf16 hi / lo planes (leading
// dimension ld), as g3_gemm_host keeps them for all the row blocks of a call.
struct PreparedB {
  const uint16_t* hi;
  const uint16_t* lo;
  int64_t ld;
};

Layout make_layout(const g3_gemm_args& a, const Plan& pl, bool b_prepared = false) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const int64_t m = a.m, n = a.n, k = a.k;
  switch (a.dtype) {
    case G3_F32_3XBF16:
      L.lda_p = round_up(k, 8);
      L.ldb_p = round_up(n, 8);
      L.a_hi = take((size_t)m * L.lda_p * 2);
      L.a_lo = take((size_t)m * L.lda_p * 2);
      if (!b_prepared) {
        L.b_hi = take((size_t)k * L.ldb_p * 2);
        L.b_lo = take((size_t)k * L.ldb_p * 2);
      }
      if (tc_mode_of(a.dtype, k) == TC_6XBF16) {
        L.a_mid = take((size_t)m * L.lda_p * 2);
        L.b_mid = take((size_t)k * L.ldb_p * 2);
      }
      break;
    case G3_TF32:   // rounded copies, binary32; B transposed (n x k, K-major)
      L.pack_a = L.pack_b = true;
      L.lda_p = round_up(k, 4);
      L.ldb_p = round_up(k, 4);
      L.a_hi = take((size_t)m * L.lda_p * 4);
      L.b_hi = take((size_t)n * L.ldb_p * 4);
      break;
    case G3_F32_3XTF32:   // hi / lo TF32 planes, binary32; B's transposed (n x k, K-major)
      L.pack_a = L.pack_b = true;
      L.lda_p = round_up(k, 4);
      L.ldb_p = round_up(k, 4);
      L.a_hi = take((size_t)m * L.lda_p * 4);
      L.a_lo = take((size_t)m * L.lda_p * 4);
      L.b_hi = take((size_t)n * L.ldb_p * 4);
      L.b_lo = take((size_t)n * L.ldb_p * 4);
      break;
    case G3_INT8:
      if (pl.member >= 0 && g_family[pl.member].raw8) {
        // int8 read as it is: only rows TMA cannot address get an aligned copy
        L.pack_a = !tma_ok(a.A, a.lda, 1);
        L.pack_b = !tma_ok(a.B, a.ldb, 1);
        L.lda_p = L.pack_a ? round_up(k, 16) : a.lda;
        L.ldb_p = L.pack_b ? round_up(n, 16) : a.ldb;
        if (L.pack_a) L.a_hi = take((size_t)m * L.lda_p);
        if (L.pack_b) L.b_hi = take((size_t)k * L.ldb_p);
        break;
      }
      L.pack_a = L.pack_b = true;
      L.lda_p = round_up(k, 8);
      L.ldb_p = round_up(n, 8);
      L.a_hi = take((size_t)m * L.lda_p * 2);
      L.b_hi = take((size_t)k * L.ldb_p * 2);
      break;
    case G3_BF16:
    case G3_FP16:
    case G3_FP8_E4M3: {
      const int es = a.dtype == G3_FP8_E4M3 ? 1 : 2;
      L.pack_a = !tma_ok(a.A, a.lda, es);
      L.pack_b = !tma_ok(a.B, a.ldb, es);
      L.lda_p = L.pack_a ? round_up(k, 16 / es) : a.lda;
      L.ldb_p = L.pack_b ? round_up(n, 16 / es) : a.ldb;
      if (L.pack_a) L.a_hi = take((size_t)m * L.lda_p * es);
      if (L.pack_b) L.b_hi = take((size_t)k * L.ldb_p * es);
      break;
    }
    default:
      break;
  }
  // split-K partial planes: rows padded to whole 128-byte lines
  if (a.dtype != G3_F32 && pl.splits > 1) L.partial = take((size_t)pl.splits * m * round_up(n, 32) * 4);
  if (a.dtype != G3_F32 && pl.sk_streams > 0) {
    const FamilyEntry& f = g_family[pl.member];
    L.partial = take((size_t)pl.sk_streams * pl.sk_segs * f.bm * 128 * f.cg * 4);
  }
  L.total = off;
  return L;
}

// Long launches claim their tiles (TcParams::tile_ctr) instead of walking
// them statically: at least kClaimMinWaves waves of work items, no stream-K
// tail, not a RAW8 member.  Over a long launch the CTAs of a static walk
// drift apart by more than the time L2 keeps a panel, so the tiles sharing a
// panel of B read it from DRAM one by one; claimed tiles run together in
// claim order.  The counter (one int, zeroed by a memset before the call's
// first launch) sits in the 256 bytes after the call's workspace layout; a
// caller-provided workspace without room for it keeps the static walk.
// G3_STATIC_WALK=1 in the environment forces the static walk (A/B timing).
constexpr int kClaimMinWaves = 16;
constexpr size_t kClaimBytes = 256;

bool claims_tiles(const Plan& pl, int sms) {
  if (pl.member < 0 || pl.sk_streams > 0) return false;
  const FamilyEntry& f = g_family[pl.member];
  if (f.raw8) return false;
  const char* e = std::getenv("G3_STATIC_WALK");
  if (e && e[0] == '1') return false;
  const int slots = f.slots(sms);
  const long long work = (long long)pl.tiles_m * pl.tiles_n * pl.splits;
  return slots > 0 && work >= (long long)kClaimMinWaves * slots;
}

// Band width of a claimed walk unless the caller forces one: as many tile
// rows (2 to 8) as keep the band's panels of A within 80 MiB of the 129 MB
// L2, so that they stay there while the B panels stream past, each read by
// the band's tiles claimed one after another.  Measured on the FP32-accurate
// 16384^3 pair member (16 MB of bf16 planes per 256-row panel), per launch:
// bands of 3, 4, 5, 6 rows 14.37, 14.06, 13.96, 13.92 ms, 8 rows 14.15-14.76
// ms (the static walk: 14.63-15.56 ms); 80 MiB gives 5 there.
constexpr double kClaimBandBytes = 80.0 * (1 << 20);

// Bytes of A one tile row of k holds in shared memory (all planes).
int staged_a_bytes(int mode) {
  switch (mode) {
    case TC_3XBF16: return 4;
    case TC_6XBF16: return 6;
    case TC_FP8: return 1;
    case TC_TF32: return 4;
    case TC_3XTF32: return 8;
    default: return 2;   // BF16, FP16, INT8 staged as bf16
  }
}

int walk_raster(const Plan& pl, bool claim, int forced) {
  if (!claim || forced > 0) return pl.raster;
  const FamilyEntry& f = g_family[pl.member];
  const double panel = (double)f.bm * pl.kb_per_split * kblock_of(f.mode) * staged_a_bytes(f.mode);
  const int band = std::max(2, std::min(8, (int)(kClaimBandBytes / std::max(panel, 1.0))));
  return std::min(band, pl.tiles_m);
}

int get_workspace(DevState& d, const g3_gemm_args& a, size_t need, uint8_t** out) {
  *out = nullptr;
  if (need == 0) return G3_OK;
  if (a.workspace) {
    if (a.workspace_bytes < need) return -(100 + 15);
    *out = static_cast<uint8_t*>(a.workspace);
    return G3_OK;
  }
  if (d.ws_bytes < need) {
    if (d.ws) {
      cudaDeviceSynchronize();
      cudaFree(d.ws);
      d.ws = nullptr;
      d.ws_bytes = 0;
    }
    const size_t sz = std::max<size_t>(round_up((int64_t)need, 64 << 20), 64 << 20);
    if (device_alloc(&d.ws, sz) != cudaSuccess) {
      cudaGetLastError();
      d.ws = nullptr;
      return G3_ERR_NOMEM;
    }
    d.ws_bytes = sz;
  }
  *out = static_cast<uint8_t*>(d.ws);
  return G3_OK;
}

// ---------------------------------------------------------------- timing
struct TimedRegion {
  cudaStream_t s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  explicit TimedRegion(cudaStream_t st) : s(st) {
    if (!g_timing) return;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  ~TimedRegion() {
    if (!e0) return;
    cudaEventRecord(e1, s);
    g_events.emplace_back(e0, e1);
  }
};

#define G3_CHECK_CUDA(expr)                   \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) {                  \
      if (std::getenv("G3_LOG"))              \
        std::fprintf(stderr, "g3gemm: %s: %s\n", #expr, cudaGetErrorString(_e)); \
      return G3_ERR_CUDA;                     \
    }                                         \
  } while (0)

// ---------------------------------------------------------------- validation
int validate(const g3_gemm_args& a) {
  if (a.m < 0) return -101;
  if (a.n < 0) return -102;
  if (a.k < 0) return -103;
  if (a.dtype < G3_F32 || a.dtype > G3_INT16) return -112;
  if (a.trans_a != 0 && a.trans_a != 1) return -119;
  if (a.trans_b != 0 && a.trans_b != 1) return -120;
  if (a.lda < std::max<int64_t>(1, a.trans_a ? a.m : a.k)) return -106;
  if (a.ldb < std::max<int64_t>(1, a.trans_b ? a.k : a.n)) return -108;
  if (a.ldc < std::max<int64_t>(1, a.n)) return -111;
  if (a.m == 0 || a.n == 0) return G3_OK;
  if (!a.C) return -110;
  if (a.k > 0 && a.alpha != 0.0) {
    if (!a.A) return -105;
    if (!a.B) return -107;
  }
  if (a.m > INT32_MAX || a.n > INT32_MAX || a.k > INT32_MAX) return G3_ERR_UNSUPPORTED;
  if (a.dtype == G3_INT8) {
    if (a.alpha != 1.0 && a.k > 0) return G3_ERR_UNSUPPORTED;
    if (a.beta != 0.0 && a.beta != 1.0) return G3_ERR_UNSUPPORTED;
    if (a.k > 131072) return G3_ERR_UNSUPPORTED;
  }
  if (a.dtype == G3_INT16) {
    if (a.alpha != 1.0 && a.k > 0) return G3_ERR_UNSUPPORTED;
    if (a.beta != 0.0 && a.beta != 1.0) return G3_ERR_UNSUPPORTED;
  }
  // the CUDA-core kernels put row blocks on grid.y: at most 65535 blocks of
  // 128 rows for FP32, of 64 rows for FP64 and INT16 (C := beta*C alone,
  // k == 0 or alpha == 0, has no such limit)
  if (a.k > 0 && a.alpha != 0.0) {
    if (a.dtype == G3_F32 && (a.m + 127) / 128 > 65535) return G3_ERR_UNSUPPORTED;
    if ((a.dtype == G3_F64 || a.dtype == G3_INT16) && (a.m + 63) / 64 > 65535) return G3_ERR_UNSUPPORTED;
  }
  return G3_OK;
}

// The FP32 SIMT kernel's blocking for an m x n x k problem: kind 0 (128 x 128
// blocks) while those fill the SMs; else kind 1 (64 x 64 blocks), with k cut
// over a cluster of 2, 4 or 8 CTAs while the grid stays within two CTAs per SM
// and every CTA keeps at least two k-blocks of 16.  split_k >= 2 (at most 8)
// forces that cluster split; split_k == 1 forbids it.
struct SimtPlan {
  int kind, splits;
};

SimtPlan simt_plan(int64_t m, int64_t n, int64_t k, int sms, int split_k) {
  const int64_t tiles128 = ((m + 127) / 128) * ((n + 127) / 128);
  const int64_t tiles64 = ((m + 63) / 64) * ((n + 63) / 64);
  const bool fits64 = (m + 63) / 64 <= 65535;
  if (split_k >= 2 && fits64) return {1, (int)std::min<int64_t>(std::min(split_k, 8), std::max<int64_t>(k, 1))};
  // enough 128 x 128 blocks for every SM: 128 x 256 blocks (8 x 16
  // micro-tiles) unless n would leave much of their width empty
  if (tiles128 >= sms || !fits64) return {(n % 256 == 0 || n >= 1024) ? 2 : 0, 1};
  if (tiles64 >= sms || split_k == 1) return {1, 1};
  int s = 1;
  for (int c = 2; c <= 8; c *= 2)
    if (tiles64 * c <= 2LL * sms && (k + c - 1) / c >= 32) s = c;
  return {1, s};
}

int run_simt(const g3_gemm_args& a, int sms, cudaStream_t s) {
  SimtParams p;
  p.m = (int)a.m;
  p.n = (int)a.n;
  p.k = (int)a.k;
  p.alpha = (float)a.alpha;
  p.beta = (float)a.beta;
  p.A = static_cast<const float*>(a.A);
  p.lda = a.lda;
  p.B = static_cast<const float*>(a.B);
  p.ldb = a.ldb;
  p.C = static_cast<float*>(a.C);
  p.ldc = a.ldc;
  const bool vec = (reinterpret_cast<uintptr_t>(a.A) % 16 == 0) && (reinterpret_cast<uintptr_t>(a.B) % 16 == 0) &&
                   (reinterpret_cast<uintptr_t>(a.C) % 16 == 0) && a.lda % 4 == 0 && a.ldb % 4 == 0 &&
                   a.ldc % 4 == 0;
  SimtPlan sp = simt_plan(a.m, a.n, a.k, sms, a.split_k);
  if (a.config >= 0 && a.config <= 3 && a.config != sp.kind) {   // a forced blocking
    if ((a.config != 1 && (a.m + 127) / 128 > 65535) || (a.config == 1 && (a.m + 63) / 64 > 65535))
      return G3_ERR_UNSUPPORTED;
    sp.kind = a.config;
    if (sp.kind != 1) sp.splits = 1;
  }
  TimedRegion tr(s);
  G3_CHECK_CUDA(launch_simt(p, vec, sp.kind, sp.splits, s));
  return G3_OK;
}

int run_simt64(const g3_gemm_args& a, cudaStream_t s) {
  SimtParams64 p;
  p.m = (int)a.m;
  p.n = (int)a.n;
  p.k = (int)a.k;
  p.alpha = a.alpha;
  p.beta = a.beta;
  p.A = static_cast<const double*>(a.A);
  p.lda = a.lda;
  p.B = static_cast<const double*>(a.B);
  p.ldb = a.ldb;
  p.C = static_cast<double*>(a.C);
  p.ldc = a.ldc;
  const bool vec = (reinterpret_cast<uintptr_t>(a.A) % 16 == 0) && (reinterpret_cast<uintptr_t>(a.B) % 16 == 0) &&
                   a.lda % 2 == 0 && a.ldb % 2 == 0;
  TimedRegion tr(s);
  G3_CHECK_CUDA(launch_simt64(p, vec, s));
  return G3_OK;
}

int run_simt_i16(const g3_gemm_args& a, cudaStream_t s) {
  SimtParamsI16 p;
  p.m = (int)a.m;
  p.n = (int)a.n;
  p.k = (int)a.k;
  p.beta = a.beta != 0.0 ? 1 : 0;
  p.A = static_cast<const int16_t*>(a.A);
  p.lda = a.lda;
  p.B = static_cast<const int16_t*>(a.B);
  p.ldb = a.ldb;
  p.C = static_cast<int64_t*>(a.C);
  p.ldc = a.ldc;
  TimedRegion tr(s);
  G3_CHECK_CUDA(launch_simt_i16(p, s));
  return G3_OK;
}

int input_esize(int dtype);
int untranspose(DevState& d, g3_gemm_args& a, cudaStream_t s);

// Whether dtype's kernels read a transposed operand in place (the one-plane
// 8- and 16-bit modes); the others get a row-major copy first.
bool reads_transposed(int dtype) { return dtype == G3_BF16 || dtype == G3_FP16 || dtype == G3_FP8_E4M3; }

int run_tc(DevState& d, const g3_gemm_args& a, cudaStream_t s, const ConvDesc* conv = nullptr,
           const PreparedB* pb = nullptr) {
  const bool dev_scales = a.dtype == G3_FP8_E4M3 && (a.scale_a || a.scale_b);
  const Plan pl = make_plan(a.m, a.n, a.k, a.dtype, d.sms, a.config, a.split_k, a.raster, !dev_scales);
  if (pl.member < 0) return G3_ERR_UNSUPPORTED;
  const FamilyEntry& fam = g_family[pl.member];
  if (a.trans_a || a.trans_b) {
    // Transposed operands are read in place when TMA can address them (16-byte
    // aligned base and row stride) and, for A stored k x m, when this CTA's
    // rows of the tile (bm / cg) fill whole 128-byte swizzle rows -- all but
    // the FP8 members with 64 rows per CTA.  Otherwise they are copied into
    // the row-major layout first.
    const int es = input_esize(a.dtype);
    const bool in_place = reads_transposed(a.dtype) && !conv && !pb &&
                          (!a.trans_a || (tma_ok(a.A, a.lda, es) && fam.bm / fam.cg * es >= 128)) &&
                          (!a.trans_b || tma_ok(a.B, a.ldb, es));
    if (!in_place) {
      g3_gemm_args c = a;
      const int st = untranspose(d, c, s);
      return st != G3_OK ? st : run_tc(d, c, s, conv, pb);
    }
  }
  if (pb && tc_mode_of(a.dtype, a.k) != TC_3XBF16) return G3_ERR_ARG;   // only the two-part split
  const Layout L = make_layout(a, pl, pb != nullptr);
  const bool claim = claims_tiles(pl, d.sms) && (!a.workspace || a.workspace_bytes >= L.total + kClaimBytes);
  uint8_t* ws = nullptr;
  int st = get_workspace(d, a, L.total + (claim ? kClaimBytes : 0), &ws);
  if (st != G3_OK) return st;
  int* tile_ctr = claim ? reinterpret_cast<int*>(ws + L.total) : nullptr;
  if (claim) G3_CHECK_CUDA(cudaMemsetAsync(tile_ctr, 0, sizeof(int), s));

  const int64_t m = a.m, n = a.n, k = a.k;
  const int es = (a.dtype == G3_FP8_E4M3) ? 1 : ((a.dtype == G3_TF32 || a.dtype == G3_F32_3XTF32) ? 4 : 2);
  const void *A_hi = a.A, *A_lo = nullptr, *B_hi = a.B, *B_lo = nullptr, *A_mid = nullptr, *B_mid = nullptr;
  int64_t lda = a.lda, ldb = a.ldb;

  // a1: operand preparation
  if (fam.mode == TC_6XBF16) {
    uint16_t *ah = (uint16_t*)(ws + L.a_hi), *am = (uint16_t*)(ws + L.a_mid), *al = (uint16_t*)(ws + L.a_lo);
    uint16_t *bh = (uint16_t*)(ws + L.b_hi), *bm = (uint16_t*)(ws + L.b_mid), *bl = (uint16_t*)(ws + L.b_lo);
    G3_CHECK_CUDA(launch_split3_bf16_pair((const float*)a.A, (int)m, (int)k, a.lda, ah, am, al, L.lda_p,
                                          (const float*)a.B, (int)k, (int)n, a.ldb, bh, bm, bl, L.ldb_p, s));
    A_hi = ah; A_mid = am; A_lo = al; B_hi = bh; B_mid = bm; B_lo = bl;
    lda = L.lda_p;
    ldb = L.ldb_p;
  } else if (a.dtype == G3_F32_3XBF16) {
    uint16_t *ah = (uint16_t*)(ws + L.a_hi), *al = (uint16_t*)(ws + L.a_lo);
    uint16_t *bh = (uint16_t*)(ws + L.b_hi), *bl = (uint16_t*)(ws + L.b_lo);
    if (!pb)
      G3_CHECK_CUDA(launch_split_bf16_pair((const float*)a.A, (int)m, (int)k, a.lda, ah, al, L.lda_p,
                                           (const float*)a.B, (int)k, (int)n, a.ldb, bh, bl, L.ldb_p, s));
    else
      G3_CHECK_CUDA(launch_split_bf16((const float*)a.A, (int)m, (int)k, a.lda, ah, al, L.lda_p, s));
    A_hi = ah; A_lo = al;
    lda = L.lda_p;
    if (pb) {
      B_hi = pb->hi; B_lo = pb->lo;
      ldb = pb->ld;
    } else {
      B_hi = bh; B_lo = bl;
      ldb = L.ldb_p;
    }
  } else if (a.dtype == G3_TF32) {
    float *ah = (float*)(ws + L.a_hi), *bh = (float*)(ws + L.b_hi);
    G3_CHECK_CUDA(launch_convert_tf32((const float*)a.A, (int)m, (int)k, a.lda, ah, L.lda_p, s));
    G3_CHECK_CUDA(launch_convert_tf32_t((const float*)a.B, (int)k, (int)n, a.ldb, bh, L.ldb_p, s));
    A_hi = ah; B_hi = bh;
    lda = L.lda_p;
    ldb = L.ldb_p;
  } else if (a.dtype == G3_F32_3XTF32) {
    float *ah = (float*)(ws + L.a_hi), *al = (float*)(ws + L.a_lo);
    float *bh = (float*)(ws + L.b_hi), *bl = (float*)(ws + L.b_lo);
    G3_CHECK_CUDA(launch_split_tf32((const float*)a.A, (int)m, (int)k, a.lda, ah, al, L.lda_p, s));
    G3_CHECK_CUDA(launch_split_tf32_t((const float*)a.B, (int)k, (int)n, a.ldb, bh, bl, L.ldb_p, s));
    A_hi = ah; A_lo = al; B_hi = bh; B_lo = bl;
    lda = L.lda_p;
    ldb = L.ldb_p;
  } else if (a.dtype == G3_INT8 && fam.raw8) {
    if (L.pack_a) {
      G3_CHECK_CUDA(launch_pack_rows(a.A, (int)m, k, a.lda, ws + L.a_hi, L.lda_p, s));
      A_hi = ws + L.a_hi;
    }
    if (L.pack_b) {
      G3_CHECK_CUDA(launch_pack_rows(a.B, (int)k, n, a.ldb, ws + L.b_hi, L.ldb_p, s));
      B_hi = ws + L.b_hi;
    }
    lda = L.lda_p;
    ldb = L.ldb_p;
  } else if (a.dtype == G3_INT8) {
    uint16_t *ah = (uint16_t*)(ws + L.a_hi), *bh = (uint16_t*)(ws + L.b_hi);
    G3_CHECK_CUDA(launch_int8_to_bf16_pair((const int8_t*)a.A, (int)m, (int)k, a.lda, ah, L.lda_p,
                                           (const int8_t*)a.B, (int)k, (int)n, a.ldb, bh, L.ldb_p, s));
    A_hi = ah; B_hi = bh;
    lda = L.lda_p;
    ldb = L.ldb_p;
  } else {
    if (L.pack_a) {
      G3_CHECK_CUDA(launch_pack_rows(a.A, (int)m, k * es, a.lda * es, ws + L.a_hi, L.lda_p * es, s));
      A_hi = ws + L.a_hi;
      lda = L.lda_p;
    }
    if (L.pack_b) {
      G3_CHECK_CUDA(launch_pack_rows(a.B, (int)k, n * es, a.ldb * es, ws + L.b_hi, L.ldb_p * es, s));
      B_hi = ws + L.b_hi;
      ldb = L.ldb_p;
    }
  }

  // TMA descriptors: A as (k inner, m rows) in boxes of BK x bm; B as (n inner,
  // k rows) in boxes of (128 bytes of n) x BK.
  const uint32_t bk = 128 / es, boxn = 128 / es;
  // Maps 2p, 2p+1 are A, B of plane p: plane 0 = hi (or the only plane),
  // plane 1 = lo (two-part split) or mid (three-part split), plane 2 = lo
  // (three-part split).  Unused planes repeat plane 0 (the kernel never loads
  // them).  Map 6 is C's store map.
  CUtensorMap maps[7];
  std::memset(maps, 0, sizeof(maps));
  const uint32_t arows = fam.bm / fam.cg;   // rows of A one CTA stages (half the tile in a pair)
  if (fam.raw8) {
    // raw int8 tiles: A as 64 bytes of k x bm rows, B as 128 columns x 64 k-rows
    if ((st = encode_raw8_2d(&maps[0], A_hi, k, m, lda, 64, fam.bm)) != G3_OK) return st;
  } else if (conv) {
    if ((st = encode_im2col(&maps[0], a.A, es, *conv, arows)) != G3_OK) return st;
  } else if (a.trans_a) {   // A stored k x m: boxes of (128 bytes of m) x bk
    if ((st = encode_2d(&maps[0], A_hi, es, m, k, lda, boxn, bk)) != G3_OK) return st;
  } else if ((st = encode_2d(&maps[0], A_hi, es, k, m, lda, bk, arows)) != G3_OK) {
    return st;
  }
  const bool b_kmajor = a.dtype == G3_TF32 || a.dtype == G3_F32_3XTF32 || a.trans_b;
  if (fam.raw8) {
    if ((st = encode_raw8_2d(&maps[1], B_hi, n, k, ldb, 128, 64)) != G3_OK) return st;
  } else if (b_kmajor) {   // B stored n x k: boxes of bk (k) x 128 (n rows)
    if ((st = encode_2d(&maps[1], B_hi, es, k, n, ldb, bk, 128)) != G3_OK) return st;
  } else if ((st = encode_2d(&maps[1], B_hi, es, n, k, ldb, boxn, bk)) != G3_OK) {
    return st;
  }
  maps[2] = maps[4] = maps[0];
  maps[3] = maps[5] = maps[1];
  if (fam.mode == TC_6XBF16) {
    if ((st = encode_2d(&maps[2], A_mid, es, k, m, lda, bk, arows)) != G3_OK) return st;
    if ((st = encode_2d(&maps[3], B_mid, es, n, k, ldb, boxn, bk)) != G3_OK) return st;
    if ((st = encode_2d(&maps[4], A_lo, es, k, m, lda, bk, arows)) != G3_OK) return st;
    if ((st = encode_2d(&maps[5], B_lo, es, n, k, ldb, boxn, bk)) != G3_OK) return st;
  } else if (a.dtype == G3_F32_3XBF16) {
    if ((st = encode_2d(&maps[2], A_lo, es, k, m, lda, bk, arows)) != G3_OK) return st;
    if ((st = encode_2d(&maps[3], B_lo, es, n, k, ldb, boxn, bk)) != G3_OK) return st;
  } else if (a.dtype == G3_F32_3XTF32) {
    if ((st = encode_2d(&maps[2], A_lo, es, k, m, lda, bk, arows)) != G3_OK) return st;
    if ((st = encode_2d(&maps[3], B_lo, es, k, n, ldb, bk, 128)) != G3_OK) return st;
  }

  TcParams p;
  std::memset(&p, 0, sizeof(p));
  p.m = (int)m;
  p.n = (int)n;
  p.k = (int)k;
  p.tiles_m = pl.tiles_m;
  p.tiles_n = pl.tiles_n;
  p.splits = pl.splits;
  p.kb_per_split = pl.kb_per_split;
  p.num_kb = pl.num_kb;
  p.raster = walk_raster(pl, claim, a.raster);
  p.alpha = (float)a.alpha;
  p.beta = (float)a.beta;
  p.scale_a = (a.dtype == G3_FP8_E4M3) ? a.scale_a : nullptr;
  p.scale_b = (a.dtype == G3_FP8_E4M3) ? a.scale_b : nullptr;
  p.C = a.C;
  p.ldc = a.ldc;
  p.timeout_ns = watchdog_ns();
  p.status = d.status;
  p.debug_withhold = -1;
  p.a_mn = a.trans_a ? 1 : 0;
  p.b_km = a.trans_b ? 1 : 0;
  p.tile_ctr = tile_ctr;
  // INT8: at most 16 k-blocks (1024 products, |sum| <= 2^24) per FP32 accumulator
  p.kchunk = (a.dtype == G3_INT8 && !fam.raw8) ? 16 : 0;
  if (conv) {
    p.conv = 1;
    p.conv_pq = (int)(conv->P * conv->Q);
    p.conv_q = (int)conv->Q;
    p.conv_sh = (int)conv->sh;
    p.conv_sw = (int)conv->sw;
    p.conv_ph = (int)conv->ph;
    p.conv_pw = (int)conv->pw;
    p.conv_dh = (int)conv->dh;
    p.conv_dw = (int)conv->dw;
    p.conv_s = (int)conv->S;
    p.conv_cblocks = (int)(conv->C / 64);
  }
  if (g_withhold_next) {
    p.debug_withhold = 0;
    p.timeout_ns = g_withhold_timeout_ns;
    g_withhold_next = false;
  }
  const bool is_int = a.dtype == G3_INT8;
  p.sk_streams = pl.sk_streams;
  p.sk_dp = pl.sk_dp;
  p.sk_tail = pl.sk_tail;
  p.sk_segs = pl.sk_segs;
  if (pl.sk_streams > 0) p.partial = reinterpret_cast<float*>(ws + L.partial);
  if (pl.splits > 1) {
    p.out_mode = OUT_PARTIAL;
    p.partial = reinterpret_cast<float*>(ws + L.partial);
    p.ldp = round_up(n, 32);
    // partial tiles leave through TMA stores into their split's plane
    if (encode_partial_3d(&maps[6], p.partial, is_int, n, m, pl.splits, p.ldp) == G3_OK) p.c_tma = 1;
  } else {
    p.out_mode = is_int ? OUT_I32 : OUT_F32;
    // C without a read of its old values goes out through TMA stores when its
    // rows are 16-byte aligned (boxes of 32 rows x 128 columns, clipped to C)
    if (a.beta == 0.0 && reinterpret_cast<uintptr_t>(a.C) % 16 == 0 && (a.ldc * 4) % 16 == 0 &&
        encode_c_2d(&maps[6], a.C, is_int, n, m, a.ldc) == G3_OK)
      p.c_tma = 1;
  }

  {
    TimedRegion tr(s);
    G3_CHECK_CUDA(fam.launch(maps, p, d.sms, s));
  }
  if (pl.splits > 1) {
    float alpha = (float)a.alpha;
    if (a.dtype == G3_FP8_E4M3 && (a.scale_a || a.scale_b)) {
      // scales live on the device: fold them in with a one-split reduce pass
      // is not possible on the host, so FP8 never splits (see make_plan callers)
      return G3_ERR_UNSUPPORTED;
    }
    G3_CHECK_CUDA(launch_splitk_reduce(p.partial, pl.splits, (int)m, (int)n, p.ldp, alpha, (float)a.beta, a.C,
                                       a.ldc, is_int, s));
  }
  if (pl.sk_streams > 0) {
    SkFixup fx;
    fx.partial = p.partial;
    fx.streams = pl.sk_streams;
    fx.segs = pl.sk_segs;
    fx.dp = pl.sk_dp;
    fx.tail = pl.sk_tail;
    fx.num_kb = pl.num_kb;
    fx.tiles_m = pl.tiles_m;
    fx.tiles_n = pl.tiles_n;
    fx.raster = pl.raster;
    fx.bm = fam.bm;
    fx.bn = 128 * fam.cg;
    fx.m = (int)m;
    fx.n = (int)n;
    fx.alpha = (float)a.alpha;
    fx.beta = (float)a.beta;
    fx.scale_a = p.scale_a;
    fx.scale_b = p.scale_b;
    fx.C = a.C;
    fx.ldc = a.ldc;
    fx.is_int = is_int;
    G3_CHECK_CUDA(launch_streamk_fixup(fx, s));
  }
  return G3_OK;
}

int input_esize(int dtype) {
  if (dtype == G3_F64) return 8;
  if (dtype == G3_INT16) return 2;
  if (dtype == G3_F32 || dtype == G3_F32_3XBF16 || dtype == G3_TF32 || dtype == G3_F32_3XTF32) return 4;
  return (dtype == G3_BF16 || dtype == G3_FP16) ? 2 : 1;
}

// Transposed operands: copy them into row-major A (m x k) / B (k x n) in the
// device's transpose buffer and point the arguments there.
int untranspose(DevState& d, g3_gemm_args& a, cudaStream_t s) {
  const int es = input_esize(a.dtype);
  const int64_t lda_t = round_up(std::max<int64_t>(a.k, 1), 16), ldb_t = round_up(a.n, 16);
  const size_t a_bytes = a.trans_a ? align256((size_t)a.m * lda_t * es) : 0;
  const size_t b_bytes = a.trans_b ? align256((size_t)a.k * ldb_t * es) : 0;
  if (d.tbuf_bytes < a_bytes + b_bytes) {
    if (d.tbuf) {
      cudaDeviceSynchronize();
      cudaFree(d.tbuf);
      d.tbuf = nullptr;
      d.tbuf_bytes = 0;
    }
    if (device_alloc(&d.tbuf, a_bytes + b_bytes) != cudaSuccess) {
      cudaGetLastError();
      return G3_ERR_NOMEM;
    }
    d.tbuf_bytes = a_bytes + b_bytes;
  }
  uint8_t* base = static_cast<uint8_t*>(d.tbuf);
  if (a.trans_a) {   // stored k x m
    G3_CHECK_CUDA(launch_transpose(a.A, (int)a.k, (int)a.m, a.lda, base, lda_t, es, s));
    a.A = base;
    a.lda = lda_t;
    a.trans_a = 0;
  }
  if (a.trans_b) {   // stored n x k
    G3_CHECK_CUDA(launch_transpose(a.B, (int)a.n, (int)a.k, a.ldb, base + a_bytes, ldb_t, es, s));
    a.B = base + a_bytes;
    a.ldb = ldb_t;
    a.trans_b = 0;
  }
  return G3_OK;
}

int gemm_impl(g3_gemm_args a, cudaStream_t s, const PreparedB* pb = nullptr) {
  int st = validate(a);
  if (st != G3_OK) return st;
  if (a.m == 0 || a.n == 0) return G3_OK;
  std::lock_guard<std::mutex> lock(g_mu);
  DevState* d = nullptr;
  if ((st = ensure_device(&d)) != G3_OK) return st;
  // the 8- and 16-bit tensor-core modes take transposed operands in run_tc
  if ((a.trans_a || a.trans_b) && a.k > 0 && a.alpha != 0.0 && !reads_transposed(a.dtype) &&
      (st = untranspose(*d, a, s)) != G3_OK)
    return st;
  const bool is_int = a.dtype == G3_INT8;
  if (a.k == 0 || a.alpha == 0.0) {
    if ((is_int || a.dtype == G3_F64 || a.dtype == G3_INT16) && a.beta == 1.0) return G3_OK;
    if (a.dtype == G3_INT16)   // beta == 0: zeros
      G3_CHECK_CUDA(cudaMemset2DAsync(a.C, a.ldc * 8, 0, a.n * 8, a.m, s));
    else if (a.dtype == G3_F64)
      G3_CHECK_CUDA(launch_scale_c_f64(static_cast<double*>(a.C), (int)a.m, (int)a.n, a.ldc, a.beta, s));
    else
      G3_CHECK_CUDA(launch_scale_c(a.C, is_int, (int)a.m, (int)a.n, a.ldc, (float)a.beta, s));
    return G3_OK;
  }
  // device scales apply in the kernel epilogue or the stream-K fix-up, which
  // the split-K reduce cannot: no split-K then
  if (a.dtype == G3_FP8_E4M3 && (a.scale_a || a.scale_b) && a.split_k > 1) a.split_k = 1;
  if (a.dtype == G3_F32) return run_simt(a, d->sms, s);
  if (a.dtype == G3_F64) return run_simt64(a, s);
  if (a.dtype == G3_INT16) return run_simt_i16(a, s);
  return run_tc(*d, a, s, nullptr, pb);
}

}  // namespace

// Services of this file for the other translation units (see internal.h).
std::mutex& api_mutex() { return g_mu; }

int current_device_info(DeviceInfo* out) {
  DevState* d = nullptr;
  const int st = ensure_device(&d);
  if (st != G3_OK) return st;
  int dev = -1;
  cudaGetDevice(&dev);
  out->device = dev;
  out->sms = d->sms;
  out->status = d->status;
  return G3_OK;
}

int encode_tensor_2d(CUtensorMap* map, const void* base, int esize, uint64_t inner, uint64_t outer, uint64_t ld,
                     uint32_t box_inner, uint32_t box_outer) {
  return encode_2d(map, base, esize, inner, outer, ld, box_inner, box_outer);
}

unsigned long long watchdog_timeout_ns() { return watchdog_ns(); }

bool kernel_timing_enabled() { return g_timing; }

void kernel_timing_push(cudaEvent_t e0, cudaEvent_t e1) { g_events.emplace_back(e0, e1); }

int tuned_grouped_bm(int64_t m, int64_t n, int64_t k, int dtype) {
  tune_env_once();
  auto it = g_tune.find(tune_key(m, n, k, dtype + kGroupedTuneTag));
  return it == g_tune.end() ? 0 : it->second.member;
}

void store_grouped_tuning(int64_t m, int64_t n, int64_t k, int dtype, int bm, double ms) {
  g_tune[tune_key(m, n, k, dtype + kGroupedTuneTag)] = TuneVal{bm, 1, ms};
}

bool take_withhold(unsigned long long* timeout_ns) {
  if (!g_withhold_next) return false;
  g_withhold_next = false;
  *timeout_ns = g_withhold_timeout_ns;
  return true;
}

}  // namespace g3

using namespace g3;

// C := beta*C + alpha*A*B with A, B, C in host memory, as a pipeline on three
// streams: copies up on `up`, compute on the caller's stream, copies down on
// `down`, ordered by events.  C is cut into row blocks (about 2048 rows, four
// to eight of them); each finished block goes down while later blocks compute.
// Every row block needs all of B, so in the plain order nothing computes until
// B has arrived.  For the FP32-accurate mode with the two-part split (k > 512)
// B goes up instead in k-slabs, after row block 0 of A (and of C): each slab
// is split into bf16 planes once -- kept for every row block of the call --
// and row block 0 accumulates slab by slab (beta for the first slab, then 1),
// so the tensor cores start after the first slab; the later blocks use the
// prepared planes.  (Row block 0 is rounded to FP32 once per slab: at most
// kHostMaxSlabs - 1 extra roundings of 2^-24 relative to its partial sums.)
// Device copies (and the block GEMMs' scratch) live in a library buffer of
// the caller's stream, so calls on different streams overlap -- one call's
// uploads run under another's compute; the caller's stream waits for the last
// download.
static int gemm_host_impl(const g3_gemm_args& a, cudaStream_t s) {
  int st = validate(a);
  if (st != G3_OK) return st;
  if (a.m == 0 || a.n == 0) return G3_OK;
  const int64_t m = a.m, n = a.n, k = a.k;
  const int es = input_esize(a.dtype);
  const int64_t lda_d = round_up(std::max<int64_t>(k, 1), 16), ldb_d = round_up(n, 16), ldc_d = round_up(n, 16);
  const size_t a_bytes = align256((size_t)m * lda_d * es), b_bytes = align256((size_t)std::max<int64_t>(k, 1) * ldb_d * es);
  const int ces = (a.dtype == G3_F64 || a.dtype == G3_INT16) ? 8 : 4;   // bytes per element of C
  const size_t c_bytes = align256((size_t)m * ldc_d * ces);
  const bool products = k > 0 && a.alpha != 0.0;
  const bool read_c = a.beta != 0.0;
  const int nb = (m >= 2048 && products) ? (int)std::max<int64_t>(4, std::min<int64_t>(kHostMaxBlocks, (m + 2047) / 2048))
                                         : 1;
  const int64_t rb = round_up((m + nb - 1) / nb, 256);
  // B in k-slabs (prepared planes): slabs of at least 2048, each above the
  // three-part split's bound so that every call takes the two-part split
  const bool prep = nb > 1 && a.dtype == G3_F32_3XBF16 && tc_mode_of(a.dtype, k) == TC_3XBF16;
  int ns = 1;
  int64_t ks = k;
  if (prep) {
    ns = (int)std::max<int64_t>(1, std::min<int64_t>(kHostMaxSlabs, k / 2048));
    for (;;) {
      ks = round_up((k + ns - 1) / ns, 64);
      ns = (int)((k + ks - 1) / ks);
      if (ns == 1 || k - (ns - 1) * ks > kSixProductMaxK) break;
      --ns;
    }
  }
  const int64_t ldp = round_up(n, 8);   // leading dimension of the prepared planes
  const size_t plane_bytes = prep ? align256((size_t)k * ldp * 2) : 0;
  uint8_t* base = nullptr;
  uint8_t *dA = nullptr, *dB = nullptr, *dC = nullptr, *dW = nullptr;
  uint16_t *Bhi = nullptr, *Blo = nullptr;
  size_t ws_bytes = 0;
  auto place = [&](uint8_t* b) {
    base = b;
    dA = base;
    dB = base + a_bytes;
    dC = base + a_bytes + b_bytes;
    Bhi = reinterpret_cast<uint16_t*>(dC + c_bytes);
    Blo = reinterpret_cast<uint16_t*>(dC + c_bytes + plane_bytes);
    dW = dC + c_bytes + 2 * plane_bytes;
  };
  auto rows_of = [&](int b, int64_t* r0, int64_t* r1) {
    *r0 = b * rb;
    *r1 = std::min(m, *r0 + rb);
    return *r0 < *r1;
  };
  auto block_args = [&](int64_t r0, int64_t r1) {
    g3_gemm_args blk = a;
    blk.m = r1 - r0;
    blk.A = dA + (size_t)r0 * lda_d * es;
    blk.lda = lda_d;
    blk.B = dB;
    blk.ldb = ldb_d;
    blk.C = dC + (size_t)r0 * ldc_d * ces;
    blk.ldc = ldc_d;
    blk.workspace = ws_bytes ? dW : nullptr;
    blk.workspace_bytes = ws_bytes;
    return blk;
  };
  auto slab_args = [&](int64_t r0, int64_t r1, int j) {   // row block r0..r1 on k-slab j
    const int64_t k0 = j * ks, k1 = std::min(k, (j + 1) * ks);
    g3_gemm_args blk = block_args(r0, r1);
    blk.k = k1 - k0;
    blk.A = dA + (size_t)r0 * lda_d * es + (size_t)k0 * es;
    blk.B = dB + (size_t)k0 * ldb_d * es;
    if (j > 0) blk.beta = 1.0;
    return blk;
  };
  cudaEvent_t* ev = nullptr;
  cudaStream_t up = nullptr, down = nullptr;
  HostPipe* P = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    DevState* d = nullptr;
    if ((st = ensure_device(&d)) != G3_OK) return st;
    // the caller stream's buffers, else a free set, else the least recently used
    for (auto& q : d->pipes)
      if (q.used && q.owner == s) P = &q;
    if (!P)
      for (auto& q : d->pipes)
        if (!q.used && !P) P = &q;
    if (!P) {
      P = &d->pipes[0];
      for (auto& q : d->pipes)
        if (q.last_use < P->last_use) P = &q;
    }
    P->used = true;
    P->owner = s;
    P->last_use = ++d->pipe_tick;
    if (!P->up) {
      if (cudaStreamCreateWithFlags(&P->up, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamCreateWithFlags(&P->down, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&P->free_ev, cudaEventDisableTiming) != cudaSuccess)
        return G3_ERR_CUDA;
      for (auto& e : P->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return G3_ERR_CUDA;
    }
    // scratch of the block GEMMs (operand planes, split-K partials): the
    // largest any block needs, laid out on a 256-byte aligned stand-in base
    place(reinterpret_cast<uint8_t*>(uintptr_t(256)));
    if (products && d->sms > 0 && a.dtype != G3_F32 && a.dtype != G3_F64 && a.dtype != G3_INT16) {
      auto need_of = [&](const g3_gemm_args& blk, bool prepared) {
        const Plan pl = make_plan(blk.m, blk.n, blk.k, blk.dtype, d->sms, blk.config, blk.split_k, blk.raster, true);
        return pl.member < 0 ? size_t(0)
                             : make_layout(blk, pl, prepared).total + (claims_tiles(pl, d->sms) ? kClaimBytes : 0);
      };
      for (int b = 0; b < nb; ++b) {
        int64_t r0, r1;
        if (!rows_of(b, &r0, &r1)) break;
        if (prep && b == 0)
          for (int j = 0; j < ns; ++j) ws_bytes = std::max(ws_bytes, need_of(slab_args(r0, r1, j), true));
        else
          ws_bytes = std::max(ws_bytes, need_of(block_args(r0, r1), prep));
      }
      ws_bytes = align256(ws_bytes);
    }
    const size_t need = a_bytes + b_bytes + c_bytes + 2 * plane_bytes + ws_bytes;
    if (P->bytes < need) {
      if (P->buf) {
        cudaDeviceSynchronize();
        cudaFree(P->buf);
        P->buf = nullptr;
        P->bytes = 0;
      }
      if (device_alloc(&P->buf, need) != cudaSuccess) {
        cudaGetLastError();
        return G3_ERR_NOMEM;
      }
      P->bytes = need;
    }
    place(static_cast<uint8_t*>(P->buf));
    ev = P->ev;
    up = P->up;
    down = P->down;
  }
  // events: 0 start, 1 + b row block b up, 1 + kHostMaxBlocks + b row block b
  // done, 2 kHostMaxBlocks + 1 last download, 2 kHostMaxBlocks + 2 + j slab j up
  cudaEvent_t* ev_up = ev + 1;
  cudaEvent_t* ev_done = ev + 1 + kHostMaxBlocks;
  cudaEvent_t ev_last = ev[2 * kHostMaxBlocks + 1];
  cudaEvent_t* ev_slab = ev + 2 * kHostMaxBlocks + 2;
  // the uploads follow the caller's earlier work on its stream and the last
  // call that used these buffers (on this stream or the one they came from)
  G3_CHECK_CUDA(cudaEventRecord(ev[0], s));
  G3_CHECK_CUDA(cudaStreamWaitEvent(up, ev[0], 0));
  if (P->free_recorded) G3_CHECK_CUDA(cudaStreamWaitEvent(up, P->free_ev, 0));
  auto up_rows = [&](int b) -> int {   // A (and C) rows of block b
    int64_t r0, r1;
    if (!rows_of(b, &r0, &r1)) return G3_OK;
    if (products)
      G3_CHECK_CUDA(cudaMemcpy2DAsync(dA + (size_t)r0 * lda_d * es, lda_d * es,
                                      static_cast<const uint8_t*>(a.A) + (size_t)r0 * a.lda * es, a.lda * es, k * es,
                                      r1 - r0, cudaMemcpyHostToDevice, up));
    if (read_c)
      G3_CHECK_CUDA(cudaMemcpy2DAsync(dC + (size_t)r0 * ldc_d * ces, ldc_d * ces,
                                      static_cast<const uint8_t*>(a.C) + (size_t)r0 * a.ldc * ces, a.ldc * ces,
                                      n * ces, r1 - r0, cudaMemcpyHostToDevice, up));
    return G3_OK;
  };
  auto up_B = [&](int64_t k0, int64_t k1) -> int {   // rows k0 .. k1-1 of B
    G3_CHECK_CUDA(cudaMemcpy2DAsync(dB + (size_t)k0 * ldb_d * es, ldb_d * es,
                                    static_cast<const uint8_t*>(a.B) + (size_t)k0 * a.ldb * es, a.ldb * es, n * es,
                                    k1 - k0, cudaMemcpyHostToDevice, up));
    return G3_OK;
  };
  auto down_rows = [&](int b, int64_t r0, int64_t r1) -> int {
    G3_CHECK_CUDA(cudaEventRecord(ev_done[b], s));
    G3_CHECK_CUDA(cudaStreamWaitEvent(down, ev_done[b], 0));
    G3_CHECK_CUDA(cudaMemcpy2DAsync(static_cast<uint8_t*>(a.C) + (size_t)r0 * a.ldc * ces, a.ldc * ces,
                                    dC + (size_t)r0 * ldc_d * ces, ldc_d * ces, n * ces, r1 - r0,
                                    cudaMemcpyDeviceToHost, down));
    return G3_OK;
  };
  if (prep) {
    // up: row block 0, the slabs of B, then the other row blocks
    if ((st = up_rows(0)) != G3_OK) return st;
    for (int j = 0; j < ns; ++j) {
      if ((st = up_B(j * ks, std::min(k, (j + 1) * ks))) != G3_OK) return st;
      G3_CHECK_CUDA(cudaEventRecord(ev_slab[j], up));
    }
    for (int b = 1; b < nb; ++b) {
      if ((st = up_rows(b)) != G3_OK) return st;
      G3_CHECK_CUDA(cudaEventRecord(ev_up[b], up));
    }
    // compute: row block 0 slab by slab, splitting each slab of B once
    int64_t r0, r1;
    rows_of(0, &r0, &r1);
    for (int j = 0; j < ns; ++j) {
      const int64_t k0 = j * ks, k1 = std::min(k, (j + 1) * ks);
      G3_CHECK_CUDA(cudaStreamWaitEvent(s, ev_slab[j], 0));
      G3_CHECK_CUDA(launch_split_bf16(reinterpret_cast<const float*>(dB + (size_t)k0 * ldb_d * es), (int)(k1 - k0),
                                      (int)n, ldb_d, Bhi + k0 * ldp, Blo + k0 * ldp, ldp, s));
      const PreparedB pb{Bhi + k0 * ldp, Blo + k0 * ldp, ldp};
      if ((st = gemm_impl(slab_args(r0, r1, j), s, &pb)) != G3_OK) return st;
    }
    if ((st = down_rows(0, r0, r1)) != G3_OK) return st;
    const PreparedB pb{Bhi, Blo, ldp};
    for (int b = 1; b < nb; ++b) {
      if (!rows_of(b, &r0, &r1)) break;
      G3_CHECK_CUDA(cudaStreamWaitEvent(s, ev_up[b], 0));
      if ((st = gemm_impl(block_args(r0, r1), s, &pb)) != G3_OK) return st;
      if ((st = down_rows(b, r0, r1)) != G3_OK) return st;
    }
  } else {
    // B up first (every row block of C needs all of it), then the row blocks
    if (products && (st = up_B(0, k)) != G3_OK) return st;
    for (int b = 0; b < nb; ++b) {
      int64_t r0, r1;
      if (!rows_of(b, &r0, &r1)) break;
      if ((st = up_rows(b)) != G3_OK) return st;
      G3_CHECK_CUDA(cudaEventRecord(ev_up[b], up));
      G3_CHECK_CUDA(cudaStreamWaitEvent(s, ev_up[b], 0));
      if ((st = gemm_impl(block_args(r0, r1), s)) != G3_OK) return st;
      if ((st = down_rows(b, r0, r1)) != G3_OK) return st;
    }
  }
  G3_CHECK_CUDA(cudaEventRecord(ev_last, down));
  G3_CHECK_CUDA(cudaStreamWaitEvent(s, ev_last, 0));
  {
    std::lock_guard<std::mutex> lock(g_mu);
    G3_CHECK_CUDA(cudaEventRecord(P->free_ev, s));
    P->free_recorded = true;
  }
  return G3_OK;
}

// Implicit-GEMM convolution: the GEMM of m = N*P*Q output pixels, n = K
// output channels and k = R*S*C taps x channels, with A read from the NHWC
// activations through an im2col tensor map instead of a materialised matrix.
static int conv2d_impl(const ConvDesc& c, double alpha, const void* x, const void* w, double beta, float* y,
                       int dtype, cudaStream_t s) {
  if (c.N < 1 || c.H < 1 || c.W < 1) return -101;
  if (c.C < 64 || c.C % 64 != 0) return G3_ERR_UNSUPPORTED;   // 64 channels = one 128-byte k-block row
  if (c.K < 1) return -105;
  if (c.R < 1 || c.S < 1 || c.sh < 1 || c.sw < 1 || c.sh > 8 || c.sw > 8 || c.dh < 1 || c.dw < 1)
    return G3_ERR_UNSUPPORTED;
  if (c.ph < 0 || c.pw < 0 || c.ph > 128 || c.pw > 128) return G3_ERR_UNSUPPORTED;
  if ((c.R - 1) * c.dh - c.ph > 128 || (c.S - 1) * c.dw - c.pw > 128 || c.P < 1 || c.Q < 1) return G3_ERR_UNSUPPORTED;
  if ((c.R - 1) * c.dh > 65535 || (c.S - 1) * c.dw > 65535) return G3_ERR_UNSUPPORTED;
  if (dtype != G3_BF16 && dtype != G3_FP16) return G3_ERR_UNSUPPORTED;
  if (!x || !w || !y) return G3_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(x) % 16 != 0) return G3_ERR_UNSUPPORTED;
  if (c.N * c.P * c.Q > INT32_MAX || c.R * c.S * c.C > INT32_MAX) return G3_ERR_UNSUPPORTED;
  g3_gemm_args a;
  g3_gemm_args_init(&a);
  a.m = c.N * c.P * c.Q;
  a.n = c.K;
  a.k = c.R * c.S * c.C;
  a.alpha = alpha;
  a.beta = beta;
  a.A = x;
  a.lda = a.k;   // not used to address A (the im2col map does); keeps the layout logic from re-packing it
  a.B = w;
  a.ldb = c.K;
  a.C = y;
  a.ldc = c.K;
  a.dtype = dtype;
  std::lock_guard<std::mutex> lock(g_mu);
  DevState* d = nullptr;
  int st = ensure_device(&d);
  if (st != G3_OK) return st;
  if (alpha == 0.0) {
    G3_CHECK_CUDA(launch_scale_c(y, false, (int)a.m, (int)a.n, a.ldc, (float)beta, s));
    return G3_OK;
  }
  return run_tc(*d, a, s, &c);
}

extern "C" {

void g3_gemm_args_init(g3_gemm_args* a) {
  if (!a) return;
  std::memset(a, 0, sizeof(*a));
  a->config = -1;
}

int g3_gemm(int64_t m, int64_t n, int64_t k, double alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
            double beta, void* C, int64_t ldc, int dtype) {
  g3_gemm_args a;
  g3_gemm_args_init(&a);
  a.m = m; a.n = n; a.k = k;
  a.alpha = alpha; a.beta = beta;
  a.A = A; a.lda = lda; a.B = B; a.ldb = ldb; a.C = C; a.ldc = ldc;
  a.dtype = dtype;
  return gemm_impl(a, g_stream);
}

int g3_set_stream(void* stream) {
  g_stream = static_cast<cudaStream_t>(stream);
  return G3_OK;
}

int g3_conv2d(int64_t N, int64_t H, int64_t W, int64_t C, int64_t K, int64_t R, int64_t S, int64_t stride_h,
              int64_t stride_w, int64_t pad_h, int64_t pad_w, int64_t dil_h, int64_t dil_w, double alpha,
              const void* x, const void* w, double beta, float* y, int dtype, void* stream) {
  ConvDesc c{N, H, W, C, K, R, S, stride_h, stride_w, pad_h, pad_w, dil_h, dil_w, 0, 0};
  if (c.sh >= 1 && c.sw >= 1) {
    c.P = (H + 2 * pad_h - dil_h * (R - 1) - 1) / stride_h + 1;
    c.Q = (W + 2 * pad_w - dil_w * (S - 1) - 1) / stride_w + 1;
  }
  return conv2d_impl(c, alpha, x, w, beta, y, dtype, stream ? static_cast<cudaStream_t>(stream) : g_stream);
}

int g3_gemm_host(int64_t m, int64_t n, int64_t k, double alpha, const void* A, int64_t lda, const void* B,
                 int64_t ldb, double beta, void* C, int64_t ldc, int dtype, void* stream) {
  g3_gemm_args a;
  g3_gemm_args_init(&a);
  a.m = m; a.n = n; a.k = k;
  a.alpha = alpha; a.beta = beta;
  a.A = A; a.lda = lda; a.B = B; a.ldb = ldb; a.C = C; a.ldc = ldc;
  a.dtype = dtype;
  return gemm_host_impl(a, stream ? static_cast<cudaStream_t>(stream) : g_stream);
}

int g3_gemm_ex(const g3_gemm_args* args, void* stream) {
  if (!args) return G3_ERR_ARG;
  return gemm_impl(*args, stream ? static_cast<cudaStream_t>(stream) : g_stream);
}

int g3_gemm_workspace_size(const g3_gemm_args* args, size_t* bytes) {
  if (!args || !bytes) return G3_ERR_ARG;
  *bytes = 0;
  int st = validate(*args);
  if (st != G3_OK) return st;
  if (args->m == 0 || args->n == 0 || args->k == 0 || args->alpha == 0.0 || args->dtype == G3_F32 ||
      args->dtype == G3_F64 || args->dtype == G3_INT16)
    return G3_OK;
  std::lock_guard<std::mutex> lock(g_mu);
  DevState* d = nullptr;
  if ((st = ensure_device(&d)) != G3_OK) return st;
  g3_gemm_args a = *args;
  const bool dev_scales = a.dtype == G3_FP8_E4M3 && (a.scale_a || a.scale_b);
  if (dev_scales && a.split_k > 1) a.split_k = 1;
  // a transposed operand is read in place (when TMA can address it) or
  // reaches the kernel as an aligned row-major copy in the transpose buffer:
  // no workspace either way
  if (a.trans_a) { a.A = d->ws ? d->ws : reinterpret_cast<void*>(uintptr_t(256)); a.lda = round_up(a.k, 16); }
  if (a.trans_b) { a.B = d->ws ? d->ws : reinterpret_cast<void*>(uintptr_t(256)); a.ldb = round_up(a.n, 16); }
  const Plan pl = make_plan(a.m, a.n, a.k, a.dtype, d->sms, a.config, a.split_k, a.raster, !dev_scales);
  *bytes = make_layout(a, pl).total;
  if (claims_tiles(pl, d->sms)) *bytes += kClaimBytes;
  return G3_OK;
}

// Arguments x, rows, cols, ldx, y are positions 1-5; ldy_pos is ldy's position.
static int prep_check(const void* x, int64_t rows, int64_t cols, int64_t ldx, const void* y, int64_t ldy,
                      int ldy_pos = 6) {
  if (rows < 0) return -102;
  if (cols < 0) return -103;
  if (ldx < std::max<int64_t>(1, cols)) return -104;
  if (rows > INT32_MAX || cols > INT32_MAX) return G3_ERR_UNSUPPORTED;
  if (rows > 0 && cols > 0 && (!x || !y)) return x ? -105 : -101;
  if (ldy < std::max<int64_t>(1, cols)) return -(100 + ldy_pos);
  return G3_OK;
}

int g3_convert_bf16(const float* x, int64_t rows, int64_t cols, int64_t ldx, void* y, int64_t ldy, void* stream) {
  int st = prep_check(x, rows, cols, ldx, y, ldy);
  if (st != G3_OK || rows == 0 || cols == 0) return st;
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_stream;
  G3_CHECK_CUDA(launch_convert_bf16(x, (int)rows, (int)cols, ldx, static_cast<uint16_t*>(y), ldy, s));
  return G3_OK;
}

int g3_split_bf16(const float* x, int64_t rows, int64_t cols, int64_t ldx, void* hi, void* lo, int64_t ldy,
                  void* stream) {
  int st = prep_check(x, rows, cols, ldx, hi, ldy, 7);
  if (st != G3_OK) return st;
  if (rows > 0 && cols > 0 && !lo) return -106;
  if (rows == 0 || cols == 0) return G3_OK;
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_stream;
  G3_CHECK_CUDA(launch_split_bf16(x, (int)rows, (int)cols, ldx, static_cast<uint16_t*>(hi),
                                  static_cast<uint16_t*>(lo), ldy, s));
  return G3_OK;
}

int g3_convert_tf32(const float* x, int64_t rows, int64_t cols, int64_t ldx, float* y, int64_t ldy, void* stream) {
  int st = prep_check(x, rows, cols, ldx, y, ldy);
  if (st != G3_OK || rows == 0 || cols == 0) return st;
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_stream;
  G3_CHECK_CUDA(launch_convert_tf32(x, (int)rows, (int)cols, ldx, y, ldy, s));
  return G3_OK;
}

int g3_split_tf32(const float* x, int64_t rows, int64_t cols, int64_t ldx, float* hi, float* lo, int64_t ldy,
                  void* stream) {
  int st = prep_check(x, rows, cols, ldx, hi, ldy, 7);
  if (st != G3_OK) return st;
  if (rows > 0 && cols > 0 && !lo) return -106;
  if (rows == 0 || cols == 0) return G3_OK;
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_stream;
  G3_CHECK_CUDA(launch_split_tf32(x, (int)rows, (int)cols, ldx, hi, lo, ldy, s));
  return G3_OK;
}

int g3_split3_bf16(const float* x, int64_t rows, int64_t cols, int64_t ldx, void* hi, void* mid, void* lo,
                   int64_t ldy, void* stream) {
  int st = prep_check(x, rows, cols, ldx, hi, ldy, 8);
  if (st != G3_OK) return st;
  if (rows > 0 && cols > 0 && !mid) return -106;
  if (rows > 0 && cols > 0 && !lo) return -107;
  if (rows == 0 || cols == 0) return G3_OK;
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_stream;
  G3_CHECK_CUDA(launch_split3_bf16(x, (int)rows, (int)cols, ldx, static_cast<uint16_t*>(hi),
                                   static_cast<uint16_t*>(mid), static_cast<uint16_t*>(lo), ldy, s));
  return G3_OK;
}

int g3_quantize_fp8(const float* x, int64_t rows, int64_t cols, int64_t ldx, uint8_t* q, int64_t ldq, float* scale,
                    void* stream) {
  int st = prep_check(x, rows, cols, ldx, q, ldq);
  if (st != G3_OK) return st;
  if (!scale) return -107;
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_stream;
  std::lock_guard<std::mutex> lock(g_mu);
  DevState* d = nullptr;
  if ((st = ensure_device(&d)) != G3_OK) return st;
  g3_gemm_args dummy;
  g3_gemm_args_init(&dummy);
  uint8_t* ws = nullptr;
  if ((st = get_workspace(*d, dummy, 256, &ws)) != G3_OK) return st;
  G3_CHECK_CUDA(launch_quantize_e4m3(x, (int)rows, (int)cols, ldx, reinterpret_cast<unsigned int*>(ws), q, ldq,
                                     scale, s));
  return G3_OK;
}

int g3_get_last_device_status(int* code) {
  std::lock_guard<std::mutex> lock(g_mu);
  DevState* d = nullptr;
  int st = ensure_device(&d);
  if (st != G3_OK) return st;
  G3_CHECK_CUDA(cudaDeviceSynchronize());
  int v = 0;
  G3_CHECK_CUDA(cudaMemcpy(&v, d->status, sizeof(int), cudaMemcpyDeviceToHost));
  const int zero = 0;
  G3_CHECK_CUDA(cudaMemcpy(d->status, &zero, sizeof(int), cudaMemcpyHostToDevice));
  if (code) *code = v;
  return v ? G3_ERR_TIMEOUT : G3_OK;
}

const char* g3_status_string(int s) {
  switch (s) {
    case G3_OK: return "ok";
    case G3_ERR_ARG: return "invalid argument";
    case G3_ERR_UNSUPPORTED: return "unsupported";
    case G3_ERR_CUDA: return "CUDA error";
    case G3_ERR_NOMEM: return "out of device memory";
    case G3_ERR_TIMEOUT: return "device wait timed out";
    case G3_ERR_NOT_INIT: return "no usable CUDA device";
    default: return s <= -100 ? "invalid argument (positional)" : "unknown status";
  }
}

int g3_family_size(void) { return G3_FAMILY_SIZE; }

int g3_family_describe(int index, char* buf, size_t len) {
  if (index < 0 || index >= G3_FAMILY_SIZE) return -101;
  if (!buf || len == 0) return -102;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    family_init();
  }
  const FamilyEntry& f = g_family[index];
  static const char* names[] = {"bf16", "3xbf16", "fp8", "int8emu", "6xbf16", "f16", "tf32", "3xtf32"};
  std::snprintf(buf, len, "mode=%s bm=%d bn=%d stages=%d smem=%d bufs=%d cg=%d", names[f.mode], f.bm, 128 * f.cg,
                f.stages, f.smem, f.bufs, f.cg);
  return G3_OK;
}

int g3_plan_query(int64_t m, int64_t n, int64_t k, int dtype, int* config, int* split_k, int* raster) {
  if (m < 0) return -101;
  if (n < 0) return -102;
  if (k < 0) return -103;
  if (dtype < G3_F32 || dtype > G3_INT16) return -104;
  std::lock_guard<std::mutex> lock(g_mu);
  DevState* d = nullptr;
  int sms = 152;
  if (ensure_device(&d) == G3_OK) sms = d->sms;
  if (dtype == G3_F32 || dtype == G3_F64 || dtype == G3_INT16) {
    if (config) *config = -1;
    if (split_k) *split_k = dtype == G3_F32 ? simt_plan(m, n, k, sms, 0).splits : 1;
    if (raster) *raster = 0;
    return G3_OK;
  }
  family_init();
  // (FP8 calls are assumed to carry device scales: no split-K)
  const Plan pl = make_plan(m, n, std::max<int64_t>(k, 1), dtype, sms, -1, 0, 0, dtype != G3_FP8_E4M3);
  if (config) *config = pl.member;
  if (split_k) *split_k = pl.sk_streams > 0 ? G3_SPLIT_STREAM_K : pl.splits;
  if (raster) *raster = walk_raster(pl, claims_tiles(pl, sms), 0);
  return G3_OK;
}

uint64_t g3_launch_count(void) { return g3::launch_count(); }

int g3_stream_traffic(const void* in, int64_t in_bytes, void* out, int64_t out_bytes, void* stream) {
  // at most 32 GiB per stream, so that the interleave products fit 64 bits
  if (in_bytes < 0 || in_bytes % 16 || in_bytes > (int64_t(1) << 35)) return -102;
  if (out_bytes < 0 || out_bytes % 16 || out_bytes > (int64_t(1) << 35)) return -104;
  if (in_bytes > 0 && (!in || reinterpret_cast<uintptr_t>(in) % 16)) return -101;
  if (out_bytes > 0 && (!out || reinterpret_cast<uintptr_t>(out) % 16)) return -103;
  int sms = 152;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    DevState* d = nullptr;
    const int st = ensure_device(&d);
    if (st != G3_OK) return st;
    sms = d->sms;
  }
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_stream;
  if (launch_stream_traffic(in, in_bytes / 16, out, out_bytes / 16, sms, s) != cudaSuccess) {
    cudaGetLastError();
    return G3_ERR_CUDA;
  }
  return G3_OK;
}

int64_t g3_debug_device_allocations(void) { return g3::g_device_allocs.load(std::memory_order_relaxed); }

int g3_debug_withhold_next(int64_t timeout_ms) {
  if (timeout_ms <= 0 || timeout_ms > 10000) return -101;
  std::lock_guard<std::mutex> lock(g_mu);
  g_withhold_next = true;
  g_withhold_timeout_ns = (unsigned long long)timeout_ms * 1000000ULL;
  return G3_OK;
}

int g3_kernel_timing(int enable) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_timing = enable != 0;
  return G3_OK;
}

int g3_kernel_time_ms(double* total_ms, int* launches, int reset) {
  std::lock_guard<std::mutex> lock(g_mu);
  double sum = 0.0;
  for (auto& ev : g_events) {
    cudaEventSynchronize(ev.second);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev.first, ev.second) == cudaSuccess) sum += ms;
    else cudaGetLastError();
  }
  if (total_ms) *total_ms = sum;
  if (launches) *launches = (int)g_events.size();
  if (reset) {
    for (auto& ev : g_events) {
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
    g_events.clear();
  }
  return G3_OK;
}

int g3_autotune(int64_t m, int64_t n, int64_t k, int dtype, int* best_config, int* best_split, double* best_ms) {
  if (m <= 0) return -101;
  if (n <= 0) return -102;
  if (k <= 0) return -103;
  if (dtype < G3_F32 || dtype > G3_INT16) return -104;
  if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX || (dtype == G3_INT8 && k > 131072)) return G3_ERR_UNSUPPORTED;
  if (dtype == G3_F32 || dtype == G3_F64 || dtype == G3_INT16) {   // not timed: the planner's choice
    int sms = 152;
    {
      std::lock_guard<std::mutex> lock(g_mu);
      DevState* d = nullptr;
      if (ensure_device(&d) == G3_OK) sms = d->sms;
    }
    if (best_config) *best_config = -1;
    if (best_split) *best_split = dtype == G3_F32 ? simt_plan(m, n, k, sms, 0).splits : 1;
    if (best_ms) *best_ms = 0.0;
    return G3_OK;
  }
  int sms = 152;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    DevState* d = nullptr;
    const int st = ensure_device(&d);
    if (st != G3_OK) return st;
    sms = d->sms;
  }
  // Candidates are timed the way layers of a captured network run: R calls
  // back to back, replayed from a CUDA graph, cycling over enough copies of
  // the operands that together they exceed L2 four times (so that each call
  // reads operands that left L2 long ago).  Per-call time = replay time / R.
  const int es_in = input_esize(dtype);
  const int64_t lda = round_up(k, 16), ldb = round_up(n, 16);
  const size_t a_bytes = (size_t)m * lda * es_in, b_bytes = (size_t)k * ldb * es_in, c_bytes = (size_t)m * n * 4;
  const size_t set_bytes = a_bytes + b_bytes + c_bytes;
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, 0) != cudaSuccess || l2 <= 0) {
    cudaGetLastError();
    l2 = 128 << 20;
  }
  const int sets = (int)std::max<size_t>(1, std::min<size_t>(16, (4 * (size_t)l2 + set_bytes - 1) / set_bytes));
  std::vector<void*> bufs;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    for (void* b : bufs) cudaFree(b);
    cudaGetLastError();
  };
  for (int q = 0; q < sets; ++q) {
    void* b = nullptr;
    if (device_alloc(&b, set_bytes) != cudaSuccess) {
      cleanup();
      return G3_ERR_NOMEM;
    }
    bufs.push_back(b);
    // small non-zero operands (0x3C in every byte): representative tensor-core power
    cudaMemset(b, 0x3C, a_bytes + b_bytes);
  }
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cleanup();
    return G3_ERR_CUDA;
  }
  const int mode = tc_mode_of(dtype, k);
  const int bk = kblock_of(mode);
  const int num_kb = (int)((k + bk - 1) / bk);
  int best_member = -1, best_sk = 1;
  double best = 1e30;
  auto args_for = [&](int set, int member, int sk) {
    g3_gemm_args a;
    g3_gemm_args_init(&a);
    uint8_t* base = static_cast<uint8_t*>(bufs[set]);
    a.m = m; a.n = n; a.k = k;
    a.alpha = 1.0; a.beta = 0.0;
    a.A = base; a.lda = lda; a.B = base + a_bytes; a.ldb = ldb; a.C = base + a_bytes + b_bytes; a.ldc = n;
    a.dtype = dtype;
    a.config = member;
    a.split_k = sk;
    return a;
  };
  // Time of one candidate (ms per call), or 1e30 if it cannot run.
  auto time_candidate = [&](int member, int sk) -> double {
    g3_gemm_args a = args_for(0, member, sk);
    if (gemm_impl(a, s) != G3_OK) return 1e30;   // warm-up (and workspace growth) outside the capture
    float ms = 0.f;
    cudaEventRecord(e0, s);
    const int st0 = gemm_impl(a, s);
    cudaEventRecord(e1, s);
    if (st0 != G3_OK || cudaEventSynchronize(e1) != cudaSuccess) return 1e30;
    cudaEventElapsedTime(&ms, e0, e1);
    // about 2 ms of replay per measurement, at least two passes over the sets
    const int reps = std::max(2 * sets, std::min(64, std::max(4, (int)(2.0 / std::max(ms, 1e-3f)))));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return 1e30;
    int st = G3_OK;
    for (int r = 0; r < reps && st == G3_OK; ++r) {
      g3_gemm_args ar = args_for(r % sets, member, sk);
      st = gemm_impl(ar, s);
    }
    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
    double t = 1e30;
    if (st == G3_OK && ce == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess &&
        cudaGraphLaunch(exec, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess) {
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, s);
        cudaGraphLaunch(exec, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          t = 1e30;
          break;
        }
        cudaEventElapsedTime(&ms, e0, e1);
        t = std::min(t, (double)ms / reps);
      }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return t;
  };
  for (int i = 0; i < G3_FAMILY_SIZE; ++i) {
    if (!g_family[i].launch || g_family[i].mode != mode) continue;
    for (int sk : {1, G3_SPLIT_STREAM_K, 2, 3, 4, 6, 8, 12, 16}) {
      if (sk > num_kb) break;
      const double t = time_candidate(i, sk);
      if (t < best) {
        best = t;
        best_member = i;
        best_sk = sk;
      }
    }
  }
  cleanup();
  if (best_member < 0) return G3_ERR_UNSUPPORTED;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_tune[tune_key(m, n, k, dtype)] = TuneVal{best_member, best_sk, best};
  }
  (void)sms;
  if (best_config) *best_config = best_member;
  if (best_split) *best_split = best_sk;
  if (best_ms) *best_ms = best;
  return G3_OK;
}

int g3_tune_cache_save(const char* path) {
  if (!path) return -101;
  std::lock_guard<std::mutex> lock(g_mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return -101;
  std::fprintf(f, "# g3gemm tuning cache: dtype log2(m) log2(n) log2(k) member split ms\n");
  for (const auto& kv : g_tune)
    std::fprintf(f, "%d %d %d %d %d %d %.6f\n", kv.first.dtype, kv.first.bm, kv.first.bn, kv.first.bk,
                 kv.second.member, kv.second.split, kv.second.ms);
  std::fclose(f);
  return G3_OK;
}

int g3_tune_cache_load(const char* path) {
  if (!path) return -101;
  std::lock_guard<std::mutex> lock(g_mu);
  const int n = tune_load_locked(path);
  return n < 0 ? n : G3_OK;
}

int g3_tune_cache_clear(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_tune.clear();
  return G3_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free FP32-accurate GEMM.
//
// The hi/lo bfloat16 copies of A and B that the 3xBF16 mode needs live in this
// fixed array of the library's device image instead of in workspace obtained
// from cudaMalloc.  The array exists on every device that loads the library,
// for the lifetime of the process.  Its device address is looked up once per
// device (cudaGetSymbolAddress, with that device current) on the first call
// there; host code only ever passes that looked-up address to the kernels.
static constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g3_noalloc_scratch[kNoAllocScratchBytes];
static void* g3_noalloc_addr[64] = {};

extern "C" int g3_gemm_3xbf16_noalloc(int64_t m, int64_t n, int64_t k, double alpha, const float* A, int64_t lda,
                                      const float* B, int64_t ldb, double beta, float* C, int64_t ldc,
                                      void* stream) {
  g3_gemm_args a;
  g3_gemm_args_init(&a);
  a.m = m; a.n = n; a.k = k;
  a.alpha = alpha; a.beta = beta;
  a.A = A; a.lda = lda; a.B = B; a.ldb = ldb; a.C = C; a.ldc = ldc;
  a.dtype = G3_F32_3XBF16;
  a.split_k = 1;   // no split-K partials: the scratch holds the operand planes only
  int st = validate(a);
  if (st != G3_OK) return st;
  if (m == 0 || n == 0) return G3_OK;
  std::lock_guard<std::mutex> lock(g_mu);
  family_init();
  if (k > 32768) return G3_ERR_UNSUPPORTED;   // one FP32 accumulator per tile: k bounded for 2e-6
  if (k > 0 && alpha != 0.0) {
    // the planes' size depends on m, n, k only, not on the tile the planner picks
    const Plan pl = make_plan(m, n, k, G3_F32_3XBF16, 152, -1, 1, 0);
    const size_t need = make_layout(a, pl).total;
    if (need > kNoAllocScratchBytes) {
      if (std::getenv("G3_LOG"))
        std::fprintf(stderr, "g3gemm: g3_gemm_3xbf16_noalloc needs %zu bytes of scratch, the maximum is %zu\n",
                     need, kNoAllocScratchBytes);
      return G3_ERR_UNSUPPORTED;
    }
  }
  DevState* d = nullptr;
  if ((st = ensure_device(&d)) != G3_OK) return st;
  int dev = -1;
  G3_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return G3_ERR_NOT_INIT;
  if (!g3_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g3_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return G3_ERR_CUDA;
    }
    g3_noalloc_addr[dev] = p;
  }
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : g_stream;
  if (k == 0 || alpha == 0.0) {
    G3_CHECK_CUDA(launch_scale_c(C, false, (int)m, (int)n, ldc, (float)beta, s));
    return G3_OK;
  }
  a.workspace = g3_noalloc_addr[dev];
  a.workspace_bytes = kNoAllocScratchBytes;
  return run_tc(*d, a, s);
}
