// grouped.cu -- many independent GEMMs of uneven shapes in one persistent launch.
//
// A plan (g3_grouped_plan_create) does all host work once: validation, the
// per-problem choice of tile height by size bucket (the per-shape selection of
// the paper's Section 8.4, applied problem by problem), the global tile list
// ordered by decreasing k-depth (heaviest tiles first, so that the static
// stride of the persistent CTAs balances), six TMA descriptors per problem in
// a device table, and the preparation jobs (FP32 hi/lo or hi/mid/lo split,
// re-packing of unaligned BF16 / FP8 operands, C := beta*C for problems
// without products).
// Executing the plan is one job kernel over all preparation jobs and one
// tc_grouped_kernel per kernel kind over its tiles -- BF16, FP8: one; FP32-accurate:
// the two-part split (3 products) for problems with k > 512 and the
// three-part split (6 products) for those with k <= 512 -- with no host
// synchronisation and no allocation.  On request (G3_GROUPED_SPLIT_IN_KERNEL)
// FP32-accurate plans split inside the kernel instead
// (tc_grouped_fused_kernel: loader-converter warps read each tile's FP32
// operands and write its bf16 parts into shared memory), with no split jobs
// and no planes.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "family_gen.inc"
#include "g3gemm.h"
#include "internal.h"
#include "bf16.cuh"

namespace g3 {
namespace {

enum PrepKind : int { PREP_SPLIT = 0, PREP_COPY16 = 1, PREP_SCALE_C = 2, PREP_SPLIT3 = 3, PREP_COPY8 = 4 };

// One preparation job of a grouped plan.
struct PrepJob {
  const void* src;
  long long ld_src;   // elements
  void* hi;           // PREP_SPLIT(3): hi plane; PREP_COPY16 / PREP_COPY8: destination
  void* lo;           // PREP_SPLIT(3): lo plane
  void* mid;          // PREP_SPLIT3: mid plane
  long long ld_dst;   // elements; destination rows start on 16-byte boundaries
  int rows, cols;
  int kind;
  float beta;         // PREP_SCALE_C
  int vec;            // float source rows 16-byte aligned: 16-byte loads
};

__device__ __forceinline__ uint32_t pack2(uint16_t a, uint16_t b) {
  return static_cast<uint32_t>(a) | (static_cast<uint32_t>(b) << 16);
}
__device__ __forceinline__ void store8(uint16_t* dst, const uint16_t (&v)[8], int cnt) {
  if (cnt == 8) {
    *reinterpret_cast<uint4*>(dst) = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
  } else {
    for (int i = 0; i < cnt; ++i) dst[i] = v[i];
  }
}

// blockIdx.y strides over jobs, the x-dimension over each job's units of 8
// consecutive elements of a row (a grouped problem is at most 2^31 elements,
// so 32-bit index arithmetic); planes are written with 16-byte stores.
__global__ void grouped_prep_kernel(const PrepJob* __restrict__ jobs, int njobs) {
  for (int jb = blockIdx.y; jb < njobs; jb += gridDim.y) {
    const PrepJob J = jobs[jb];
    if (J.kind == PREP_SCALE_C) {
      const unsigned total = (unsigned)J.rows * (unsigned)J.cols;
      const unsigned cols = (unsigned)J.cols;
      for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const unsigned r = e / cols, c = e - r * cols;
        float* p = static_cast<float*>(const_cast<void*>(J.src)) + r * J.ld_src + c;
        *p = (J.beta == 0.f) ? 0.f : J.beta * *p;
      }
      continue;
    }
    if (J.kind == PREP_COPY8) {   // 8-bit elements, 16 per unit, destination rows 16-byte aligned
      const unsigned upr8 = ((unsigned)J.cols + 15u) >> 4;
      const unsigned total8 = (unsigned)J.rows * upr8;
      for (unsigned u = blockIdx.x * blockDim.x + threadIdx.x; u < total8; u += gridDim.x * blockDim.x) {
        const unsigned r = u / upr8, c0 = (u - r * upr8) << 4;
        const int cnt = min(16, J.cols - (int)c0);
        const uint8_t* xr = static_cast<const uint8_t*>(J.src) + (long long)r * J.ld_src + c0;
        uint8_t* yr = static_cast<uint8_t*>(J.hi) + (long long)r * J.ld_dst + c0;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        for (int i = 0; i < cnt; ++i) w[i >> 2] |= static_cast<uint32_t>(xr[i]) << (8 * (i & 3));
        *reinterpret_cast<uint4*>(yr) = make_uint4(w[0], w[1], w[2], w[3]);
      }
      continue;
    }
    const unsigned upr = ((unsigned)J.cols + 7u) >> 3;   // units per row
    const unsigned total = (unsigned)J.rows * upr;
    for (unsigned u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
      const unsigned r = u / upr, c0 = (u - r * upr) << 3;
      const int cnt = min(8, J.cols - (int)c0);
      const long long dofs = (long long)r * J.ld_dst + c0;
      if (J.kind == PREP_COPY16) {
        const uint16_t* xr = static_cast<const uint16_t*>(J.src) + (long long)r * J.ld_src + c0;
        uint16_t v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = i < cnt ? xr[i] : 0;
        store8(static_cast<uint16_t*>(J.hi) + dofs, v, cnt);
        continue;
      }
      const float* xr = static_cast<const float*>(J.src) + (long long)r * J.ld_src + c0;
      float x[8];
      if (J.vec && cnt == 8) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(xr));
        const float4 b = __ldcs(reinterpret_cast<const float4*>(xr) + 1);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = i < cnt ? xr[i] : 0.f;
      }
      uint16_t h[8], l[8];
      if (J.kind == PREP_SPLIT3) {
        uint16_t md[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          h[i] = bf16_bits(x[i]);
          const float d = x[i] - bf16_value(h[i]);
          md[i] = bf16_bits(d);
          l[i] = bf16_bits(d - bf16_value(md[i]));
        }
        store8(static_cast<uint16_t*>(J.mid) + dofs, md, cnt);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          h[i] = bf16_bits(x[i]);
          l[i] = bf16_bits(x[i] - bf16_value(h[i]));
        }
      }
      store8(static_cast<uint16_t*>(J.hi) + dofs, h, cnt);
      store8(static_cast<uint16_t*>(J.lo) + dofs, l, cnt);
    }
  }
}

GroupedEntry g_grouped[G3_GROUPED_SIZE];
bool g_grouped_ready = false;

void grouped_init() {
  if (g_grouped_ready) return;
  std::memset(g_grouped, 0, sizeof(g_grouped));
  register_grouped_bf16(g_grouped);
  register_grouped_3xbf16(g_grouped);
  register_grouped_fp8(g_grouped);
  register_grouped_int8emu(g_grouped);
  register_grouped_6xbf16(g_grouped);
  g_grouped_ready = true;
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
bool aligned16(const void* p, int64_t ld, int es) {
  return reinterpret_cast<uintptr_t>(p) % 16 == 0 && (ld * es) % 16 == 0;
}

}  // namespace
}  // namespace g3

using namespace g3;

struct g3_grouped_plan {
  int device = -1;
  int dtype = 0;
  int count = 0;
  int total_tiles = 0;
  int njobs = 0;
  int sms = 0;
  void* dmem = nullptr;  // one allocation: maps | problems | tile list | jobs | operand planes
  // one persistent launch per kernel kind: its grouped kernel (index into the
  // table) and its part of the tile list
  int nparts = 0;
  int entry[2] = {-1, -1};
  GroupedParams params[2]{};
  PrepJob* d_jobs = nullptr;
  // per problem: tile height and kernel kind (0: the plan's first launch, 1:
  // the three-part split), -1 / -1 for problems without products
  std::vector<int> bms, kinds;
  bool fused = false;   // FP32-accurate split inside the grouped kernels
  // Two kernel kinds with preparation jobs each (FP32-accurate, split in a
  // pre-pass): kind 0's jobs and launch run on a plan-owned side stream,
  // forked from and joined back into the caller's stream, beside kind 1's.
  int njobs0 = 0;       // jobs of kind 0 (and the C := beta*C jobs) first, then kind 1's
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

// force_bm > 0: every problem takes tiles of force_bm rows (g3_autotune_grouped);
// otherwise the tuning record of the problem's size bucket, else the fixed
// rule (64 rows for m <= 64, 128 above).  flags & G3_GROUPED_SPLIT_IN_KERNEL:
// FP32-accurate plans split inside the kernel, on 64-row tiles.
int plan_create(int count, const g3_gemm_desc* descs, int dtype, int force_bm, int flags, g3_grouped_plan** out) {
  if (!out) return G3_ERR_ARG;
  *out = nullptr;
  if (count < 0) return -101;
  if (count > 0 && !descs) return -102;
  if (dtype != G3_BF16 && dtype != G3_F32_3XBF16 && dtype != G3_FP8_E4M3) return G3_ERR_UNSUPPORTED;
  if (flags & ~G3_GROUPED_SPLIT_IN_KERNEL) return G3_ERR_ARG;
  const bool fp8 = dtype == G3_FP8_E4M3;
  const bool fused = dtype == G3_F32_3XBF16 && (flags & G3_GROUPED_SPLIT_IN_KERNEL) && force_bm <= 0;
  for (int i = 0; i < count; ++i) {
    const g3_gemm_desc& d = descs[i];
    const int code = i < 900 ? -(100 + i) : G3_ERR_ARG;
    if (d.m < 0 || d.n < 0 || d.k < 0) return code;
    if (d.m > INT32_MAX || d.n > INT32_MAX || d.k > INT32_MAX) return G3_ERR_UNSUPPORTED;
    // every operand and C of one problem must fit 32-bit element indexing
    if (d.m * d.k > INT32_MAX || d.k * d.n > INT32_MAX || d.m * d.n > INT32_MAX) return G3_ERR_UNSUPPORTED;
    if (d.lda < std::max<int64_t>(1, d.k) || d.ldb < std::max<int64_t>(1, d.n) ||
        d.ldc < std::max<int64_t>(1, d.n))
      return code;
    if (d.m > 0 && d.n > 0) {
      if (!d.C) return code;
      if (d.k > 0 && d.alpha != 0.0 && (!d.A || !d.B)) return code;
    }
    if (fp8 && !(std::isfinite(d.scale_a) && std::isfinite(d.scale_b) && d.scale_a > 0.f && d.scale_b > 0.f))
      return code;
  }
  std::lock_guard<std::mutex> lock(api_mutex());
  DeviceInfo dev;
  int st = current_device_info(&dev);
  if (st != G3_OK) return st;
  grouped_init();
  // FP32-accurate problems with k <= 512 take the three-part split (6
  // products), where the two-part split's dropped terms exceed 2e-6 of
  // sum |a||b|; deeper ones the two-part split (3 products).  Each kind runs
  // as its own persistent launch (part 0: BF16 or the two-part split; part 1:
  // the three-part split).
  auto entry_of = [fused](int mode) {
    int e = -1;
    for (int i = 0; i < G3_GROUPED_SIZE; ++i)
      if (g_grouped[i].launch && g_grouped[i].mode == mode && (g_grouped[i].fused != 0) == fused) e = i;
    return e;
  };
  const bool split_mode = dtype == G3_F32_3XBF16;
  const int entries[2] = {entry_of(dtype == G3_BF16 ? TC_BF16 : (fp8 ? TC_FP8 : TC_3XBF16)),
                          split_mode ? entry_of(TC_6XBF16) : -1};
  if (entries[0] < 0 || (split_mode && entries[1] < 0)) return G3_ERR_UNSUPPORTED;
  auto part_of = [&](int64_t k) { return (split_mode && k <= 512) ? 1 : 0; };
  const int es = fp8 ? 1 : 2;          // bytes per operand element on the tensor core
  const int bk = fp8 ? 128 : 64;       // k per k-block: one 128-byte row
  const int bm_max = std::min(g_grouped[entries[0]].bm_max, entries[1] >= 0 ? g_grouped[entries[1]].bm_max : 1 << 30);

  // ---- per-problem tiling, jobs and plane sizes (host)
  std::vector<GroupDesc> groups(count);
  std::vector<PrepJob> jobs;
  std::vector<int> job_kind;   // kernel kind whose launch reads the job's output (0 for C := beta*C)
  struct Operands { size_t a_off = 0, a_lo_off = 0, b_off = 0, b_lo_off = 0, a_mid_off = 0, b_mid_off = 0;
                    int64_t lda = 0, ldb = 0;
                    bool pack_a = false, pack_b = false; bool active = false; };
  std::vector<Operands> ops(count);
  size_t planes = 0;
  auto take = [&](size_t bytes) { size_t o = planes; planes = align256(planes + bytes); return o; };
  long long total_tiles = 0;
  for (int i = 0; i < count; ++i) {
    const g3_gemm_desc& d = descs[i];
    GroupDesc& g = groups[i];
    std::memset(&g, 0, sizeof(g));
    g.m = (int)d.m; g.n = (int)d.n; g.k = (int)d.k;
    g.alpha = (float)(fp8 ? d.alpha * (double)d.scale_a * (double)d.scale_b : d.alpha);
    g.beta = (float)d.beta;
    g.C = static_cast<float*>(d.C);
    g.ldc = d.ldc;
    if (fused) {   // the loader-converter warps read the FP32 operands in place
      g.A = static_cast<const float*>(d.A);
      g.B = static_cast<const float*>(d.B);
      g.lda = d.lda;
      g.ldb = d.ldb;
    }
    const int tuned = fused ? 0 : (force_bm > 0 ? force_bm : tuned_grouped_bm(d.m, d.n, d.k, dtype));
    g.bm = std::min(tuned > 0 ? tuned : ((d.m <= 64) ? 64 : 128), bm_max);   // size bucket
    if (d.m == 0 || d.n == 0) continue;
    if (d.k == 0 || d.alpha == 0.0) {
      PrepJob J{};
      J.src = d.C; J.ld_src = d.ldc; J.rows = g.m; J.cols = g.n; J.kind = PREP_SCALE_C; J.beta = (float)d.beta;
      jobs.push_back(J);
      job_kind.push_back(0);
      continue;
    }
    Operands& o = ops[i];
    o.active = true;
    g.tiles_m = (g.m + g.bm - 1) / g.bm;
    g.tiles_n = (g.n + 127) / 128;
    g.num_kb = (g.k + bk - 1) / bk;
    total_tiles += (long long)g.tiles_m * g.tiles_n;
    if (fused) {
      // no planes, no jobs
    } else if (dtype == G3_F32_3XBF16) {
      o.lda = round_up(d.k, 8);
      o.ldb = round_up(d.n, 8);
      o.a_off = take((size_t)d.m * o.lda * 2);
      o.a_lo_off = take((size_t)d.m * o.lda * 2);
      o.b_off = take((size_t)d.k * o.ldb * 2);
      o.b_lo_off = take((size_t)d.k * o.ldb * 2);
      if (part_of(d.k) == 1) {
        o.a_mid_off = take((size_t)d.m * o.lda * 2);
        o.b_mid_off = take((size_t)d.k * o.ldb * 2);
      }
    } else {
      o.pack_a = !aligned16(d.A, d.lda, es);
      o.pack_b = !aligned16(d.B, d.ldb, es);
      o.lda = o.pack_a ? round_up(d.k, 16 / es) : d.lda;
      o.ldb = o.pack_b ? round_up(d.n, 16 / es) : d.ldb;
      if (o.pack_a) o.a_off = take((size_t)d.m * o.lda * es);
      if (o.pack_b) o.b_off = take((size_t)d.k * o.ldb * es);
    }
  }
  if (total_tiles > INT32_MAX) return G3_ERR_UNSUPPORTED;

  // ---- device memory: maps | problems | tile list | jobs | planes
  const size_t maps_bytes = align256(sizeof(CUtensorMap) * kMapsPerProblem * (size_t)std::max(count, 1));
  const size_t groups_bytes = align256(sizeof(GroupDesc) * (size_t)std::max(count, 1));
  const size_t tiles_bytes = align256(sizeof(int2) * (size_t)std::max<long long>(total_tiles, 1));
  const size_t njobs_max = jobs.size() + 2 * (size_t)count;
  const size_t jobs_bytes = align256(sizeof(PrepJob) * std::max<size_t>(njobs_max, 1));
  const size_t header = maps_bytes + groups_bytes + tiles_bytes + jobs_bytes;
  g3_grouped_plan* plan = new g3_grouped_plan();
  if (device_alloc(&plan->dmem, header + planes) != cudaSuccess) {
    cudaGetLastError();
    delete plan;
    return G3_ERR_NOMEM;
  }
  uint8_t* base = static_cast<uint8_t*>(plan->dmem);
  CUtensorMap* d_maps = reinterpret_cast<CUtensorMap*>(base);
  GroupDesc* d_groups = reinterpret_cast<GroupDesc*>(base + maps_bytes);
  int2* d_tiles = reinterpret_cast<int2*>(base + maps_bytes + groups_bytes);
  PrepJob* d_jobs = reinterpret_cast<PrepJob*>(base + maps_bytes + groups_bytes + tiles_bytes);
  uint8_t* d_planes = base + header;

  std::vector<CUtensorMap> maps(kMapsPerProblem * (size_t)std::max(count, 1));
  std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
  for (int i = 0; i < count && st == G3_OK; ++i) {
    if (!ops[i].active || fused) continue;   // the fused kernels use no tensor maps
    const g3_gemm_desc& d = descs[i];
    const Operands& o = ops[i];
    const GroupDesc& g = groups[i];
    const void *a = d.A, *b = d.B, *a_lo = nullptr, *b_lo = nullptr, *a_mid = nullptr, *b_mid = nullptr;
    const bool split3 = part_of(d.k) == 1;
    if (dtype == G3_F32_3XBF16) {
      a = d_planes + o.a_off; a_lo = d_planes + o.a_lo_off;
      b = d_planes + o.b_off; b_lo = d_planes + o.b_lo_off;
      const int kind = split3 ? PREP_SPLIT3 : PREP_SPLIT;
      if (split3) {
        a_mid = d_planes + o.a_mid_off;
        b_mid = d_planes + o.b_mid_off;
      }
      const int va = aligned16(d.A, d.lda, 4) ? 1 : 0, vb = aligned16(d.B, d.ldb, 4) ? 1 : 0;
      jobs.push_back(PrepJob{d.A, d.lda, (void*)a, (void*)a_lo, (void*)a_mid, o.lda, g.m, g.k, kind, 0.f, va});
      jobs.push_back(PrepJob{d.B, d.ldb, (void*)b, (void*)b_lo, (void*)b_mid, o.ldb, g.k, g.n, kind, 0.f, vb});
      job_kind.push_back(part_of(d.k));
      job_kind.push_back(part_of(d.k));
    } else {
      const int copy = fp8 ? PREP_COPY8 : PREP_COPY16;
      if (o.pack_a) {
        a = d_planes + o.a_off;
        jobs.push_back(PrepJob{d.A, d.lda, (void*)a, nullptr, nullptr, o.lda, g.m, g.k, copy, 0.f, 0});
        job_kind.push_back(0);
      }
      if (o.pack_b) {
        b = d_planes + o.b_off;
        jobs.push_back(PrepJob{d.B, d.ldb, (void*)b, nullptr, nullptr, o.ldb, g.k, g.n, copy, 0.f, 0});
        job_kind.push_back(0);
      }
    }
    // maps 2p, 2p+1 = A, B of plane p: hi; then lo (two-part) or mid, lo
    // (three-part); unused planes repeat plane 0
    CUtensorMap* mp = &maps[kMapsPerProblem * (size_t)i];
    // A: boxes of one 128-byte k-block row x bm rows; B: 128 bytes of n x one k-block
    st = encode_tensor_2d(&mp[0], a, es, g.k, g.m, o.lda, bk, g.bm);
    if (st == G3_OK) st = encode_tensor_2d(&mp[1], b, es, g.n, g.k, o.ldb, 128 / es, bk);
    mp[2] = mp[4] = mp[0];
    mp[3] = mp[5] = mp[1];
    const void* p1a = split3 ? a_mid : a_lo;
    const void* p1b = split3 ? b_mid : b_lo;
    if (st == G3_OK && dtype == G3_F32_3XBF16) {
      st = encode_tensor_2d(&mp[2], p1a, 2, g.k, g.m, o.lda, 64, g.bm);
      if (st == G3_OK) st = encode_tensor_2d(&mp[3], p1b, 2, g.n, g.k, o.ldb, 64, 64);
    }
    if (st == G3_OK && split3) {
      st = encode_tensor_2d(&mp[4], a_lo, 2, g.k, g.m, o.lda, 64, g.bm);
      if (st == G3_OK) st = encode_tensor_2d(&mp[5], b_lo, 2, g.n, g.k, o.ldb, 64, 64);
    }
  }
  if (st != G3_OK) {
    cudaFree(plan->dmem);
    delete plan;
    return st;
  }

  // tile list: part 0 then part 1, each heaviest (deepest k) problems first;
  // ties keep problem order
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return groups[x].num_kb * groups[x].bm > groups[y].num_kb * groups[y].bm; });
  std::vector<int2> tiles;
  tiles.reserve((size_t)total_tiles);
  int part_tiles[2] = {0, 0};
  for (int part = 0; part < 2; ++part)
    for (int i : order) {
      if (!ops[i].active || part_of(descs[i].k) != part) continue;
      const int nt = groups[i].tiles_m * groups[i].tiles_n;
      for (int t = 0; t < nt; ++t) tiles.push_back(make_int2(i, t));
      part_tiles[part] += nt;
    }

  // kind 0's jobs first, then kind 1's (order kept within each)
  std::vector<PrepJob> ordered;
  ordered.reserve(jobs.size());
  for (int kind = 0; kind < 2; ++kind)
    for (size_t q = 0; q < jobs.size(); ++q)
      if (job_kind[q] == kind) ordered.push_back(jobs[q]);
  const int njobs0 = (int)std::count(job_kind.begin(), job_kind.end(), 0);
  jobs.swap(ordered);
  bool ok = true;
  ok = ok && cudaMemcpy(d_maps, maps.data(), sizeof(CUtensorMap) * kMapsPerProblem * (size_t)count,
                        cudaMemcpyHostToDevice) ==
                 cudaSuccess;
  ok = ok && cudaMemcpy(d_groups, groups.data(), sizeof(GroupDesc) * (size_t)count, cudaMemcpyHostToDevice) ==
                 cudaSuccess;
  if (!tiles.empty())
    ok = ok && cudaMemcpy(d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!jobs.empty())
    ok = ok && cudaMemcpy(d_jobs, jobs.data(), sizeof(PrepJob) * jobs.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cudaFree(plan->dmem);
    delete plan;
    return G3_ERR_CUDA;
  }
  plan->bms.assign(count, -1);
  plan->kinds.assign(count, -1);
  for (int i = 0; i < count; ++i)
    if (ops[i].active) {
      plan->bms[i] = groups[i].bm;
      plan->kinds[i] = part_of(descs[i].k);
    }
  plan->device = dev.device;
  plan->dtype = dtype;
  plan->fused = fused;
  plan->count = count;
  plan->total_tiles = (int)total_tiles;
  plan->njobs = (int)jobs.size();
  plan->njobs0 = njobs0;
  plan->sms = dev.sms;
  plan->d_jobs = d_jobs;
  int first = 0;
  for (int part = 0; part < 2; ++part) {
    if (part_tiles[part] == 0) continue;
    GroupedParams& p = plan->params[plan->nparts];
    p.groups = d_groups;
    p.maps = d_maps;
    p.tile_info = d_tiles + first;
    p.total_tiles = part_tiles[part];
    p.timeout_ns = watchdog_timeout_ns();
    p.status = dev.status;
    p.debug_withhold = -1;
    plan->entry[plan->nparts] = entries[part];
    ++plan->nparts;
    first += part_tiles[part];
  }
  if (plan->nparts == 2 && plan->njobs0 > 0 && plan->njobs > plan->njobs0) {
    if (cudaStreamCreateWithFlags(&plan->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      g3_grouped_plan_destroy(plan);
      return G3_ERR_CUDA;
    }
  }
  *out = plan;
  return G3_OK;
}

}  // namespace

extern "C" {

int g3_grouped_plan_create(int count, const g3_gemm_desc* descs, int dtype, g3_grouped_plan** out) {
  return plan_create(count, descs, dtype, 0, 0, out);
}

int g3_grouped_plan_create_ex(int count, const g3_gemm_desc* descs, int dtype, int flags, g3_grouped_plan** out) {
  return plan_create(count, descs, dtype, 0, flags, out);
}

int g3_grouped_plan_describe(const g3_grouped_plan* plan, int index, int* bm, int* kind) {
  if (!plan) return -101;
  if (index < 0 || index >= plan->count) return -102;
  if (bm) *bm = plan->bms[index];
  if (kind) *kind = plan->kinds[index];
  return G3_OK;
}

int g3_grouped_plan_execute(g3_grouped_plan* plan, void* stream) {
  if (!plan) return -101;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) {
    cudaGetLastError();
    return G3_ERR_ARG;
  }
  auto prep = [&](const PrepJob* jobs, int n, cudaStream_t st) -> bool {
    if (n <= 0) return true;
    const dim3 grid(16, (unsigned)std::min(n, 65535));
    grouped_prep_kernel<<<grid, 256, 0, st>>>(jobs, n);
    count_launch();
    return cudaGetLastError() == cudaSuccess;
  };
  const bool forked = plan->side != nullptr && plan->total_tiles > 0;
  if (!forked && !prep(plan->d_jobs, plan->njobs, s)) return G3_ERR_CUDA;
  if (plan->total_tiles == 0) return G3_OK;
  GroupedParams p[2] = {plan->params[0], plan->params[1]};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  {
    std::lock_guard<std::mutex> lock(api_mutex());
    unsigned long long t = 0;
    if (take_withhold(&t)) {   // failure-detection test hook: the first launch
      p[0].debug_withhold = 0;
      p[0].timeout_ns = t;
    }
    if (kernel_timing_enabled()) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
    }
  }
  if (e0) cudaEventRecord(e0, s);
  cudaError_t e = cudaSuccess;
  if (forked) {
    // kind 0's jobs and launch on the side stream, kind 1's on the caller's
    // (measured: the two kinds' split passes together reach more bandwidth
    // than one; kind 0's jobs first, then its launch beside kind 1's jobs,
    // gained nothing), then join
    if (cudaEventRecord(plan->ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(plan->side, plan->ev_fork, 0) != cudaSuccess)
      return G3_ERR_CUDA;
    if (!prep(plan->d_jobs, plan->njobs0, plan->side)) return G3_ERR_CUDA;
    e = g_grouped[plan->entry[0]].launch(p[0], std::min(p[0].total_tiles, plan->sms), plan->side);
    if (e == cudaSuccess && !prep(plan->d_jobs + plan->njobs0, plan->njobs - plan->njobs0, s)) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = g_grouped[plan->entry[1]].launch(p[1], std::min(p[1].total_tiles, plan->sms), s);
    if (e == cudaSuccess && (cudaEventRecord(plan->ev_join, plan->side) != cudaSuccess ||
                             cudaStreamWaitEvent(s, plan->ev_join, 0) != cudaSuccess))
      e = cudaErrorUnknown;
  } else {
    for (int part = 0; part < plan->nparts && e == cudaSuccess; ++part) {
      const int grid = std::min(p[part].total_tiles, plan->sms);
      e = g_grouped[plan->entry[part]].launch(p[part], grid, s);
    }
  }
  if (e1) {
    cudaEventRecord(e1, s);
    std::lock_guard<std::mutex> lock(api_mutex());
    kernel_timing_push(e0, e1);
  }
  if (e != cudaSuccess) {
    if (std::getenv("G3_LOG")) std::fprintf(stderr, "g3gemm: grouped launch: %s\n", cudaGetErrorString(e));
    return G3_ERR_CUDA;
  }
  return G3_OK;
}

int g3_grouped_plan_destroy(g3_grouped_plan* plan) {
  if (!plan) return G3_OK;
  if (plan->dmem) {
    cudaFree(plan->dmem);   // synchronises with work still using the plan
    cudaGetLastError();
  }
  if (plan->side) cudaStreamDestroy(plan->side);
  if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
  if (plan->ev_join) cudaEventDestroy(plan->ev_join);
  cudaGetLastError();
  delete plan;
  return G3_OK;
}

int g3_gemm_grouped(int count, const g3_gemm_desc* descs, int dtype, void* stream) {
  g3_grouped_plan* plan = nullptr;
  int st = g3_grouped_plan_create(count, descs, dtype, &plan);
  if (st != G3_OK) return st;
  st = g3_grouped_plan_execute(plan, stream);
  if (st == G3_OK && cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    cudaGetLastError();
    st = G3_ERR_CUDA;
  }
  g3_grouped_plan_destroy(plan);
  return st;
}

// Per size bucket: a plan of P problems of shape m x n x k (about two waves
// of 128-row tiles, at most 256 problems and 1 GiB of operands) is timed with
// every problem on tiles of 64 rows and of 128 rows, each as a CUDA graph of
// back-to-back plan executions; the faster height is recorded for the bucket.
int g3_autotune_grouped(int64_t m, int64_t n, int64_t k, int dtype, int* best_bm, double* best_ms) {
  if (m <= 0) return -101;
  if (n <= 0) return -102;
  if (k <= 0) return -103;
  if (dtype != G3_BF16 && dtype != G3_F32_3XBF16 && dtype != G3_FP8_E4M3) return -104;
  if (m * k > INT32_MAX || k * n > INT32_MAX || m * n > INT32_MAX) return G3_ERR_UNSUPPORTED;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lock(api_mutex());
    DeviceInfo dev;
    const int st = current_device_info(&dev);
    if (st != G3_OK) return st;
    sms = dev.sms;
  }
  const int es = dtype == G3_F32_3XBF16 ? 4 : (dtype == G3_FP8_E4M3 ? 1 : 2);
  const int64_t lda = round_up(k, 16), ldb = round_up(n, 16);
  const size_t a_bytes = align256((size_t)m * lda * es), b_bytes = align256((size_t)k * ldb * es);
  const size_t c_bytes = align256((size_t)m * n * 4);
  const size_t per = a_bytes + b_bytes + c_bytes;
  const long long tiles128 = ((m + 127) / 128) * ((n + 127) / 128);
  int P = (int)std::min<long long>(256, std::max<long long>(4, (2LL * sms + tiles128 - 1) / tiles128));
  while (P > 1 && (size_t)P * per > (size_t(1) << 30)) --P;
  void* buf = nullptr;
  if (device_alloc(&buf, (size_t)P * per) != cudaSuccess) {
    cudaGetLastError();
    return G3_ERR_NOMEM;
  }
  cudaMemset(buf, 0x3C, (size_t)P * per);   // small non-zero operands in every format
  std::vector<g3_gemm_desc> descs(P);
  for (int i = 0; i < P; ++i) {
    uint8_t* base = static_cast<uint8_t*>(buf) + (size_t)i * per;
    g3_gemm_desc& d = descs[i];
    std::memset(&d, 0, sizeof(d));
    d.m = m; d.n = n; d.k = k;
    d.lda = lda; d.ldb = ldb; d.ldc = n;
    d.alpha = 1.0; d.beta = 0.0;
    d.A = base; d.B = base + a_bytes; d.C = base + a_bytes + b_bytes;
    d.scale_a = d.scale_b = 1.0f;
  }
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = G3_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    st = G3_ERR_CUDA;
  int best = 0;
  double best_t = 1e30;
  for (int bm : {128, 64}) {
    if (st != G3_OK) break;
    g3_grouped_plan* plan = nullptr;
    if (plan_create(P, descs.data(), dtype, bm, 0, &plan) != G3_OK) continue;
    float ms = 0.f;
    double t = 1e30;
    cudaEventRecord(e0, s);
    const int st0 = g3_grouped_plan_execute(plan, s);
    cudaEventRecord(e1, s);
    if (st0 == G3_OK && cudaEventSynchronize(e1) == cudaSuccess) {
      cudaEventElapsedTime(&ms, e0, e1);
      const int reps = std::min(64, std::max(4, (int)(2.0 / std::max(ms, 1e-3f))));
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      int sc = G3_OK;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        for (int r = 0; r < reps && sc == G3_OK; ++r) sc = g3_grouped_plan_execute(plan, s);
        const cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (sc == G3_OK && ce == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess &&
            cudaGraphLaunch(exec, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess) {
          for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, s);
            cudaGraphLaunch(exec, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, (double)ms / reps);
          }
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
      }
    }
    cudaGetLastError();
    g3_grouped_plan_destroy(plan);
    if (t < best_t) {
      best_t = t;
      best = bm;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(buf);
  cudaGetLastError();
  if (st != G3_OK) return st;
  if (best == 0) return G3_ERR_UNSUPPORTED;
  {
    std::lock_guard<std::mutex> lock(api_mutex());
    store_grouped_tuning(m, n, k, dtype, best, best_t);
  }
  if (best_bm) *best_bm = best;
  if (best_ms) *best_ms = best_t;
  return G3_OK;
}

}  // extern "C"
