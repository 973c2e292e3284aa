// tc_family_tu.cuh -- instantiates the members of the generated family whose
// mode is G3_TU_MODE and registers their launchers under G3_TU_REGISTER.
#include "family_gen.inc"
#include "internal.h"

#include <algorithm>

namespace g3 {
namespace {

// Launch with programmatic stream serialisation: the kernel may start while
// the previous kernel of the stream drains; it waits (griddepcontrol.wait)
// before touching global memory.
inline cudaLaunchConfig_t pdl_config(int grid, int threads, size_t smem, cudaStream_t s,
                                     cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

inline void set_cluster(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int cg) {
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = cg;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.numAttrs = 2;
}

// Tiles a member can have in flight at once (its persistent slots): the SM
// count, or for pairs the number of two-CTA clusters the GPU can co-schedule
// with this kernel's shared memory (queried once per member).  0 on error.
template <int BM, int ST, int MODE, int CG>
int tc_slots(int sms) {
  if constexpr (CG == 1) {
    return sms;
  } else {
    using Cfg = TcConfig<BM, ST, MODE, CG>;
    static int max_clusters = 0;
    if (max_clusters <= 0) {
      auto kern = tc_gemm_kernel<BM, ST, MODE, CG>;
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmemBytes) !=
          cudaSuccess)
        return 0;
      cudaLaunchAttribute attr[2];
      cudaLaunchConfig_t cfg = pdl_config(CG, Cfg::kThreads, Cfg::kSmemBytes, nullptr, attr);
      set_cluster(cfg, attr, CG);
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return 0;
      }
      max_clusters = std::min(n, sms / CG);
    }
    return max_clusters;
  }
}

// Persistent grid: one CTA (or CTA pair) per tile up to the member's slots;
// with a stream-K tail exactly p.sk_streams of them (one per stream).
// RAW8 members (single-CTA INT8 reading the int8 operands as they are) take
// the raw int8 maps of A and B and C's map.
template <int BM, int ST, int MODE, int CG, bool RAW8>
cudaError_t launch_tc(const CUtensorMap* maps, const TcParams& p, int sms, cudaStream_t s) {
  using Cfg = TcConfig<BM, ST, MODE, CG, false, RAW8>;
  const int slots = tc_slots<BM, ST, MODE, CG>(sms);
  if (slots <= 0) return cudaErrorInvalidConfiguration;
  const long long work = (long long)p.tiles_m * p.tiles_n * p.splits;
  const long long clusters = p.sk_streams > 0 ? p.sk_streams : std::min<long long>(work, slots);
  cudaLaunchAttribute attr[2];
  cudaLaunchConfig_t cfg = pdl_config((int)(CG * clusters), Cfg::kThreads, Cfg::kSmemBytes, s, attr);
  if constexpr (CG > 1) set_cluster(cfg, attr, CG);
  cudaError_t e;
  if constexpr (RAW8) {
    auto kern = tc_gemm_raw8_kernel<BM, ST, MODE>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmemBytes);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernelEx(&cfg, kern, maps[0], maps[1], maps[6], p);
  } else {
    auto kern = tc_gemm_kernel<BM, ST, MODE, CG>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmemBytes);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernelEx(&cfg, kern, maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], maps[6], p);
  }
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int IDX, int MODE, int BM, int ST, int CG, int RAW8>
void add_member(FamilyEntry* t) {
  if constexpr (MODE == G3_TU_MODE) {
    using Cfg = TcConfig<BM, ST, MODE, CG, false, RAW8 != 0>;
    t[IDX] = FamilyEntry{IDX, MODE, BM, ST, (int)Cfg::kSmemBytes, (int)Cfg::kNumBufs, CG,
                         &launch_tc<BM, ST, MODE, CG, RAW8 != 0>, &tc_slots<BM, ST, MODE, CG>,
                         TcStreamK<BM, MODE>::value, RAW8 != 0};
  }
}

template <int BM, int ST, int MODE, bool FUSED>
cudaError_t launch_grouped(const GroupedParams& p, int grid, cudaStream_t s) {
  using Cfg = TcConfig<BM, ST, MODE, 1, FUSED>;
  void (*kern)(const GroupedParams);
  if constexpr (FUSED) kern = tc_grouped_fused_kernel<BM, ST, MODE>;
  else kern = tc_grouped_kernel<BM, ST, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmemBytes);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = pdl_config(grid, Cfg::kThreads, Cfg::kSmemBytes, s, attr);
  e = cudaLaunchKernelEx(&cfg, kern, p);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int IDX, int MODE, int BM, int ST, int FUSED>
void add_grouped(GroupedEntry* t) {
  if constexpr (MODE == G3_TU_MODE) {
    t[IDX] = GroupedEntry{IDX, MODE, BM, ST, (int)TcConfig<BM, ST, MODE, 1, FUSED != 0>::kSmemBytes,
                          &launch_grouped<BM, ST, MODE, FUSED != 0>, FUSED};
  }
}

}  // namespace

#define G3_ADD_MEMBER(idx, mode, bm, st, cg, raw8) add_member<idx, mode, bm, st, cg, raw8>(table);
void G3_TU_REGISTER(FamilyEntry* table) { G3_FAMILY_LIST(G3_ADD_MEMBER) }
#undef G3_ADD_MEMBER

#define G3_ADD_GROUPED(idx, mode, bm, st, fused) add_grouped<idx, mode, bm, st, fused>(table);
void G3_TU_REGISTER_GROUPED(GroupedEntry* table) { G3_GROUPED_LIST(G3_ADD_GROUPED) }
#undef G3_ADD_GROUPED

}  // namespace g3
