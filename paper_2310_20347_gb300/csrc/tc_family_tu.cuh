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

// Persistent grid: one CTA (or CTA pair) per tile up to what can be resident
// at once -- the SM count, or for pairs the number of two-CTA clusters the GPU
// can co-schedule with this kernel's shared memory (queried once per member).
template <int BM, int ST, int MODE, int CG>
cudaError_t launch_tc(const CUtensorMap* maps, const TcParams& p, int sms, cudaStream_t s) {
  using Cfg = TcConfig<BM, ST, MODE, CG>;
  auto kern = tc_gemm_kernel<BM, ST, MODE, CG>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmemBytes);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)p.tiles_m * p.tiles_n * p.splits;
  cudaLaunchAttribute attr[2];
  if constexpr (CG == 1) {
    const int grid = (int)std::min<long long>(tiles, sms);
    const cudaLaunchConfig_t cfg = pdl_config(grid, Cfg::kThreads, Cfg::kSmemBytes, s, attr);
    e = cudaLaunchKernelEx(&cfg, kern, maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], maps[6], p);
  } else {
    static int max_clusters = 0;
    cudaLaunchConfig_t cfg = pdl_config(CG, Cfg::kThreads, Cfg::kSmemBytes, s, attr);
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = CG;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.numAttrs = 2;
    if (max_clusters <= 0) {
      int n = 0;
      e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
      if (e != cudaSuccess) return e;
      if (n <= 0) return cudaErrorInvalidConfiguration;
      max_clusters = std::min(n, sms / CG);
    }
    cfg.gridDim = dim3((unsigned)(CG * std::min<long long>(tiles, max_clusters)), 1, 1);
    e = cudaLaunchKernelEx(&cfg, kern, maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], maps[6], p);
  }
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int IDX, int MODE, int BM, int ST, int CG>
void add_member(FamilyEntry* t) {
  if constexpr (MODE == G3_TU_MODE) {
    using Cfg = TcConfig<BM, ST, MODE, CG>;
    t[IDX] = FamilyEntry{IDX, MODE, BM, ST, (int)Cfg::kSmemBytes, (int)Cfg::kNumBufs, CG, &launch_tc<BM, ST, MODE, CG>};
  }
}

template <int BM, int ST, int MODE>
cudaError_t launch_grouped(const GroupedParams& p, int grid, cudaStream_t s) {
  using Cfg = TcConfig<BM, ST, MODE>;
  auto kern = tc_grouped_kernel<BM, ST, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmemBytes);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = pdl_config(grid, Cfg::kThreads, Cfg::kSmemBytes, s, attr);
  e = cudaLaunchKernelEx(&cfg, kern, p);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int IDX, int MODE, int BM, int ST>
void add_grouped(GroupedEntry* t) {
  if constexpr (MODE == G3_TU_MODE) {
    t[IDX] = GroupedEntry{IDX, MODE, BM, ST, (int)TcConfig<BM, ST, MODE>::kSmemBytes, &launch_grouped<BM, ST, MODE>};
  }
}

}  // namespace

#define G3_ADD_MEMBER(idx, mode, bm, st, cg) add_member<idx, mode, bm, st, cg>(table);
void G3_TU_REGISTER(FamilyEntry* table) { G3_FAMILY_LIST(G3_ADD_MEMBER) }
#undef G3_ADD_MEMBER

#define G3_ADD_GROUPED(idx, mode, bm, st) add_grouped<idx, mode, bm, st>(table);
void G3_TU_REGISTER_GROUPED(GroupedEntry* table) { G3_GROUPED_LIST(G3_ADD_GROUPED) }
#undef G3_ADD_GROUPED

}  // namespace g3
