// fmm_fused_ts.cu -- instantiations and launcher of the fused kernel whose A-operand sums are
// held in tensor memory (fmm_fused_ts.cuh).
#include <cuda_runtime.h>
#include <algorithm>
#include "fmm_fused_ts.cuh"
#include "launch.h"

namespace fmm {

template <int TERMS, bool A_MN, bool B_KM, bool F16 = false, bool S16 = false>
static cudaError_t launch_fused_ts_t(const FusedParams& p, int grid, cudaStream_t s) {
  using Cfg = FusedTsCfg<TERMS>;
  static_assert(Cfg::kSmemBytes <= 232448, "shared memory per CTA");
  auto kern = fmm_fused_ts_kernel<TERMS, A_MN, B_KM, F16, S16>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(Cfg::kSmemBytes));
  if (e != cudaSuccess) return e;
  if (grid < 2 || grid % 2 != 0) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(fused_threads<8>(), 1, 1);
  cfg.dynamicSmemBytes = Cfg::kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // at most one wave of CTA pairs (how many fit depends on how the SMs are grouped)
  cfg.gridDim = dim3(static_cast<unsigned>(grid), 1, 1);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters >= 1)
    grid = std::min(grid, 2 * clusters);
  else
    cudaGetLastError();
  cfg.gridDim = dim3(static_cast<unsigned>(grid), 1, 1);
  return cudaLaunchKernelEx(&cfg, kern, p);
}

cudaError_t launch_fused_ts(const FusedParams& p, int terms, bool a_mn, bool b_mn, bool f16, bool s16, int grid,
                            cudaStream_t s) {
  // forward (A K-major, B MN-major), dA = dC B^T (B stored by rows of n), dB = A^T dC (A
  // stored by rows of k); FP16 operands with panel scaling, and 16-bit source tiles: forward
  // only
  const bool fwd = !a_mn && b_mn;
  if (s16) {
    if (terms != 1 || !fwd) return cudaErrorInvalidValue;
    return f16 ? launch_fused_ts_t<1, false, false, true, true>(p, grid, s)
               : launch_fused_ts_t<1, false, false, false, true>(p, grid, s);
  }
  if (f16) return (terms == 1 && fwd) ? launch_fused_ts_t<1, false, false, true>(p, grid, s) : cudaErrorInvalidValue;
  if (!a_mn && b_mn) {
    if (terms == 3) return launch_fused_ts_t<3, false, false>(p, grid, s);
    if (terms == 1) return launch_fused_ts_t<1, false, false>(p, grid, s);
  } else if (!a_mn && !b_mn) {
    if (terms == 3) return launch_fused_ts_t<3, false, true>(p, grid, s);
    if (terms == 1) return launch_fused_ts_t<1, false, true>(p, grid, s);
  } else if (a_mn && b_mn) {
    if (terms == 3) return launch_fused_ts_t<3, true, false>(p, grid, s);
    if (terms == 1) return launch_fused_ts_t<1, true, false>(p, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fmm
