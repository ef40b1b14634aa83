// fmm_packed_launch.cuh -- launch of one instantiation of the packed tensor-core kernel
// (shared by the single-CTA and the CTA-pair translation units).
#pragma once
#include <cuda_runtime.h>
#include "fmm_kernels.cuh"

namespace fmm {

// Largest grid (in CTAs) of `kern` that runs in one wave: CTA pairs are clusters of two, and
// how many of them fit at once depends on how the SMs are grouped, so ask the runtime.
template <class Kern>
static int pair_wave_ctas(Kern kern, uint32_t smem_bytes, int requested) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(requested), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem_bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return requested;
  }
  return std::min(requested, 2 * clusters);
}

template <int BN, int TERMS, int STAGES, bool BF16, bool A_MN, bool B_MN, int BK, bool PAIR>
static cudaError_t launch_cfg(const KernelArgs& p, int grid, cudaStream_t s) {
  using Cfg = PackedCfg<BN, TERMS, STAGES, BK, PAIR>;
  static_assert(Cfg::kSmemBytes <= 232448, "shared memory per CTA");
  auto kern = fmm_packed_kernel<BN, TERMS, STAGES, BF16, A_MN, B_MN, BK, PAIR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(Cfg::kSmemBytes));
  if (e != cudaSuccess) return e;
  if (!PAIR) {
    kern<<<grid, kThreads, Cfg::kSmemBytes, s>>>(p);
    return cudaGetLastError();
  }
  if (grid < 2 || grid % 2 != 0) return cudaErrorInvalidValue;
  grid = pair_wave_ctas(kern, Cfg::kSmemBytes, grid);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = Cfg::kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p);
}

}  // namespace fmm
