// fmm_fused.cu -- instantiations and launcher of the fused (on-chip operand sums) kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include "fmm_fused.cuh"
#include "launch.h"

namespace fmm {

template <int TERMS>
static cudaError_t launch_fused_t(const FusedParams& p, int grid, cudaStream_t s) {
  using Cfg = FusedCfg<TERMS>;
  auto kern = fmm_fused_kernel<TERMS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(Cfg::kSmemBytes));
  if (e != cudaSuccess) return e;
  kern<<<grid, kFusedThreads, Cfg::kSmemBytes, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fused(const FusedParams& p, int terms, int grid, cudaStream_t s) {
  if (terms == 3) return launch_fused_t<3>(p, grid, s);
  if (terms == 1) return launch_fused_t<1>(p, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace fmm
