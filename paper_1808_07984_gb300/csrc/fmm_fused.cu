// fmm_fused.cu -- instantiations and launcher of the fused (on-chip operand sums) kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include "fmm_fused.cuh"
#include "launch.h"

namespace fmm {

template <int TERMS, int TW>
static cudaError_t launch_fused_t(const FusedParams& p, int grid, cudaStream_t s) {
  using Cfg = FusedCfg<TERMS>;
  auto kern = fmm_fused_kernel<TERMS, TW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(Cfg::kSmemBytes));
  if (e != cudaSuccess) return e;
  kern<<<grid, fused_threads<TW>(), Cfg::kSmemBytes, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fused(const FusedParams& p, int terms, int transform_warps, int grid, cudaStream_t s) {
  if (transform_warps == 16) {
    if (terms == 3) return launch_fused_t<3, 16>(p, grid, s);
    if (terms == 1) return launch_fused_t<1, 16>(p, grid, s);
  } else if (transform_warps == 8) {
    if (terms == 3) return launch_fused_t<3, 8>(p, grid, s);
    if (terms == 1) return launch_fused_t<1, 8>(p, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fmm
