// fmm_packed.cu -- instantiations and launcher of the tensor-core kernel over packed operand sums.
#include <cuda_runtime.h>
#include "fmm_kernels.cuh"
#include "launch.h"

namespace fmm {

template <int BN, int TERMS, int STAGES, bool BF16>
static cudaError_t launch_cfg(const PackedParams& p, int grid, cudaStream_t s) {
  using Cfg = PackedCfg<BN, TERMS, STAGES>;
  auto kern = fmm_packed_kernel<BN, TERMS, STAGES, BF16>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(Cfg::kSmemBytes));
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, Cfg::kSmemBytes, s>>>(p);
  return cudaGetLastError();
}

bool packed_config_supported(int tile_n, int terms, bool bf16) {
  if (tile_n != 128 && tile_n != 256) return false;
  if (terms != 1 && terms != 3) return false;
  if (terms == 3 && !bf16) return false;
  return true;
}

cudaError_t launch_packed(const PackedParams& p, int tile_n, int terms, bool bf16, int grid,
                          cudaStream_t s) {
  if (tile_n == 128) {
    if (terms == 3) return launch_cfg<128, 3, 3, true>(p, grid, s);
    return bf16 ? launch_cfg<128, 1, 6, true>(p, grid, s) : launch_cfg<128, 1, 6, false>(p, grid, s);
  }
  if (tile_n == 256) {
    if (terms == 3) return launch_cfg<256, 3, 2, true>(p, grid, s);
    return bf16 ? launch_cfg<256, 1, 4, true>(p, grid, s) : launch_cfg<256, 1, 4, false>(p, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fmm
