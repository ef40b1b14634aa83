// fmm_packed.cu -- instantiations and launcher of the tensor-core kernel over packed operand sums.
#include <cuda_runtime.h>
#include "fmm_kernels.cuh"
#include "launch.h"

namespace fmm {

template <int BN, int TERMS, int STAGES, bool BF16, bool A_MN, bool B_MN, int BK = kBK>
static cudaError_t launch_cfg(const KernelArgs& p, int grid, cudaStream_t s) {
  using Cfg = PackedCfg<BN, TERMS, STAGES, BK>;
  auto kern = fmm_packed_kernel<BN, TERMS, STAGES, BF16, A_MN, B_MN, BK>;
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

template <bool A_MN, bool B_MN>
static cudaError_t launch_mn(const KernelArgs& p, int tile_n, int terms, bool bf16, int bk, int grid,
                             cudaStream_t s) {
  if (bk == 32) {
    // split3 only: 32-deep stages (64-byte swizzle) give 256-wide tiles four stages
    if (terms != 3) return cudaErrorInvalidValue;
    if (tile_n == 128) return launch_cfg<128, 3, 6, true, A_MN, B_MN, 32>(p, grid, s);
    if (tile_n == 256) return launch_cfg<256, 3, 4, true, A_MN, B_MN, 32>(p, grid, s);
    return cudaErrorInvalidValue;
  }
  if (tile_n == 128) {
    if (terms == 3) return launch_cfg<128, 3, 3, true, A_MN, B_MN>(p, grid, s);
    return bf16 ? launch_cfg<128, 1, 6, true, A_MN, B_MN>(p, grid, s)
                : launch_cfg<128, 1, 6, false, A_MN, B_MN>(p, grid, s);
  }
  if (tile_n == 256) {
    if (terms == 3) return launch_cfg<256, 3, 2, true, A_MN, B_MN>(p, grid, s);
    return bf16 ? launch_cfg<256, 1, 4, true, A_MN, B_MN>(p, grid, s)
                : launch_cfg<256, 1, 4, false, A_MN, B_MN>(p, grid, s);
  }
  return cudaErrorInvalidValue;
}

// Operand layouts built: forward (A K-major, B MN-major), dA = dC B^T (A K-major, B K-major),
// dB = A^T dC (A MN-major, B MN-major).
cudaError_t launch_packed(const KernelArgs& p, int tile_n, int terms, bool bf16, bool a_mn, bool b_mn,
                          int bk, int grid, cudaStream_t s) {
  if (!a_mn && b_mn) return launch_mn<false, true>(p, tile_n, terms, bf16, bk, grid, s);
  if (!a_mn && !b_mn) return launch_mn<false, false>(p, tile_n, terms, bf16, bk, grid, s);
  if (a_mn && b_mn) return launch_mn<true, true>(p, tile_n, terms, bf16, bk, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace fmm
