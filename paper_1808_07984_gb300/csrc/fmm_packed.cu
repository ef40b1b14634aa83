// fmm_packed.cu -- single-CTA instantiations and the launcher of the tensor-core kernel over
// packed operand sums (the CTA-pair instantiations are in fmm_packed_pair.cu).
#include <cuda_runtime.h>
#include <algorithm>
#include "fmm_packed_launch.cuh"
#include "launch.h"

namespace fmm {

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
    if (tile_n == 128) return launch_cfg<128, 3, 6, true, A_MN, B_MN, 32, false>(p, grid, s);
    if (tile_n == 256) return launch_cfg<256, 3, 4, true, A_MN, B_MN, 32, false>(p, grid, s);
    return cudaErrorInvalidValue;
  }
  if (tile_n == 128) {
    if (terms == 3) return launch_cfg<128, 3, 3, true, A_MN, B_MN, 64, false>(p, grid, s);
    return bf16 ? launch_cfg<128, 1, 6, true, A_MN, B_MN, 64, false>(p, grid, s)
                : launch_cfg<128, 1, 6, false, A_MN, B_MN, 64, false>(p, grid, s);
  }
  if (tile_n == 256) {
    if (terms == 3) return launch_cfg<256, 3, 2, true, A_MN, B_MN, 64, false>(p, grid, s);
    return bf16 ? launch_cfg<256, 1, 4, true, A_MN, B_MN, 64, false>(p, grid, s)
                : launch_cfg<256, 1, 4, false, A_MN, B_MN, 64, false>(p, grid, s);
  }
  return cudaErrorInvalidValue;
}

// Single-CTA kernels are built for the forward layout (A K-major, B MN-major) that
// fmm_gemm_ex can select; the backward products (dA: A and B K-major, dB: both MN-major) and
// batched launches always run as CTA pairs.
cudaError_t launch_packed(const KernelArgs& p, int tile_n, int terms, bool bf16, bool a_mn, bool b_mn,
                          int bk, bool pair, int grid, cudaStream_t s) {
  if (pair) return launch_packed_pair(p, tile_n, terms, bf16, a_mn, b_mn, bk, grid, s);
  if (!a_mn && b_mn) return launch_mn<false, true>(p, tile_n, terms, bf16, bk, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace fmm
