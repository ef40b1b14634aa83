// fmm_packed_pair.cu -- CTA-pair instantiations of the packed tensor-core kernel: 256-row
// pair tiles, each CTA of a cluster of two holding 128 rows of A and half of B per stage.
#include <algorithm>
#include "fmm_packed_launch.cuh"
#include "launch.h"

namespace fmm {

// Stages per tile width and term count, filling the 192 KB left beside the epilogue staging:
// one stage holds (A 128 x 64 + B 64 x BN/2) BF16 per term.
template <bool A_MN, bool B_MN>
static cudaError_t launch_pair_mn(const KernelArgs& p, int tile_n, int terms, bool bf16, int grid,
                                  cudaStream_t s) {
  if (tile_n == 128) {
    if (terms == 3) return launch_cfg<128, 3, 4, true, A_MN, B_MN, 64, true>(p, grid, s);
    return bf16 ? launch_cfg<128, 1, 8, true, A_MN, B_MN, 64, true>(p, grid, s)
                : launch_cfg<128, 1, 8, false, A_MN, B_MN, 64, true>(p, grid, s);
  }
  if (tile_n == 256) {
    if (terms == 3) return launch_cfg<256, 3, 3, true, A_MN, B_MN, 64, true>(p, grid, s);
    return bf16 ? launch_cfg<256, 1, 6, true, A_MN, B_MN, 64, true>(p, grid, s)
                : launch_cfg<256, 1, 6, false, A_MN, B_MN, 64, true>(p, grid, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_packed_pair(const KernelArgs& p, int tile_n, int terms, bool bf16, bool a_mn, bool b_mn,
                               int bk, int grid, cudaStream_t s) {
  if (bk != 64) return cudaErrorInvalidValue;
  if (!a_mn && b_mn) return launch_pair_mn<false, true>(p, tile_n, terms, bf16, grid, s);
  if (!a_mn && !b_mn) return launch_pair_mn<false, false>(p, tile_n, terms, bf16, grid, s);
  if (a_mn && b_mn) return launch_pair_mn<true, true>(p, tile_n, terms, bf16, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace fmm
