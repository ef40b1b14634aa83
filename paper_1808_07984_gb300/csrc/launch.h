// launch.h -- host-side launchers shared by the C-ABI translation unit.
#pragma once
#include <cuda_runtime.h>
#include <string>
#include "fmm_bases.h"
#include "fmm_kernels.cuh"

namespace fmm {

enum InType { kInF32 = 0, kInBF16 = 1, kInF16 = 2 };

// Sets the calling thread's message returned by fmm_last_error().
void set_last_error(const std::string& msg);

// Operand sums of all 7^levels products of A (is_b = false, coefficients U) or B (V).  With
// transq the stored source is the transpose of the operand, so block (i, j) of the source takes
// the coefficient of operand block (j, i) at every level.
cudaError_t launch_operand_sums(const SumParams& p, int levels, bool is_b, bool transq, int in_type,
                                int out16, int num_sms, cudaStream_t s);
// Panel maxima of the seven one-level operand sums of an FP32 matrix (A: panels of
// panel_w rows, B: of panel_w columns) into p.maxbits, without storing the sums: the scale
// pass of the hybrid scheme's FP16 bottom level.
cudaError_t launch_operand_maxima(const SumParams& p, bool is_b, int num_sms, cudaStream_t s);
// Panel maxima of the 7^levels operand sums of an FP16 operand (forward layout), without
// storing the sums: the scale pass of FP16 products whose sums are formed on chip.
cudaError_t launch_operand_maxima_f16(const SumParams& p, int levels, bool is_b, int num_sms, cudaStream_t s);
// Operand sums of every product of a basis table (see TableSumParams) for one operand.
cudaError_t launch_table_sums(const TableSumParams& tp, int in_type, int out16, int num_sms, cudaStream_t s);
cudaError_t launch_beta(float* C, int64_t m, int64_t n, int64_t ldc, float beta, int num_sms,
                        cudaStream_t s);
cudaError_t launch_debug_wait(unsigned* err, uint64_t timeout_ns, cudaStream_t s);
// Outside power-of-two scaling: float bits of max |x| of the rows of A (m x k) and of the
// columns of B (k x n); and C <- 2^(sign (e_row + e_col)) * beta * C.
cudaError_t launch_outer_maxbits(const void* A, int64_t m, int64_t k, int64_t lda, const void* B, int64_t n,
                                int64_t ldb, int in_type, unsigned* row_bits, unsigned* col_bits, int num_sms,
                                cudaStream_t s);
cudaError_t launch_outer_rescale(float* C, int64_t m, int64_t n, int64_t ldc, const unsigned* row_bits,
                                 const unsigned* col_bits, int sign, float beta, int num_sms, cudaStream_t s);

// Tensor-core kernel over packed operand sums.  tile_n in {128, 256}; terms in {1, 3};
// bf16 selects BF16 (true) or FP16 (false) operands; pair selects the CTA-pair kernel
// (256-row tiles, clusters of two CTAs, grid even; bk = 64 only).
cudaError_t launch_packed(const KernelArgs& p, int tile_n, int terms, bool bf16, bool a_mn, bool b_mn,
                          int bk, bool pair, int grid, cudaStream_t s);
cudaError_t launch_packed_pair(const KernelArgs& p, int tile_n, int terms, bool bf16, bool a_mn, bool b_mn,
                               int bk, int grid, cudaStream_t s);
bool packed_config_supported(int tile_n, int terms, bool bf16);

// Tensor-core kernel that forms the operand sums on chip from FP32 source tiles (tile
// 128 x 128, or 256 x 256 for a CTA pair; terms in {1, 3}).  transform_warps: warps that
// form the operand sums (8 built; 16 measured slower on GB300).
constexpr int kFusedTransformWarps = 8;
cudaError_t launch_fused(const FusedParams& p, int terms, int transform_warps, bool pair, int grid,
                         cudaStream_t s);
// The same products in CTA pairs with the A-operand sums held in tensor memory
// (fmm_fused_ts.cuh); terms in {1, 3}.  a_mn: A' stored by rows of k; b_mn: B' stored by
// rows of k (false: by rows of n).  Built: (a_mn, b_mn) = (0, 1), (0, 0), (1, 1).  f16: FP16
// UMMAs on panel-scaled sums (terms 1, forward; p.c.maxbits_a / maxbits_b set).  s16: the
// source maps are 16-bit (BF16, or FP16 with f16; A box 32 x 128 with 64-byte swizzle, B box
// 128 x 32; terms 1, forward).
cudaError_t launch_fused_ts(const FusedParams& p, int terms, bool a_mn, bool b_mn, bool f16, bool s16, int grid,
                            cudaStream_t s);

}  // namespace fmm
