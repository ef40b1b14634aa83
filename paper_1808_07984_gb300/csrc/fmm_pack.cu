// fmm_pack.cu -- streaming passes around the tensor-core kernel:
//   * operand-sum pass: forms the 7^L signed sums of A-blocks (and of B-blocks,
//     transposed to K-major) in FP32 and stores them rounded to 16 bits, or split
//     into BF16 hi/lo halves (hi = bf16(P), lo = bf16(P - hi));
//   * beta pass: C = beta * C (beta == 0 writes zeros without reading C);
//   * a one-CTA kernel that exercises the bounded-wait failure path.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include "fmm_kernels.cuh"
#include "launch.h"

namespace fmm {

template <typename T>
__device__ __forceinline__ float load_as_float(const T* p);
template <>
__device__ __forceinline__ float load_as_float<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_as_float<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <>
__device__ __forceinline__ float load_as_float<__half>(const __half* p) { return __half2float(*p); }

// OUT16: 0 = bfloat16 output, 1 = float16 output
template <int OUT16>
__device__ __forceinline__ uint16_t round16(float x) {
  if (OUT16 == 0) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
  return __half_as_ushort(__float2half_rn(x));
}

// A-side: out[r][i][l] = sum_t sign_t * X[block(src_t) origin + (i, l)], i < hr, l < hc.
// Each thread handles 4 consecutive l of one row.
template <typename T, int OUT16, int NSRC>
__global__ void __launch_bounds__(256) pack_rows_kernel(const __grid_constant__ PackParams p) {
  const T* X = static_cast<const T*>(p.X);
  const int64_t quads_per_row = (p.hc + 3) / 4;  // a partial last quad writes into the row padding
  const int64_t total = static_cast<int64_t>(p.hr) * quads_per_row;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / quads_per_row;
    const int64_t l0 = (idx - i * quads_per_row) * 4;
    float v[NSRC][4];
#pragma unroll
    for (int s = 0; s < NSRC; ++s) {
      const int bi = s / p.gdim, bj = s - (s / p.gdim) * p.gdim;
      const int64_t gr = static_cast<int64_t>(bi) * p.hr + i;
      const int64_t gc = static_cast<int64_t>(bj) * p.hc + l0;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        v[s][e] = (gr < p.rows && gc + e < p.cols && l0 + e < p.hc)
                      ? load_as_float<T>(X + gr * p.ldx + gc + e)
                      : 0.f;
      }
    }
    for (int r = 0; r < p.nprod; ++r) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const int cnt = p.cnt[r];
      for (int t = 0; t < cnt; ++t) {
        const SrcTerm st = p.term[r][t];
#pragma unroll
        for (int s = 0; s < NSRC; ++s) {
          if (s == st.src) {
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[e] = st.sign > 0 ? acc[e] + v[s][e] : acc[e] - v[s][e];
          }
        }
      }
      const int64_t o = r * p.prod_stride + i * p.ld_out + l0;
      ushort4 hi, lo;
      if (p.terms == 3) {
        uint16_t h[4], w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const __nv_bfloat16 hb = __float2bfloat16_rn(acc[e]);
          h[e] = __bfloat16_as_ushort(hb);
          w[e] = __bfloat16_as_ushort(__float2bfloat16_rn(acc[e] - __bfloat162float(hb)));
        }
        hi = make_ushort4(h[0], h[1], h[2], h[3]);
        lo = make_ushort4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<ushort4*>(p.out_lo + o) = lo;
      } else {
        hi = make_ushort4(round16<OUT16>(acc[0]), round16<OUT16>(acc[1]), round16<OUT16>(acc[2]),
                          round16<OUT16>(acc[3]));
      }
      *reinterpret_cast<ushort4*>(p.out_hi + o) = hi;
    }
  }
}

// B-side, transposed: X is the (k x n) matrix B; out[r][j][l] = sum_t sign_t * X[origin + (l, j)]
// for j < hc (n direction) and l < hr (k direction), i.e. each operand sum is written K-major.
// A 32 x 32 (l, j) tile of every source block is staged in shared memory.
template <typename T, int OUT16, int NSRC>
__global__ void __launch_bounds__(256) pack_cols_kernel(const __grid_constant__ PackParams p) {
  extern __shared__ float tile[];  // [NSRC][32][33]
  const T* X = static_cast<const T*>(p.X);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  const int tiles_l = (p.hr + 31) / 32;
  const int tiles_j = (p.hc + 31) / 32;
  const int64_t ntiles = static_cast<int64_t>(tiles_l) * tiles_j;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int l0 = static_cast<int>(t / tiles_j) * 32;
    const int j0 = static_cast<int>(t % tiles_j) * 32;
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NSRC; ++s) {
      const int bi = s / p.gdim, bj = s - (s / p.gdim) * p.gdim;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int l = l0 + ty + 8 * u;
        const int j = j0 + tx;
        const int64_t gr = static_cast<int64_t>(bi) * p.hr + l;
        const int64_t gc = static_cast<int64_t>(bj) * p.hc + j;
        float x = 0.f;
        if (l < p.hr && j < p.hc && gr < p.rows && gc < p.cols) x = load_as_float<T>(X + gr * p.ldx + gc);
        tile[(s * 32 + ty + 8 * u) * 33 + tx] = x;
      }
    }
    __syncthreads();
    for (int r = 0; r < p.nprod; ++r) {
      const int cnt = p.cnt[r];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + ty + 8 * u;
        const int l = l0 + tx;
        float acc = 0.f;
        for (int t2 = 0; t2 < cnt; ++t2) {
          const SrcTerm st = p.term[r][t2];
          const float x = tile[(st.src * 32 + tx) * 33 + ty + 8 * u];
          acc = st.sign > 0 ? acc + x : acc - x;
        }
        if (j < p.hc && l < p.hr) {
          const int64_t o = r * p.prod_stride + static_cast<int64_t>(j) * p.ld_out + l;
          if (p.terms == 3) {
            const __nv_bfloat16 hb = __float2bfloat16_rn(acc);
            p.out_hi[o] = __bfloat16_as_ushort(hb);
            p.out_lo[o] = __bfloat16_as_ushort(__float2bfloat16_rn(acc - __bfloat162float(hb)));
          } else {
            p.out_hi[o] = round16<OUT16>(acc);
          }
        }
      }
    }
  }
}

__global__ void beta_kernel(float* C, int64_t m, int64_t n, int64_t ldc, float beta) {
  const int64_t total = m * n;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / n, j = idx - (idx / n) * n;
    float* c = C + i * ldc + j;
    *c = (beta == 0.f) ? 0.f : beta * *c;
  }
}

__global__ void debug_wait_kernel(unsigned* err, uint64_t timeout_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // nothing ever arrives: the wait must give up by itself
    if (!mbar_wait(smem_u32(&bar), 0, timeout_ns, &abort_flag)) atomicOr(err, kErrDebugWait);
  }
}

// ------------------------------------------------------------------ launchers
template <typename T, int OUT16>
static cudaError_t launch_pack_t(const PackParams& p, bool transpose, int num_sms, cudaStream_t s) {
  const int nsrc = p.nsrc;
  if (!transpose) {
    const int64_t total = static_cast<int64_t>(p.hr) * ((p.hc + 3) / 4);
    if (total == 0) return cudaSuccess;
    const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, int64_t(num_sms) * 8));
    switch (nsrc) {
      case 1: pack_rows_kernel<T, OUT16, 1><<<grid, 256, 0, s>>>(p); break;
      case 4: pack_rows_kernel<T, OUT16, 4><<<grid, 256, 0, s>>>(p); break;
      case 16: pack_rows_kernel<T, OUT16, 16><<<grid, 256, 0, s>>>(p); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    const int64_t ntiles = static_cast<int64_t>((p.hr + 31) / 32) * ((p.hc + 31) / 32);
    if (ntiles == 0) return cudaSuccess;
    const int grid = static_cast<int>(std::min<int64_t>(ntiles, int64_t(num_sms) * 4));
    const size_t smem = static_cast<size_t>(nsrc) * 32 * 33 * sizeof(float);
    switch (nsrc) {
      case 1: pack_cols_kernel<T, OUT16, 1><<<grid, 256, smem, s>>>(p); break;
      case 4: pack_cols_kernel<T, OUT16, 4><<<grid, 256, smem, s>>>(p); break;
      case 16: {
        cudaError_t e = cudaFuncSetAttribute(pack_cols_kernel<T, OUT16, 16>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        pack_cols_kernel<T, OUT16, 16><<<grid, 256, smem, s>>>(p);
        break;
      }
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_pack(const PackParams& p, int in_type, int out16, bool transpose, int num_sms,
                        cudaStream_t s) {
  if (in_type == kInF32) {
    return out16 ? launch_pack_t<float, 1>(p, transpose, num_sms, s)
                 : launch_pack_t<float, 0>(p, transpose, num_sms, s);
  }
  if (in_type == kInBF16) return launch_pack_t<__nv_bfloat16, 0>(p, transpose, num_sms, s);
  if (in_type == kInF16) return launch_pack_t<__half, 1>(p, transpose, num_sms, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_beta(float* C, int64_t m, int64_t n, int64_t ldc, float beta, int num_sms,
                        cudaStream_t s) {
  const int64_t total = m * n;
  if (total == 0) return cudaSuccess;
  const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, int64_t(num_sms) * 16));
  beta_kernel<<<grid, 256, 0, s>>>(C, m, n, ldc, beta);
  return cudaGetLastError();
}

cudaError_t launch_debug_wait(unsigned* err, uint64_t timeout_ns, cudaStream_t s) {
  debug_wait_kernel<<<1, 32, 0, s>>>(err, timeout_ns);
  return cudaGetLastError();
}

}  // namespace fmm
