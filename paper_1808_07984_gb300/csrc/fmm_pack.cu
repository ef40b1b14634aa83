// fmm_pack.cu -- streaming passes around the tensor-core kernel:
//   * operand-sum pass: forms the 7^L signed sums of A-blocks (or B-blocks) in FP32 and
//     stores them, in the source's own row-major layout, rounded to 16 bits or split into
//     BF16 hi/lo halves (hi = bf16(P), lo = bf16(P - hi));
//   * beta pass: C = beta * C (beta == 0 writes zeros without reading C);
//   * a one-CTA kernel that exercises the bounded-wait failure path.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstring>
#include "fmm_bases.h"
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

// Operand sums of all 7^L products of one operand, row-major in and row-major out.
//   X is (rows x cols), viewed as a 2^L x 2^L grid of hr x hc blocks (zero outside X);
//   out[r][i][l] = sum_q coef(r, q) * X_q[i, l] for i < hr, l < hc, in FP32, then either
//   rounded once to 16 bits or split into hi = bf16(P), lo = bf16(P - hi).
// coef is strassen_u for A and strassen_v for B (Eq. 3); for two levels the product
// (r1, r2) takes block (q1, q2) with coefficient coef(r1, q1) * coef(r2, q2) and the sum is
// formed as sum_q2 coef(r2, q2) * (sum_q1 coef(r1, q1) * X_(q1, q2)).
// Each thread handles EPT consecutive columns of one row.
template <bool IS_B, bool TRANSQ>
__device__ __forceinline__ constexpr int coef(int r, int q) {
  // TRANSQ: the source is stored transposed, so its quadrant (i, j) is operand quadrant (j, i)
  const int qq = TRANSQ ? 2 * (q % 2) + q / 2 : q;
  return IS_B ? strassen_v(r, qq) : strassen_u(r, qq);
}

template <int TERMS, int OUT16, int EPT>
__device__ __forceinline__ void store_sum(const SumParams& p, int64_t o, const float (&acc)[EPT]) {
  if (TERMS == 0) {
#pragma unroll
    for (int e = 0; e < EPT; e += 4)
      *reinterpret_cast<float4*>(p.out_f32 + o + e) = make_float4(acc[e], acc[e + 1], acc[e + 2], acc[e + 3]);
  } else if (TERMS == 3) {
    uint16_t h[EPT], w[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const __nv_bfloat16 hb = __float2bfloat16_rn(acc[e]);
      h[e] = __bfloat16_as_ushort(hb);
      w[e] = __bfloat16_as_ushort(__float2bfloat16_rn(acc[e] - __bfloat162float(hb)));
    }
    if (EPT == 8) {
      *reinterpret_cast<uint4*>(p.out_hi + o) =
          make_uint4(h[0] | (uint32_t(h[1]) << 16), h[2] | (uint32_t(h[3]) << 16),
                     h[4] | (uint32_t(h[5]) << 16), h[6] | (uint32_t(h[7]) << 16));
      *reinterpret_cast<uint4*>(p.out_lo + o) =
          make_uint4(w[0] | (uint32_t(w[1]) << 16), w[2] | (uint32_t(w[3]) << 16),
                     w[4] | (uint32_t(w[5]) << 16), w[6] | (uint32_t(w[7]) << 16));
    } else {
      *reinterpret_cast<uint2*>(p.out_hi + o) =
          make_uint2(h[0] | (uint32_t(h[1]) << 16), h[2] | (uint32_t(h[3]) << 16));
      *reinterpret_cast<uint2*>(p.out_lo + o) =
          make_uint2(w[0] | (uint32_t(w[1]) << 16), w[2] | (uint32_t(w[3]) << 16));
    }
  } else {
    uint16_t h[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) h[e] = round16<OUT16>(acc[e]);
    if (EPT == 8) {
      *reinterpret_cast<uint4*>(p.out_hi + o) =
          make_uint4(h[0] | (uint32_t(h[1]) << 16), h[2] | (uint32_t(h[3]) << 16),
                     h[4] | (uint32_t(h[5]) << 16), h[6] | (uint32_t(h[7]) << 16));
    } else {
      *reinterpret_cast<uint2*>(p.out_hi + o) =
          make_uint2(h[0] | (uint32_t(h[1]) << 16), h[2] | (uint32_t(h[3]) << 16));
    }
  }
}

// Hand one group of EPT sums of product r to its destination: store it (SCALE 0), fold its
// largest magnitude into the panel maximum (SCALE 1), or store it scaled by 2^-s (SCALE 2).
template <int SCALE, int TERMS, int OUT16, int EPT>
__device__ __forceinline__ void emit(const SumParams& p, int r, int64_t i, int64_t l0, int64_t o,
                                     float (&acc)[EPT]) {
  if (SCALE == 0) {
    store_sum<TERMS, OUT16, EPT>(p, o, acc);
    return;
  }
  const int panel = static_cast<int>((p.scale_rows ? i : l0) / p.panel_w);
  if (SCALE == 1) {
    float mx = 0.f;
#pragma unroll
    for (int e = 0; e < EPT; ++e) mx = fmaxf(mx, fabsf(acc[e]));
    const unsigned bits = __float_as_uint(mx);
    const unsigned active = __activemask();
    const unsigned same = __match_any_sync(active, panel);
    const unsigned red = __reduce_max_sync(same, bits);
    if ((threadIdx.x & 31) == __ffs(same) - 1) atomicMax(&p.maxbits[r * p.npanels + panel], red);
    return;
  }
  const int sft = panel_shift(p.maxbits[r * p.npanels + panel]);
#pragma unroll
  for (int e = 0; e < EPT; ++e) acc[e] = ldexpf(acc[e], -sft);
  store_sum<TERMS, OUT16, EPT>(p, o, acc);
}

// 2^-e for an exponent of outer_exp (e in [-126, 127]), built from its bits: a normal float
// for e <= 126 and the subnormal 2^-127 for e = 127.  Multiplying by it rounds once, exactly
// as scaling by ldexp does.
__device__ __forceinline__ float pow2_inverse(int e) {
  return e <= 126 ? __int_as_float((127 - e) << 23) : __int_as_float(0x00400000);
}

template <typename T, int EPT>
__device__ __forceinline__ void load_group(const SumParams& p, const T* X, int64_t gr, int64_t gc,
                                           int64_t l0, float (&v)[EPT]) {
  const bool row_ok = gr < p.rows;
  if (row_ok && p.vec_ok && gc + EPT <= p.cols && l0 + EPT <= p.hc) {
    const T* src = X + gr * p.ldx + gc;
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int e = 0; e < EPT; e += 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(src + e));
        v[e] = q.x; v[e + 1] = q.y; v[e + 2] = q.z; v[e + 3] = q.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < EPT; e += 4) {
        const uint2 q = __ldg(reinterpret_cast<const uint2*>(src + e));
        T t[4];
        memcpy(t, &q, sizeof q);
#pragma unroll
        for (int u = 0; u < 4; ++u) v[e + u] = load_as_float<T>(&t[u]);
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      v[e] = (row_ok && gc + e < p.cols && l0 + e < p.hc) ? load_as_float<T>(X + gr * p.ldx + gc + e) : 0.f;
  }
  if (p.row_maxbits && row_ok) {  // outside scaling: exact powers of two
    const float f = pow2_inverse(outer_exp(p.row_maxbits[gr]));
#pragma unroll
    for (int e = 0; e < EPT; ++e) v[e] *= f;
  }
  if (p.col_maxbits) {
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      if (gc + e < p.cols) v[e] *= pow2_inverse(outer_exp(p.col_maxbits[gc + e]));
  }
}

template <typename T, int OUT16, int L, bool IS_B, bool TRANSQ, int TERMS, int EPT, int SCALE>
__global__ void __launch_bounds__(256) operand_sums_kernel(const __grid_constant__ SumParams p) {
  const T* X = static_cast<const T*>(p.X);
  const int64_t groups = (p.hc + EPT - 1) / EPT;
  const int64_t total = p.hr * groups;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / groups;
    const int64_t l0 = (idx - i * groups) * EPT;
    const int64_t orow = i * p.ld_out + l0;
    if (L == 0) {
      float v[EPT];
      load_group<T, EPT>(p, X, i, l0, l0, v);
      emit<SCALE, TERMS, OUT16, EPT>(p, 0, i, l0, orow, v);
    } else if (p.chunk >= 0) {
      // one top-level product: read only the quadrants it combines
      float S[L == 1 ? 1 : 4][EPT];
#pragma unroll
      for (int q2 = 0; q2 < (L == 1 ? 1 : 4); ++q2)
#pragma unroll
        for (int e = 0; e < EPT; ++e) S[q2][e] = 0.f;
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1) {
        const int c = p.c1[q1];
        if (c == 0) continue;
#pragma unroll
        for (int q2 = 0; q2 < (L == 1 ? 1 : 4); ++q2) {
          float v[EPT];
          if (L == 1) {
            load_group<T, EPT>(p, X, (q1 / 2) * p.hr + i, (q1 % 2) * p.hc + l0, l0, v);
          } else {
            const int bi = 2 * (q1 / 2) + q2 / 2, bj = 2 * (q1 % 2) + q2 % 2;
            load_group<T, EPT>(p, X, bi * p.hr + i, bj * p.hc + l0, l0, v);
          }
#pragma unroll
          for (int e = 0; e < EPT; ++e) S[q2][e] = c > 0 ? S[q2][e] + v[e] : S[q2][e] - v[e];
        }
      }
      if (L == 1) {
        emit<SCALE, TERMS, OUT16, EPT>(p, p.chunk, i, l0, p.chunk * p.prod_stride + orow, S[0]);
      } else {
#pragma unroll
        for (int r2 = 0; r2 < 7; ++r2) {
          float acc[EPT];
#pragma unroll
          for (int e = 0; e < EPT; ++e) acc[e] = 0.f;
#pragma unroll
          for (int q2 = 0; q2 < 4; ++q2) {
            const int c = coef<IS_B, TRANSQ>(r2, q2);
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
              if (c > 0) acc[e] += S[q2 < (L == 1 ? 1 : 4) ? q2 : 0][e];
              if (c < 0) acc[e] -= S[q2 < (L == 1 ? 1 : 4) ? q2 : 0][e];
            }
          }
          const int r = p.chunk * 7 + r2;
          emit<SCALE, TERMS, OUT16, EPT>(p, r, i, l0, r * p.prod_stride + orow, acc);
        }
      }
    } else if (L == 1) {
      float v[4][EPT];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        load_group<T, EPT>(p, X, (q / 2) * p.hr + i, (q % 2) * p.hc + l0, l0, v[q]);
#pragma unroll
      for (int r = 0; r < 7; ++r) {
        float acc[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) acc[e] = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = coef<IS_B, TRANSQ>(r, q);
#pragma unroll
          for (int e = 0; e < EPT; ++e) {
            if (c > 0) acc[e] += v[q][e];
            if (c < 0) acc[e] -= v[q][e];
          }
        }
        emit<SCALE, TERMS, OUT16, EPT>(p, r, i, l0, r * p.prod_stride + orow, acc);
      }
    } else {
      // source (q1, q2) is block (2*(q1/2) + q2/2, 2*(q1%2) + q2%2) of the 4 x 4 grid
      float v[16][EPT];
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
          const int bi = 2 * (q1 / 2) + q2 / 2, bj = 2 * (q1 % 2) + q2 % 2;
          load_group<T, EPT>(p, X, bi * p.hr + i, bj * p.hc + l0, l0, v[q1 * 4 + q2]);
        }
#pragma unroll
      for (int r1 = 0; r1 < 7; ++r1) {
        float S[4][EPT];
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
#pragma unroll
          for (int e = 0; e < EPT; ++e) S[q2][e] = 0.f;
#pragma unroll
          for (int q1 = 0; q1 < 4; ++q1) {
            const int c = coef<IS_B, TRANSQ>(r1, q1);
#pragma unroll
            for (int e = 0; e < EPT; ++e) S[q2][e] = c > 0 ? S[q2][e] + v[q1 * 4 + q2][e]
                                                   : (c < 0 ? S[q2][e] - v[q1 * 4 + q2][e] : S[q2][e]);
          }
        }
#pragma unroll
        for (int r2 = 0; r2 < 7; ++r2) {
          float acc[EPT];
#pragma unroll
          for (int e = 0; e < EPT; ++e) acc[e] = 0.f;
#pragma unroll
          for (int q2 = 0; q2 < 4; ++q2) {
            const int c = coef<IS_B, TRANSQ>(r2, q2);
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
              if (c > 0) acc[e] += S[q2][e];
              if (c < 0) acc[e] -= S[q2][e];
            }
          }
          emit<SCALE, TERMS, OUT16, EPT>(p, r1 * 7 + r2, i, l0, (r1 * 7 + r2) * p.prod_stride + orow, acc);
        }
      }
    }
  }
}

// Operand sums of a basis given as a table (TableSumParams): each thread loads EPT
// consecutive columns of one row position from every stored block, then forms each
// product's signed sum in FP32 (blocks in ascending order) and hands it to emit().
template <typename T, int OUT16, int NB, int TERMS, int EPT, int SCALE>
__global__ void __launch_bounds__(256) table_sums_kernel(const __grid_constant__ TableSumParams tp) {
  const SumParams& p = tp.p;
  const T* X = static_cast<const T*>(p.X);
  const int64_t groups = (p.hc + EPT - 1) / EPT;
  const int64_t total = p.hr * groups;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / groups;
    const int64_t l0 = (idx - i * groups) * EPT;
    const int64_t orow = i * p.ld_out + l0;
    float v[NB][EPT];
#pragma unroll
    for (int sb = 0; sb < NB; ++sb)
      load_group<T, EPT>(p, X, (sb / tp.grid_c) * p.hr + i, (sb % tp.grid_c) * p.hc + l0, l0, v[sb]);
    for (int r = 0; r < tp.nprod; ++r) {
      float acc[EPT];
#pragma unroll
      for (int e = 0; e < EPT; ++e) acc[e] = 0.f;
#pragma unroll
      for (int sb = 0; sb < NB; ++sb) {
        const int c = tp.coef[sb][r];
        if (c > 0) {
#pragma unroll
          for (int e = 0; e < EPT; ++e) acc[e] += v[sb][e];
        } else if (c < 0) {
#pragma unroll
          for (int e = 0; e < EPT; ++e) acc[e] -= v[sb][e];
        }
      }
      emit<SCALE, TERMS, OUT16, EPT>(p, r, i, l0, r * p.prod_stride + orow, acc);
    }
  }
}

// Outside scaling: float bits of max |x| of every row of X (rows x cols, leading dimension
// ld), one block per row.
template <typename T>
__global__ void row_maxbits_kernel(const T* X, int64_t rows, int64_t cols, int64_t ld, unsigned int* out) {
  __shared__ float red[8];
  for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
    float mx = 0.f;
    for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) mx = fmaxf(mx, fabsf(load_as_float<T>(X + i * ld + j)));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
      out[i] = __float_as_uint(mx);
    }
    __syncthreads();
  }
}

// Float bits of max |x| of every column of X: thread per column over a chunk of rows,
// combined by atomicMax (non-negative floats order like their bit patterns).
template <typename T>
__global__ void col_maxbits_kernel(const T* X, int64_t rows, int64_t cols, int64_t ld, int64_t rows_per_chunk,
                                   unsigned int* out) {
  const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (j >= cols) return;
  const int64_t r0 = blockIdx.y * rows_per_chunk, r1 = min(rows, r0 + rows_per_chunk);
  float mx = 0.f;
  for (int64_t i = r0; i < r1; ++i) mx = fmaxf(mx, fabsf(load_as_float<T>(X + i * ld + j)));
  if (mx > 0.f) atomicMax(out + j, __float_as_uint(mx));
}

// C[i][j] *= 2^(sign * (e_row(i) + e_col(j))) (sign -1 scales beta * C into the scaled
// problem before the products, +1 takes the result back out of it).
// One row per blockIdx.y step; 4 consecutive columns per thread (vector access when the rows
// are 16-byte aligned).
__global__ void outer_rescale_kernel(float* C, int64_t m, int64_t n, int64_t ldc, const unsigned int* row_maxbits,
                                     const unsigned int* col_maxbits, int sign, float beta, int vec4) {
  for (int64_t i = blockIdx.y; i < m; i += gridDim.y) {
    const int er = outer_exp(row_maxbits[i]);
    float* row = C + i * ldc;
    for (int64_t j = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) * 4; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x * 4) {
      if (vec4 && j + 4 <= n) {
        float4 v = *reinterpret_cast<float4*>(row + j);
        const uint4 cb = *reinterpret_cast<const uint4*>(col_maxbits + j);
        v.x = ldexpf(beta * v.x, sign * (er + outer_exp(cb.x)));
        v.y = ldexpf(beta * v.y, sign * (er + outer_exp(cb.y)));
        v.z = ldexpf(beta * v.z, sign * (er + outer_exp(cb.z)));
        v.w = ldexpf(beta * v.w, sign * (er + outer_exp(cb.w)));
        *reinterpret_cast<float4*>(row + j) = v;
      } else {
        for (int64_t jj = j; jj < min(n, j + 4); ++jj)
          row[jj] = ldexpf(beta * row[jj], sign * (er + outer_exp(col_maxbits[jj])));
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
template <typename T, int OUT16, int L, bool IS_B, bool TQ, int TERMS, int SCALE = 0>
static cudaError_t launch_sums_t(const SumParams& p, int num_sms, cudaStream_t s) {
  constexpr int EPT = L == 2 ? 4 : 8;
  const int64_t total = p.hr * ((p.hc + EPT - 1) / EPT);
  if (total == 0) return cudaSuccess;
  const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, int64_t(num_sms) * 16));
  operand_sums_kernel<T, OUT16, L, IS_B, TQ, TERMS, EPT, SCALE><<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename T, int OUT16, bool IS_B, bool TQ, int TERMS, int SCALE = 0>
static cudaError_t launch_sums_l(const SumParams& p, int levels, int num_sms, cudaStream_t s) {
  switch (levels) {
    case 0: return launch_sums_t<T, OUT16, 0, IS_B, TQ, TERMS, SCALE>(p, num_sms, s);
    case 1: return launch_sums_t<T, OUT16, 1, IS_B, TQ, TERMS, SCALE>(p, num_sms, s);
    case 2: return launch_sums_t<T, OUT16, 2, IS_B, TQ, TERMS, SCALE>(p, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

template <bool IS_B, bool TQ>
static cudaError_t launch_sums_b(const SumParams& p, int levels, int in_type, int out16, int num_sms,
                                 cudaStream_t s) {
  if (in_type == kInF32) {
    if (p.terms == 3) return launch_sums_l<float, 0, IS_B, TQ, 3>(p, levels, num_sms, s);
    if (p.terms == 0) return levels == 1 ? launch_sums_t<float, 0, 1, IS_B, TQ, 0>(p, num_sms, s)
                                         : cudaErrorInvalidValue;
    return out16 ? launch_sums_l<float, 1, IS_B, TQ, 1>(p, levels, num_sms, s)
                 : launch_sums_l<float, 0, IS_B, TQ, 1>(p, levels, num_sms, s);
  }
  if (in_type == kInBF16 && p.terms == 1 && !out16)
    return launch_sums_l<__nv_bfloat16, 0, IS_B, TQ, 1>(p, levels, num_sms, s);
  // FP32 sums of 16-bit operands (top level of the hybrid scheme)
  if (in_type == kInBF16 && p.terms == 0)
    return levels == 1 ? launch_sums_t<__nv_bfloat16, 0, 1, IS_B, TQ, 0>(p, num_sms, s) : cudaErrorInvalidValue;
  if (in_type == kInF16 && p.terms == 0)
    return levels == 1 ? launch_sums_t<__half, 0, 1, IS_B, TQ, 0>(p, num_sms, s) : cudaErrorInvalidValue;
  if (in_type == kInF16 && p.terms == 1 && out16) {
    if (!p.maxbits) return launch_sums_l<__half, 1, IS_B, TQ, 1>(p, levels, num_sms, s);
    // two passes: panel maxima, then the sums scaled by 2^-s (maxbits zeroed by the caller)
    cudaError_t e = launch_sums_l<__half, 1, IS_B, TQ, 1, 1>(p, levels, num_sms, s);
    if (e != cudaSuccess) return e;
    return launch_sums_l<__half, 1, IS_B, TQ, 1, 2>(p, levels, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int OUT16, int NB, int TERMS, int SCALE = 0>
static cudaError_t launch_table_t(const TableSumParams& tp, int num_sms, cudaStream_t s) {
  constexpr int EPT = NB <= 6 ? 8 : 4;
  const int64_t total = tp.p.hr * ((tp.p.hc + EPT - 1) / EPT);
  if (total == 0 || tp.nprod == 0) return cudaSuccess;
  const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, int64_t(num_sms) * 16));
  table_sums_kernel<T, OUT16, NB, TERMS, EPT, SCALE><<<grid, 256, 0, s>>>(tp);
  return cudaGetLastError();
}

template <typename T, int OUT16, int TERMS, int SCALE = 0>
static cudaError_t launch_table_nb(const TableSumParams& tp, int num_sms, cudaStream_t s) {
  switch (tp.grid_r * tp.grid_c) {
    case 4: return launch_table_t<T, OUT16, 4, TERMS, SCALE>(tp, num_sms, s);
    case 6: return launch_table_t<T, OUT16, 6, TERMS, SCALE>(tp, num_sms, s);
    case 9: return launch_table_t<T, OUT16, 9, TERMS, SCALE>(tp, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_table_sums(const TableSumParams& tp, int in_type, int out16, int num_sms, cudaStream_t s) {
  if (tp.nprod < 0 || tp.nprod > kMaxTableRank) return cudaErrorInvalidValue;
  const SumParams& p = tp.p;
  if (in_type == kInF32) {
    if (p.terms == 3) return launch_table_nb<float, 0, 3>(tp, num_sms, s);
    if (p.terms == 1)
      return out16 ? launch_table_nb<float, 1, 1>(tp, num_sms, s) : launch_table_nb<float, 0, 1>(tp, num_sms, s);
    return cudaErrorInvalidValue;
  }
  if (in_type == kInBF16 && p.terms == 1 && !out16) return launch_table_nb<__nv_bfloat16, 0, 1>(tp, num_sms, s);
  if (in_type == kInF16 && p.terms == 1 && out16) {
    if (!p.maxbits) return launch_table_nb<__half, 1, 1>(tp, num_sms, s);
    // two passes: panel maxima, then the sums scaled by 2^-s (maxbits zeroed by the caller)
    cudaError_t e = launch_table_nb<__half, 1, 1, 1>(tp, num_sms, s);
    if (e != cudaSuccess) return e;
    return launch_table_nb<__half, 1, 1, 2>(tp, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_operand_sums(const SumParams& p, int levels, bool is_b, bool transq, int in_type,
                                int out16, int num_sms, cudaStream_t s) {
  if (is_b) {
    return transq ? launch_sums_b<true, true>(p, levels, in_type, out16, num_sms, s)
                  : launch_sums_b<true, false>(p, levels, in_type, out16, num_sms, s);
  }
  return transq ? launch_sums_b<false, true>(p, levels, in_type, out16, num_sms, s)
                : launch_sums_b<false, false>(p, levels, in_type, out16, num_sms, s);
}

cudaError_t launch_operand_maxima(const SumParams& p, bool is_b, int num_sms, cudaStream_t s) {
  // one level of sums of an FP32 matrix, only their panel maxima (maxbits zeroed by the caller)
  return is_b ? launch_sums_t<float, 1, 1, true, false, 1, 1>(p, num_sms, s)
              : launch_sums_t<float, 1, 1, false, false, 1, 1>(p, num_sms, s);
}

cudaError_t launch_operand_maxima_f16(const SumParams& p, int levels, bool is_b, int num_sms, cudaStream_t s) {
  // SCALE 1: only the panel maxima (maxbits zeroed by the caller)
  return is_b ? launch_sums_l<__half, 1, true, false, 1, 1>(p, levels, num_sms, s)
              : launch_sums_l<__half, 1, false, false, 1, 1>(p, levels, num_sms, s);
}

cudaError_t launch_beta(float* C, int64_t m, int64_t n, int64_t ldc, float beta, int num_sms,
                        cudaStream_t s) {
  const int64_t total = m * n;
  if (total == 0) return cudaSuccess;
  if (beta == 0.f && ldc == n) return cudaMemsetAsync(C, 0, static_cast<size_t>(total) * sizeof(float), s);
  const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, int64_t(num_sms) * 16));
  beta_kernel<<<grid, 256, 0, s>>>(C, m, n, ldc, beta);
  return cudaGetLastError();
}

cudaError_t launch_outer_maxbits(const void* A, int64_t m, int64_t k, int64_t lda, const void* B, int64_t n,
                                int64_t ldb, int in_type, unsigned* row_bits, unsigned* col_bits, int num_sms,
                                cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(col_bits, 0, static_cast<size_t>(n) * 4, s);
  if (e != cudaSuccess) return e;
  const int rgrid = static_cast<int>(std::min<int64_t>(m, int64_t(num_sms) * 32));
  const int64_t chunk = 256;
  const dim3 cgrid(static_cast<unsigned>((n + 255) / 256), static_cast<unsigned>((k + chunk - 1) / chunk));
  if (in_type == kInF32) {
    row_maxbits_kernel<float><<<rgrid, 256, 0, s>>>(static_cast<const float*>(A), m, k, lda, row_bits);
    col_maxbits_kernel<float><<<cgrid, 256, 0, s>>>(static_cast<const float*>(B), k, n, ldb, chunk, col_bits);
  } else if (in_type == kInBF16) {
    row_maxbits_kernel<__nv_bfloat16><<<rgrid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(A), m, k, lda, row_bits);
    col_maxbits_kernel<__nv_bfloat16><<<cgrid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(B), k, n, ldb, chunk,
                                                             col_bits);
  } else {
    row_maxbits_kernel<__half><<<rgrid, 256, 0, s>>>(static_cast<const __half*>(A), m, k, lda, row_bits);
    col_maxbits_kernel<__half><<<cgrid, 256, 0, s>>>(static_cast<const __half*>(B), k, n, ldb, chunk, col_bits);
  }
  return cudaGetLastError();
}

cudaError_t launch_outer_rescale(float* C, int64_t m, int64_t n, int64_t ldc, const unsigned* row_bits,
                                 const unsigned* col_bits, int sign, float beta, int num_sms, cudaStream_t s) {
  if (m == 0 || n == 0) return cudaSuccess;
  // column bits start 256-byte aligned in the workspace; C rows need 16-byte alignment
  const int vec4 = (reinterpret_cast<uintptr_t>(C) % 16 == 0 && ldc % 4 == 0 &&
                    reinterpret_cast<uintptr_t>(col_bits) % 16 == 0) ? 1 : 0;
  const int64_t col_threads = (n + 3) / 4;
  const dim3 grid(static_cast<unsigned>(std::min<int64_t>((col_threads + 255) / 256, 64)),
                  static_cast<unsigned>(std::min<int64_t>(m, 65535)));
  outer_rescale_kernel<<<grid, 256, 0, s>>>(C, m, n, ldc, row_bits, col_bits, sign, beta, vec4);
  return cudaGetLastError();
}

cudaError_t launch_debug_wait(unsigned* err, uint64_t timeout_ns, cudaStream_t s) {
  debug_wait_kernel<<<1, 32, 0, s>>>(err, timeout_ns);
  return cudaGetLastError();
}

}  // namespace fmm
