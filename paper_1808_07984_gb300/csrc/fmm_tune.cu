// fmm_tune.cu -- native autotuner: measures the (levels, tile width) candidates of square
// products through the library's own entry point and turns the fastest per probe size into
// the size classes of an fmm_tune_table.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "fmm.h"
#include "launch.h"

namespace fmm {
namespace {

// Deterministic values in [-1, 1) for timing inputs (a 32-bit integer mix of the index; the
// values only need to be non-trivial, not random in any statistical sense).
__global__ void fill_timing_input(void* X, int64_t n, int type, uint32_t seed) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    uint32_t h = static_cast<uint32_t>(i) * 0x9E3779B1u ^ seed ^ static_cast<uint32_t>(i >> 32);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    const float v = static_cast<float>(h >> 8) * (2.0f / 16777216.0f) - 1.0f;
    if (type == kInF32)
      static_cast<float*>(X)[i] = v;
    else if (type == kInBF16)
      static_cast<__nv_bfloat16*>(X)[i] = __float2bfloat16_rn(v);
    else
      static_cast<__half*>(X)[i] = __float2half_rn(v);
  }
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" fmm_status fmm_tune_measure(int variant, const int64_t* sizes, int count, int reps,
                                       fmm_tune_table* out, float* times_ms, void* stream) {
  if (!sizes || count < 1 || count > 8 || !out || reps < 1) {
    set_last_error("fmm_tune_measure: sizes, 1..8 probe sizes, reps >= 1 and out are required");
    return FMM_ERR_ARG;
  }
  for (int i = 0; i < count; ++i)
    if (sizes[i] < 1 || (i > 0 && sizes[i] <= sizes[i - 1])) {
      set_last_error("fmm_tune_measure: probe sizes must be positive and increasing");
      return FMM_ERR_ARG;
    }
  int in_type;
  switch (variant) {
    case FMM_F32_SPLIT3_BF16:
    case FMM_F32_PLAIN_BF16: in_type = kInF32; break;
    case FMM_BF16: in_type = kInBF16; break;
    case FMM_F16_SCALED: in_type = kInF16; break;
    default: set_last_error("fmm_tune_measure: variant not built"); return FMM_ERR_UNSUPPORTED;
  }
  const size_t eb = in_type == kInF32 ? 4 : 2;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int tiles[2] = {128, 256};
  int best_l[8], best_t[8];
  for (int i = 0; i < count; ++i) {
    const int64_t d = sizes[i];
    size_t ws = 0;
    for (int L = 0; L < 3; ++L)
      for (int t : tiles) {
        fmm_options o = {};
        o.tile_n = t;
        const size_t w = fmm_workspace_size_ex(d, d, d, L, variant, &o);
        if (w == static_cast<size_t>(-1)) {
          set_last_error("fmm_tune_measure: unsupported probe");
          return FMM_ERR_UNSUPPORTED;
        }
        ws = std::max(ws, w);
      }
    DevBuf A, B, C, W;
    cudaError_t e = cudaMalloc(&A.p, static_cast<size_t>(d * d) * eb);
    if (e == cudaSuccess) e = cudaMalloc(&B.p, static_cast<size_t>(d * d) * eb);
    if (e == cudaSuccess) e = cudaMalloc(&C.p, static_cast<size_t>(d * d) * 4);
    if (e == cudaSuccess && ws > 0) e = cudaMalloc(&W.p, ws);
    if (e != cudaSuccess) {
      set_last_error(std::string("fmm_tune_measure: cudaMalloc failed: ") + cudaGetErrorString(e));
      return FMM_ERR_CUDA;
    }
    const int grid = static_cast<int>(std::min<int64_t>((d * d + 255) / 256, 4096));
    fill_timing_input<<<grid, 256, 0, s>>>(A.p, d * d, in_type, 17u + static_cast<uint32_t>(i));
    fill_timing_input<<<grid, 256, 0, s>>>(B.p, d * d, in_type, 91u + static_cast<uint32_t>(i));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return FMM_ERR_CUDA;
    float best = INFINITY;
    fmm_status st = FMM_OK;
    for (int L = 0; L < 3 && st == FMM_OK; ++L)
      for (int ti = 0; ti < 2 && st == FMM_OK; ++ti) {
        fmm_options o = {};
        o.tile_n = tiles[ti];
        auto call = [&]() {
          return fmm_gemm_ex(d, d, d, 1.0f, A.p, d, B.p, d, 0.0f, static_cast<float*>(C.p), d, L, variant,
                             W.p, ws, s, &o);
        };
        st = call();  // warm-up
        if (st != FMM_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == FMM_OK; ++r) st = call();
        cudaEventRecord(e1, s);
        if (st != FMM_OK) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
          st = FMM_ERR_CUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= static_cast<float>(reps);
        if (times_ms) times_ms[i * 6 + L * 2 + ti] = ms;
        if (ms < best) {
          best = ms;
          best_l[i] = L;
          best_t[i] = tiles[ti];
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == FMM_OK) st = fmm_device_status(stream);
    if (st != FMM_OK) return st;
  }
  // classes: probe i covers dimensions up to the geometric mean with probe i + 1; neighbours
  // with the same choice merge
  fmm_tune_table t = {};
  for (int i = 0; i < count; ++i) {
    const int64_t upper = i + 1 < count ? static_cast<int64_t>(std::sqrt(static_cast<double>(sizes[i]) * sizes[i + 1]))
                                        : INT64_MAX;
    if (t.count > 0 && t.levels[t.count - 1] == best_l[i] && t.tile_n[t.count - 1] == best_t[i]) {
      t.max_dim[t.count - 1] = upper;
    } else {
      t.max_dim[t.count] = upper;
      t.levels[t.count] = best_l[i];
      t.tile_n[t.count] = best_t[i];
      ++t.count;
    }
  }
  *out = t;
  return FMM_OK;
}
