// fmm_noalloc.cu -- fmm_gemm for callers that cannot allocate device memory.
//
// fmm_gemm takes a caller-provided workspace for the operand sums.  Some callers have no
// way to provide one: a plug-in running inside a host application that owns all device
// memory through its own pool and forbids allocations outside it, or a latency-critical
// caller that must not call cudaMalloc / cudaFree because those calls can synchronise the
// whole device.  fmm_gemm_noalloc serves them from a fixed scratch array that is part of
// this library's device image, so no device memory is allocated by the call.
//
// Limits and sharing rules (also stated in include/fmm.h):
//  * the scratch holds kNoallocScratchBytes (64 MiB); problems that need a larger
//    workspace are rejected with FMM_ERR_WORKSPACE.  fmm_workspace_size does not know
//    the operands' addresses, so for a classical product of 16-bit operands it counts a
//    conversion workspace that aligned operands (read in place) do not need: such a call
//    is tried without any workspace first;
//  * every GPU on which the library is loaded keeps this array until the process exits;
//  * all calls share the one array per device, and it keeps whatever the previous call
//    left in it; calls whose work overlaps on the GPU (for example on two streams at once)
//    race on it and must be serialised by the caller;
//  * nothing in the scratch has to start at zero: every byte the kernels read is written
//    earlier in the same call;
//  * the first call on each device looks up the array's device address (with that device
//    current); make that first call before any stream capture begins.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "fmm.h"
#include "launch.h"

namespace fmm {
namespace {

constexpr size_t kNoallocScratchBytes = size_t(64) << 20;

// Device scratch for the operand sums.  In host code this name is only a handle for the
// runtime; the device address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

}  // namespace
}  // namespace fmm

extern "C" fmm_status fmm_gemm_noalloc(int64_t m, int64_t n, int64_t k, float alpha,
                                       const void* A, int64_t lda, const void* B, int64_t ldb,
                                       float beta, float* C, int64_t ldc, int levels, int variant,
                                       void* stream) {
  using namespace fmm;
  const size_t need = fmm_workspace_size(m, n, k, levels, variant);
  if (need == static_cast<size_t>(-1)) {
    // unsupported combination: let fmm_gemm report exactly what is wrong (it launches nothing)
    return fmm_gemm(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, levels, variant, nullptr, 0,
                    stream);
  }
  if (need > kNoallocScratchBytes) {
    // The estimate may count a workspace this call does not need (16-bit operands read in
    // place).  fmm_gemm checks every argument, the workspace included, before it launches
    // anything, so a call without workspace either runs or fails with nothing enqueued.
    const fmm_status st = fmm_gemm(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, levels, variant,
                                   nullptr, 0, stream);
    if (st != FMM_ERR_WORKSPACE) return st;
    char msg[160];
    std::snprintf(msg, sizeof msg,
                  "fmm_gemm_noalloc: this problem needs %zu bytes of scratch; the built-in "
                  "scratch holds %zu bytes (use fmm_gemm with a workspace)",
                  need, kNoallocScratchBytes);
    set_last_error(msg);
    return FMM_ERR_WORKSPACE;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    set_last_error("fmm_gemm_noalloc: no current CUDA device");
    return FMM_ERR_CUDA;
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_last_error(std::string("fmm_gemm_noalloc: cudaGetSymbolAddress failed: ") +
                       cudaGetErrorString(e));
        return FMM_ERR_CUDA;
      }
      g_noalloc_addr[dev] = p;
    }
    scratch = g_noalloc_addr[dev];
  }
  return fmm_gemm(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, levels, variant, scratch,
                  kNoallocScratchBytes, stream);
}
