// fmm_api.cu -- the C ABI (include/fmm.h): argument checks, the Strassen planner (block
// sizes, the 7^L product table, destination maps, tensor maps) and the launch sequence.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "fmm.h"
#include "fmm_kernels.cuh"
#include "fmm_bases.h"
#include "launch.h"
#include "fmm_fused.cuh"

namespace fmm {

// Device error record written by bounded waits inside the kernels (read and cleared by
// fmm_device_status): [0] error bits, [1] site of the first wait that gave up, [2] its work
// item, [3] its k-step (low 16 bits) and block index (high 16 bits).
__device__ unsigned int g_device_err[4];

namespace {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_timeout_ns{2000000000ull};

// ------------------------------------------------------------- phase profiling
// When enabled, every launch of a phase is bracketed by two CUDA events recorded on
// the launching stream; fmm_profile_read sums their elapsed times.
enum Phase { kPhaseBeta = 0, kPhasePack = 1, kPhaseTensor = 2, kNumPhases = 3 };
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  int phase = 0;
  int launches = 1;  // kernel launches the scope brackets
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<EventPair> g_prof_pool;  // recorded, not yet read
std::vector<EventPair> g_prof_free;

struct PhaseScope {
  EventPair ev;
  cudaStream_t s;
  bool on = false;
  PhaseScope(int phase, cudaStream_t stream, int launches = 1) : s(stream) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    if (!g_prof_free.empty()) {
      ev = g_prof_free.back();
      g_prof_free.pop_back();
    } else {
      if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) return;
    }
    ev.phase = phase;
    ev.launches = launches;
    on = cudaEventRecord(ev.a, s) == cudaSuccess;
  }
  ~PhaseScope() {
    if (!on) return;
    cudaEventRecord(ev.b, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_pool.push_back(ev);
  }
};

fmm_status fail(fmm_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
fmm_status cuda_fail(cudaError_t e, const char* what) {
  return fail(FMM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct DeviceInfo {
  bool init = false;
  int sms = 0;
  unsigned* err = nullptr;
};

std::mutex g_mu;
DeviceInfo g_dev[64];
EncodeTiledFn g_encode = nullptr;

fmm_status device_info(DeviceInfo& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(FMM_ERR_CUDA, "device ordinal out of range");
  // The tensor maps are encoded through the driver API, which needs the device's primary
  // context current in this thread.  A thread that has made no runtime call yet (for example
  // autograd's device thread running this library's backward first) does not have it.
  thread_local bool ctx_current[64] = {};
  if (!ctx_current[dev]) {
    e = cudaSetDevice(dev);
    if (e == cudaSuccess) e = cudaFree(nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "making the device's context current");
    ctx_current[dev] = true;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceInfo& d = g_dev[dev];
  if (!d.init) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) {
      return fail(FMM_ERR_UNSUPPORTED, "this library is built for sm_103a (GB300); device is sm_" +
                                           std::to_string(major) + std::to_string(minor));
    }
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&d.err), g_device_err);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_device_err)");
    d.init = true;
  }
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(FMM_ERR_CUDA, "cuTensorMapEncodeTiled entry point not available");
    g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  out = d;
  return FMM_OK;
}

// ---------------------------------------------------------------- planner
struct Term {
  int block;  // bi * 2^L + bj
  int sign;
};
struct Product {
  std::vector<Term> a, b, c;
};

int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

// Multi-level products (Section 3.4): product (r_1..r_L) takes block (q_1..q_L) -- block q_L
// of ... of quadrant q_1 -- with coefficient prod_i X[r_i][q_i] (the Kronecker power).
std::vector<Product> make_products(int L, int basis = kBasisStrassen) {
  if (basis == kBasis323 && L == 1) {
    // a basis table: A blocks a = i*g_k + l, B blocks l*g_n + j, C blocks i*g_n + j
    std::vector<Product> out(15);
    for (int r = 0; r < 15; ++r) {
      for (int a = 0; a < 6; ++a)
        if (kB323U[a][r]) out[r].a.push_back({a, kB323U[a][r]});
      for (int b = 0; b < 6; ++b)
        if (kB323V[b][r]) out[r].b.push_back({b, kB323V[b][r]});
      for (int c = 0; c < 9; ++c)
        if (kB323W[c][r]) out[r].c.push_back({c, kB323W[c][r]});
    }
    return out;
  }
  if (basis == kBasis232 && L == 1) {
    // A blocks a = i*3 + l, B blocks b = l*2 + j, C blocks c = i*2 + j; Strassen's quadrant
    // q = 2*row + col of the leading 2 x 2 x 2 part maps to those numbers
    std::vector<Product> out(11);
    for (int r = 0; r < 7; ++r)
      for (int q = 0; q < 4; ++q) {
        const int row = q / 2, col = q % 2;
        if (const int u = strassen_u(r, q)) out[r].a.push_back({row * 3 + col, u});
        if (const int v = strassen_v(r, q)) out[r].b.push_back({row * 2 + col, v});
        if (const int w = strassen_w(r, q)) out[r].c.push_back({row * 2 + col, w});
      }
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        Product& pr = out[7 + 2 * i + j];
        pr.a.push_back({i * 3 + 2, 1});
        pr.b.push_back({2 * 2 + j, 1});
        pr.c.push_back({i * 2 + j, 1});
      }
    return out;
  }
  const int R = ipow(7, L), Q = ipow(4, L), g = 1 << L;
  std::vector<Product> out(R);
  for (int r = 0; r < R; ++r) {
    int rd[2] = {0, 0};
    for (int i = L - 1, t = r; i >= 0; --i, t /= 7) rd[i] = t % 7;
    for (int qi = 0; qi < Q; ++qi) {
      int qd[2] = {0, 0};
      for (int i = L - 1, t = qi; i >= 0; --i, t /= 4) qd[i] = t % 4;
      int cu = 1, cv = 1, cw = 1, br = 0, bc = 0;
      for (int i = 0; i < L; ++i) {
        cu *= basis_u(basis, rd[i], qd[i]);
        cv *= basis_v(basis, rd[i], qd[i]);
        cw *= basis_w(basis, rd[i], qd[i]);
        br = 2 * br + qd[i] / 2;
        bc = 2 * bc + qd[i] % 2;
      }
      const int blk = br * g + bc;
      if (cu) out[r].a.push_back({blk, cu});
      if (cv) out[r].b.push_back({blk, cv});
      if (cw) out[r].c.push_back({blk, cw});
    }
  }
  return out;
}

// Block grid (g_m, g_k, g_n) and product count R of `levels` levels of a basis; false for a
// combination that is not built.
struct BasisShape {
  int gm, gk, gn, R;
};
bool basis_shape(int levels, int basis, BasisShape& out) {
  if (levels < 0 || levels > 2) return false;
  if (levels == 0) {
    out = {1, 1, 1, 1};
    return true;
  }
  if (basis == kBasisStrassen || basis == kBasisWinograd) {
    const int g = 1 << levels;
    out = {g, g, g, ipow(7, levels)};
    return true;
  }
  if (basis == kBasis323 && levels == 1) {
    out = {3, 2, 3, 15};
    return true;
  }
  if (basis == kBasis232 && levels == 1) {
    out = {2, 3, 2, 11};
    return true;
  }
  return false;
}

// Block size of a dimension d split g ways (Section 3.5 padding, blocks rounded up to 8).
int64_t grid_block(int64_t d, int g) {
  if (g == 1) return d;
  const int64_t h = (d + g - 1) / g;
  return (h + 7) / 8 * 8;
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct Plan {
  int L = 0, R = 1, terms = 3, in_type = kInF32;
  bool bf16 = true;
  // Operand layouts of the GEMM C (M x N) = A' (M x K) B' (K x N):
  //   A' K-major: source stored M rows x K cols;  A' MN-major (a_mn): stored K rows x M cols;
  //   B' MN-major (b_mn): stored K rows x N cols; B' K-major: stored N rows x K cols.
  bool a_mn = false, b_mn = true;
  int tile_n = 128;
  int bk = 64;  // k-elements per pipeline stage of the packed kernel (64, or 32 for split3)
  bool pair = false;  // packed kernel in CTA pairs: 256-row tiles shared by two CTAs
  bool fused_ts = false;  // fused kernel with the A-operand sums in tensor memory
  int pipeline_mode = 0;  // fmm_options.pipeline: 0 automatic, 1 off, 2 on
  int basis = kBasisStrassen;  // coefficient tables (Strassen, Strassen-Winograd, <3,2,3> or <2,3,2>)
  int gm = 1, gk = 1, gn = 1;  // block grid of A (gm x gk), B (gk x gn) and C (gm x gn)
  bool deterministic = false;  // ownership mode (fixed order of the C updates)
  bool outer_scaling = false;  // power-of-two row (A) / column (B) scaling around the product
  size_t outer_off = 0;        // workspace offset of the row and column maxima
  bool pipeline = false;  // sum passes per top-level product, overlapped with the products
  int algo = FMM_ALGO_PACKED;
  int schedule = kSchedProductMajor;
  bool scaled = false;      // FP16 operands with power-of-two scaling per panel
  size_t scale_bytes = 0;   // panel maxima of A and B sums (scaled variant)
  int64_t panels_a = 0, panels_b = 0;
  int64_t hm = 0, hn = 0, hk = 0;
  int64_t lda_w = 0;  // row stride of the stored A-operand sums (rounded up to 8)
  int64_t ldb_w = 0;  // row stride of the stored B-operand sums
  size_t a_bytes = 0, b_bytes = 0;  // per term array
  size_t ws = 0;
};

fmm_status make_plan(int64_t m, int64_t n, int64_t k, int levels, int variant, const fmm_options* opt,
                     bool a_mn, bool b_mn, Plan& pl) {
  if (m < 0 || n < 0 || k < 0) return fail(FMM_ERR_ARG, "negative dimension");
  if (levels < 0 || levels > 2) return fail(FMM_ERR_UNSUPPORTED, "levels must be 0, 1 or 2");
  pl.L = levels;
  pl.a_mn = a_mn;
  pl.b_mn = b_mn;
  switch (variant) {
    case FMM_F32_SPLIT3_BF16: pl.terms = 3; pl.in_type = kInF32; pl.bf16 = true; break;
    case FMM_F32_PLAIN_BF16: pl.terms = 1; pl.in_type = kInF32; pl.bf16 = true; break;
    case FMM_BF16: pl.terms = 1; pl.in_type = kInBF16; pl.bf16 = true; break;
    case FMM_F16_SCALED: pl.terms = 1; pl.in_type = kInF16; pl.bf16 = false; pl.scaled = true; break;
    default: return fail(FMM_ERR_UNSUPPORTED, "variant not built");
  }
  if (pl.scaled && (a_mn || !b_mn))
    return fail(FMM_ERR_UNSUPPORTED, "the scaled FP16 variant is built for the forward product");
  const int algo = opt ? opt->algo : 0;
  if (algo < FMM_ALGO_AUTO || algo > FMM_ALGO_HYBRID) return fail(FMM_ERR_UNSUPPORTED, "algorithm not built");
  if (algo == FMM_ALGO_HYBRID && levels != 2)
    return fail(FMM_ERR_UNSUPPORTED, "the hybrid algorithm is a two-level scheme (levels = 2)");
  pl.algo = algo == FMM_ALGO_AUTO ? FMM_ALGO_PACKED : algo;
  const bool on_chip = pl.algo == FMM_ALGO_FUSED || pl.algo == FMM_ALGO_HYBRID;
  // the fused kernels read FP32 source tiles: the caller's FP32 operands (fused), or the FP32
  // top-level sums the hybrid scheme forms from FP32 or BF16 operands
  if (pl.algo == FMM_ALGO_HYBRID && (a_mn || !b_mn))
    return fail(FMM_ERR_UNSUPPORTED, "the hybrid algorithm is built for the forward product");
  pl.tile_n = (opt && opt->tile_n) ? opt->tile_n : 0;
  const int sched = opt ? opt->schedule : 0;
  if (sched < 0 || sched > 2) return fail(FMM_ERR_ARG, "schedule must be 0, 1 or 2");
  const int basis = opt ? opt->basis : 0;
  if (basis < kBasisStrassen || basis > kBasis232) return fail(FMM_ERR_ARG, "basis must be 0, 1, 2 or 3");
  if (basis == kBasisWinograd && (levels > 1 || pl.algo == FMM_ALGO_HYBRID))
    return fail(FMM_ERR_UNSUPPORTED, "the Winograd basis is built for one level (packed or fused)");
  const bool table_basis = basis == kBasis323 || basis == kBasis232;
  if (table_basis && levels > 1)
    return fail(FMM_ERR_UNSUPPORTED, "the <3,2,3> and <2,3,2> bases are built for one level");
  if (table_basis && levels == 1 && pl.algo == FMM_ALGO_HYBRID)
    return fail(FMM_ERR_UNSUPPORTED, "the hybrid algorithm is a two-level Strassen scheme");
  if (table_basis && levels == 1 && opt && opt->pipeline == 2)
    return fail(FMM_ERR_UNSUPPORTED, "the <3,2,3> and <2,3,2> bases form their sums in one pass (no pipelining)");
  pl.basis = levels == 0 ? kBasisStrassen : basis;
  BasisShape shape;
  if (!basis_shape(levels, pl.basis, shape)) return fail(FMM_ERR_UNSUPPORTED, "basis and levels not built");
  pl.gm = shape.gm;
  pl.gk = shape.gk;
  pl.gn = shape.gn;
  pl.R = shape.R;
  pl.hm = grid_block(m, pl.gm);
  pl.hn = grid_block(n, pl.gn);
  pl.hk = grid_block(k, pl.gk);
  // automatic choice (measured on GB300): tile rounds, which keep the destination blocks of
  // a round in L2; with the sums formed on chip, product-major order (all pairs on one
  // product, so the source tiles of its blocks are shared in L2 by every tile in flight:
  // +9 % one level, +7 % hybrid at 16384^3 over tile rounds of one tile per pair)
  const bool on_chip_algo = pl.algo == FMM_ALGO_FUSED || pl.algo == FMM_ALGO_HYBRID;
  pl.schedule = (sched == 1 || (sched == 0 && on_chip_algo)) ? kSchedProductMajor : kSchedTileRounds;
  const int bk = opt ? opt->bk : 0;
  const int cta_pair = opt ? opt->cta_pair : 0;
  if (cta_pair < 0 || cta_pair > 2) return fail(FMM_ERR_ARG, "cta_pair must be 0, 1 or 2");
  if (cta_pair == 2 && bk == 32)
    return fail(FMM_ERR_UNSUPPORTED, "CTA pairs use 64-deep stages (bk = 64)");
  if (on_chip && bk == 32) return fail(FMM_ERR_UNSUPPORTED, "the fused and hybrid algorithms use bk = 64");
  // automatic choice: CTA pairs (each CTA loads, or forms, half of the B tile)
  pl.pair = bk != 32 && cta_pair != 1;
  if (on_chip) {
    // fused tiles: 128 x 128 per CTA, 256 x 256 per CTA pair
    const int fused_n = pl.pair ? 2 * kFusedTileN : kFusedTileN;
    if (pl.tile_n != 0 && pl.tile_n != fused_n)
      return fail(FMM_ERR_UNSUPPORTED, pl.pair ? "the fused and hybrid algorithms use 256-wide tiles in CTA pairs"
                                               : "the fused and hybrid algorithms use 128-wide tiles");
    pl.tile_n = fused_n;
  }
  if (opt && (opt->store_first < 0 || opt->store_first > 2)) return fail(FMM_ERR_ARG, "store_first must be 0, 1 or 2");
  const int fk = opt ? opt->fused_kernel : 0;
  if (fk < 0 || fk > 2) return fail(FMM_ERR_ARG, "fused_kernel must be 0, 1 or 2");
  if (fk == 2 && on_chip && !pl.pair)
    return fail(FMM_ERR_UNSUPPORTED, "the tensor-memory fused kernel runs in CTA pairs");
  if (on_chip && pl.scaled && (!pl.pair || fk == 1))
    return fail(FMM_ERR_UNSUPPORTED, "scaled FP16 products with on-chip sums run in the tensor-memory kernel");
  pl.fused_ts = on_chip && pl.pair && fk != 1;
  // 16-bit operands: the hybrid scheme (FP32 top-level sums), or the tensor-memory kernel on
  // the caller's BF16 / FP16 source tiles (forward products; FP16 panel scaling: Strassen)
  if (pl.algo == FMM_ALGO_FUSED && pl.in_type != kInF32 &&
      (!pl.fused_ts || a_mn || !b_mn || (pl.scaled && pl.basis != kBasisStrassen)))
    return fail(FMM_ERR_UNSUPPORTED,
                "the fused algorithm takes BF16 and FP16 operands in the tensor-memory kernel (CTA pairs, "
                "forward products; FP16 with Strassen's basis)");
  // the backward products (A' stored by rows of k, or B' by rows of n) run on chip in the
  // tensor-memory kernel
  if (on_chip && (a_mn || !b_mn) && (!pl.fused_ts || (a_mn && !b_mn)))
    return fail(FMM_ERR_UNSUPPORTED,
                "the fused algorithm runs the backward products in the tensor-memory kernel (CTA pairs)");
  if (!on_chip && !pl.pair && (a_mn || !b_mn))
    return fail(FMM_ERR_UNSUPPORTED, "single-CTA tiles are built for the forward product only");
  const int pipe = opt ? opt->pipeline : 0;
  if (pipe < 0 || pipe > 2) return fail(FMM_ERR_ARG, "pipeline must be 0, 1 or 2");
  const int det = opt ? opt->deterministic : 0;
  if (det < 0 || det > 1) return fail(FMM_ERR_ARG, "deterministic must be 0 or 1");
  pl.deterministic = det == 1;
  if (pl.deterministic) pl.schedule = kSchedTileRounds;  // ownership needs whole-tile rounds
  const int osc = opt ? opt->outer_scaling : 0;
  if (osc < 0 || osc > 1) return fail(FMM_ERR_ARG, "outer_scaling must be 0 or 1");
  if (osc == 1 && (on_chip || a_mn || !b_mn))
    return fail(FMM_ERR_UNSUPPORTED, "outside scaling is built for the packed forward product");
  pl.outer_scaling = osc == 1;
  if (pl.outer_scaling) pl.pipeline = false;
  pl.pipeline_mode = pipe;
  pl.pipeline = !on_chip && levels >= 1 && pipe == 2;  // automatic: decided with C (prepare_packed)
  const int row_tile = pl.pair ? 2 * kBM : kBM;
  if (pl.tile_n == 0) {
    // 256-wide tiles halve the A-operand traffic; keep 128 when that leaves fewer than four
    // work items per SM (per CTA pair) on a 152-SM GB300
    const int64_t items256 = static_cast<int64_t>(pl.R) * ((pl.hm + row_tile - 1) / row_tile) * ((pl.hn + 255) / 256);
    pl.tile_n = items256 >= 4 * (pl.pair ? 76 : 152) ? 256 : 128;
  }
  if (!packed_config_supported(pl.tile_n, pl.terms, pl.bf16))
    return fail(FMM_ERR_UNSUPPORTED, "tile_n must be 128 or 256");
  if (bk != 0 && bk != 32 && bk != 64) return fail(FMM_ERR_ARG, "bk must be 0, 32 or 64");
  if (bk == 32 && pl.terms != 3) return fail(FMM_ERR_UNSUPPORTED, "32-deep stages are built for split3");
  pl.bk = bk == 0 ? 64 : bk;
  if (pl.hm >= (int64_t(1) << 31) || pl.hn >= (int64_t(1) << 31) || pl.hk >= (int64_t(1) << 31))
    return fail(FMM_ERR_ARG, "dimension too large");
  const int64_t a_rows = a_mn ? pl.hk : pl.hm;
  pl.lda_w = round_up(std::max<int64_t>(a_mn ? pl.hm : pl.hk, 1), 8);
  const int64_t b_rows = b_mn ? pl.hk : pl.hn;
  pl.ldb_w = round_up(std::max<int64_t>(b_mn ? pl.hn : pl.hk, 1), 8);
  pl.a_bytes = static_cast<size_t>(round_up(static_cast<int64_t>(pl.R) * a_rows * pl.lda_w * 2, 256));
  pl.b_bytes = static_cast<size_t>(round_up(static_cast<int64_t>(pl.R) * b_rows * pl.ldb_w * 2, 256));
  const size_t arrays = pl.terms == 3 ? 2 : 1;
  pl.ws = (m == 0 || n == 0 || k == 0 || pl.algo == FMM_ALGO_FUSED) ? 0 : arrays * (pl.a_bytes + pl.b_bytes);
  const bool fused_scaled = pl.algo == FMM_ALGO_FUSED && pl.scaled && m > 0 && n > 0 && k > 0;
  if (pl.scaled && (pl.ws > 0 || fused_scaled)) {
    // FP16: the panel maxima of the operand sums (the only workspace of a fused FP16 product)
    pl.panels_a = (pl.hm + kBM - 1) / kBM;
    pl.panels_b = (pl.hn + pl.tile_n - 1) / pl.tile_n;
    pl.scale_bytes = static_cast<size_t>(round_up(pl.R * (pl.panels_a + pl.panels_b) * 4, 256));
    pl.ws += pl.scale_bytes;
  }
  if (pl.algo == FMM_ALGO_HYBRID && pl.ws > 0) {
    // seven top-level sums of each operand in FP32, blocks of 2h x 2h
    pl.a_bytes = static_cast<size_t>(round_up(7 * (2 * pl.hm) * (2 * pl.hk) * 4, 256));
    pl.b_bytes = static_cast<size_t>(round_up(7 * (2 * pl.hk) * (2 * pl.hn) * 4, 256));
    pl.ws = pl.a_bytes + pl.b_bytes + (pl.scaled ? pl.scale_bytes : 0);
  }
  if (pl.outer_scaling && pl.ws > 0) {
    // float bits of max |x| of the m rows of A and the n columns of B
    pl.outer_off = pl.ws;
    pl.ws += static_cast<size_t>(round_up((m + n) * 4, 256));
  }
  return FMM_OK;
}

// One GEMM operand as the caller stores it (row-major, leading dimension ld, element type).
struct Operand {
  const void* X;
  int64_t ld;
  int type;
};

bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  if (!a || !b || abytes == 0 || bbytes == 0) return false;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
  return a0 < b0 + bbytes && b0 < a0 + abytes;
}

fmm_status encode_3d(CUtensorMap* map, void* base, int64_t inner, int64_t rows, int64_t depth,
                     int64_t ld_elems, int box_inner, int box_rows,
                     CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(rows),
                              static_cast<cuuint64_t>(depth)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld_elems * 2),
                                 static_cast<cuuint64_t>(ld_elems * 2 * rows)};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(box_inner), static_cast<cuuint32_t>(box_rows), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(FMM_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
  return FMM_OK;
}

size_t elem_bytes(int in_type) { return in_type == kInF32 ? 4 : 2; }

int64_t block_extent(int64_t d, int64_t h, int b) {
  return std::min<int64_t>(std::max<int64_t>(d - b * h, 0), h);
}

// C bytes that the items of one tile round may update (a quarter of the 129 MB L2 of a GB300,
// so that the operand panels of the round stay resident beside them).
constexpr int64_t kRoundL2Bytes = int64_t(32) << 20;

// Work list, destination maps and C tensor maps shared by both tensor-core kernels.
// `live` lists the products that run (their kernel-side index is their position in it).
fmm_status fill_common(CommonParams& c, const Plan& pl, const std::vector<Product>& prods,
                       const std::vector<int>& live, int64_t m, int64_t n, float alpha, float* C,
                       int64_t ldc, const DeviceInfo& dev, const fmm_options* opt, int& grid) {
  const int gn = pl.gn, nblocks = pl.gm * pl.gn;  // C blocks c = bi * gn + bj
  c.C = C;
  c.ldc = ldc;
  c.alpha = alpha;
  c.schedule = pl.schedule;
  c.c_tma = (reinterpret_cast<uintptr_t>(C) % 16 == 0 && ldc % 4 == 0) ? 1 : 0;
  c.c_vec4 = c.c_tma;
  c.err = dev.err;
  c.timeout_ns = g_timeout_ns.load();
  const int row_tile = pl.pair ? 2 * kBM : kBM;  // rows of one work item's output tile
  c.tiles_m = static_cast<int32_t>((pl.hm + row_tile - 1) / row_tile);
  c.tiles_n = static_cast<int32_t>((pl.hn + pl.tile_n - 1) / pl.tile_n);
  c.nk = static_cast<int32_t>((pl.hk + pl.bk - 1) / pl.bk);  // fused and hybrid plans keep bk = 64
  const int64_t items = static_cast<int64_t>(live.size()) * c.tiles_m * c.tiles_n;
  if (items >= (int64_t(1) << 31)) return fail(FMM_ERR_ARG, "too many tiles");
  c.num_items = static_cast<int32_t>(items);
  c.num_products = static_cast<int32_t>(live.size());
  for (size_t i = 0; i < live.size(); ++i) {
    int cnt = 0;
    for (const Term& t : prods[live[i]].c) {
      const int br = t.block / gn, bc = t.block % gn;
      const int64_t rows = block_extent(m, pl.hm, br), cols = block_extent(n, pl.hn, bc);
      if (rows == 0 || cols == 0) continue;
      DestEntry& de = c.prod[i].d[cnt++];
      de.offset = br * pl.hm * ldc + bc * pl.hn;
      de.rows = static_cast<int32_t>(rows);
      de.cols = static_cast<int32_t>(cols);
      de.coef = alpha * static_cast<float>(t.sign);
      de.block = t.block;
      de.store = 0;
      de.pad = 0;
    }
    c.prod[i].count = cnt;
    c.prod[i].sum_index = static_cast<int32_t>(i);
  }
  if (c.c_tma) {
    // one FP32 map per non-empty destination block, clipped to the block's extent in C
    for (int b = 0; b < nblocks; ++b) {
      const int64_t rows = block_extent(m, pl.hm, b / gn), cols = block_extent(n, pl.hn, b % gn);
      if (rows == 0 || cols == 0) continue;
      const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
      const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ldc * 4)};
      const cuuint32_t box[2] = {32, 32};
      const cuuint32_t estr[2] = {1, 1};
      CUresult cr = g_encode(&c.tmC[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                             C + ((b / gn) * pl.hm * ldc + (b % gn) * pl.hn), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (cr != CUDA_SUCCESS)
        return fail(FMM_ERR_CUDA, "cuTensorMapEncodeTiled (C) failed (" + std::to_string(cr) + ")");
    }
  }
  grid = opt && opt->num_ctas > 0 ? opt->num_ctas : dev.sms;
  if (pl.pair)  // whole pairs, at most one per item
    grid = 2 * static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(grid / 2, items)));
  else
    grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(grid, items)));
  // Tile rounds.  When an item moves at least half as many C bytes (read and write of each
  // destination tile) as operand bytes, keep the C blocks of a round (every destination block
  // of its tile positions: one tile in each of the g_m x g_n blocks) within kRoundL2Bytes; otherwise one tile per worker,
  // which shares operand panels between the most concurrent items.  Element-wise reductions
  // (C rows not 16-byte aligned) keep one tile per worker: small rounds make concurrent items
  // add into the same C elements, and those atomics serialise.  Measured on GB300.
  const int workers = pl.pair ? grid / 2 : grid;
  int64_t dests = 0;
  for (size_t i = 0; i < live.size(); ++i) dests += c.prod[i].count;
  const double c_bytes = live.empty() ? 0.0 : 8.0 * row_tile * pl.tile_n * dests / live.size();
  const double op_bytes = 2.0 * (row_tile + pl.tile_n) * pl.hk * (pl.terms == 3 ? 2 : 1);
  const int64_t footprint = static_cast<int64_t>(nblocks) * row_tile * pl.tile_n * 4;
  int64_t rt = workers;
  if (opt && opt->round_tiles > 0)
    rt = opt->round_tiles;
  else if (c.c_tma && c_bytes >= 0.5 * op_bytes)
    rt = std::max<int64_t>(1, kRoundL2Bytes / footprint);
  c.round_tiles = rt >= workers ? 0 : static_cast<int32_t>(rt);
  if (pl.deterministic) {
    // ownership: rounds of exactly one tile per worker, the last round padded with empty
    // items, so that worker b runs every product of tile position b of each round
    const int64_t tiles = static_cast<int64_t>(c.tiles_m) * c.tiles_n;
    const int64_t rounds = (tiles + workers - 1) / workers;
    const int64_t padded = rounds * workers * static_cast<int64_t>(live.size());
    if (padded >= (int64_t(1) << 31)) return fail(FMM_ERR_ARG, "too many tiles");
    c.deterministic = 1;
    c.round_tiles = workers;
    c.num_items = static_cast<int32_t>(padded);
  }
  return FMM_OK;
}

// Fused path: FP32 source tiles are summed on chip; no workspace.
// 16-bit operands (forward products, tensor-memory kernel): the source tiles are the caller's
// BF16 or FP16 values; an FP16 product first records the panel maxima of its operand sums in
// `ws` (the only workspace it takes).
fmm_status gemm_fused(const Plan& pl, int64_t m, int64_t n, int64_t k, float alpha, const void* A,
                      int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, void* ws,
                      const DeviceInfo& dev, const fmm_options* opt, cudaStream_t s) {
  const bool s16 = pl.in_type != kInF32;
  const size_t esz = s16 ? 2 : 4;
  const CUtensorMapDataType dtype = !s16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                         : (pl.in_type == kInF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  const std::vector<Product> prods = make_products(pl.L, pl.basis);
  // A blocks a = i * g_k + l (g_m x g_k grid), B blocks b = l * g_n + j (g_k x g_n grid)
  const int na_blk = pl.gm * pl.gk, nb_blk = pl.gk * pl.gn;
  if (na_blk > kMaxFusedSources || nb_blk > kMaxFusedSources)
    return fail(FMM_ERR_UNSUPPORTED, "too many source blocks for the fused kernel");
  FusedParams* fp = new FusedParams;
  std::memset(fp, 0, sizeof(FusedParams));
  fmm_status st = FMM_OK;
  std::vector<bool> a_live(na_blk, false), b_live(nb_blk, false);
  for (int b = 0; b < std::max(na_blk, nb_blk) && st == FMM_OK; ++b) {
    const uint8_t* Af = static_cast<const uint8_t*>(A);
    const uint8_t* Bf = static_cast<const uint8_t*>(B);
    // A block b = (bi, bj): rows of m, columns of k
    const int bi = b / pl.gk, bj = b % pl.gk;
    const int64_t ar = b < na_blk ? block_extent(m, pl.hm, bi) : 0;
    const int64_t ac = b < na_blk ? block_extent(k, pl.hk, bj) : 0;
    if (ar > 0 && ac > 0) {
      // A' stored m x k (box 32 k x 128 rows, 128-byte swizzle), or by rows of k (a_mn: the
      // block (bi, bj) of A' is the source's block (bj, bi); box 128 m x 32 k)
      const cuuint64_t dims[2] = {static_cast<cuuint64_t>(pl.a_mn ? ar : ac), static_cast<cuuint64_t>(pl.a_mn ? ac : ar)};
      const cuuint64_t strides[1] = {static_cast<cuuint64_t>(lda * esz)};
      const cuuint32_t box[2] = {pl.a_mn ? 128u : 32u, pl.a_mn ? 32u : 128u};
      const cuuint32_t estr[2] = {1, 1};
      const uint8_t* base = Af + esz * (pl.a_mn ? (bj * pl.hk * lda + bi * pl.hm) : (bi * pl.hm * lda + bj * pl.hk));
      // rows of 32 FP32 values (128 bytes, 128-byte swizzle) or 32 16-bit values (64 bytes)
      const CUtensorMapSwizzle swz = pl.a_mn ? CU_TENSOR_MAP_SWIZZLE_NONE
                                             : (s16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
      CUresult cr = g_encode(&fp->tmSA[b], dtype, 2, const_cast<uint8_t*>(base), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (cr != CUDA_SUCCESS) st = fail(FMM_ERR_CUDA, "cuTensorMapEncodeTiled (A block) failed");
      a_live[b] = true;
    }
    // B block b = (bl, bn): rows of k, columns of n
    const int bl = b / pl.gn, bn = b % pl.gn;
    const int64_t br = b < nb_blk ? block_extent(k, pl.hk, bl) : 0;
    const int64_t bc = b < nb_blk ? block_extent(n, pl.hn, bn) : 0;
    if (st == FMM_OK && br > 0 && bc > 0) {
      // B' stored k x n (box 128 n x 32 k), or by rows of n (!b_mn: the block (bl, bn) of B' is
      // the source's block (bn, bl); box 32 k x 128 n-rows, 128-byte swizzle)
      const bool kmaj = !pl.b_mn;
      const cuuint64_t dims[2] = {static_cast<cuuint64_t>(kmaj ? br : bc), static_cast<cuuint64_t>(kmaj ? bc : br)};
      const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ldb * esz)};
      const cuuint32_t box[2] = {kmaj ? 32u : static_cast<cuuint32_t>(kFusedTileN),
                                 kmaj ? static_cast<cuuint32_t>(kFusedTileN) : 32u};
      const cuuint32_t estr[2] = {1, 1};
      const uint8_t* base = Bf + esz * (kmaj ? (bn * pl.hn * ldb + bl * pl.hk) : (bl * pl.hk * ldb + bn * pl.hn));
      CUresult cr = g_encode(&fp->tmSB[b], dtype, 2, const_cast<uint8_t*>(base), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE,
                             kmaj ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (cr != CUDA_SUCCESS) st = fail(FMM_ERR_CUDA, "cuTensorMapEncodeTiled (B block) failed");
      b_live[b] = true;
    }
  }
  // products whose A- or B-operand has no block inside the matrices contribute nothing
  std::vector<int> live;
  for (int r = 0; r < pl.R && st == FMM_OK; ++r) {
    ProductSrc ps;
    std::memset(&ps, 0, sizeof ps);
    if (prods[r].a.size() > static_cast<size_t>(kMaxDest) || prods[r].b.size() > static_cast<size_t>(kMaxDest)) {
      st = fail(FMM_ERR_UNSUPPORTED, "a product combines more source blocks than the fused kernel takes");
      break;
    }
    for (const Term& t : prods[r].a)
      if (a_live[t.block]) {
        ps.a_block[ps.na] = static_cast<int8_t>(t.block);
        if (t.sign < 0) ps.a_neg |= static_cast<uint8_t>(1u << ps.na);
        ps.a_sign[ps.na++] = static_cast<int8_t>(t.sign);
      }
    for (const Term& t : prods[r].b)
      if (b_live[t.block]) {
        ps.b_block[ps.nb] = static_cast<int8_t>(t.block);
        if (t.sign < 0) ps.b_neg |= static_cast<uint8_t>(1u << ps.nb);
        ps.b_sign[ps.nb++] = static_cast<int8_t>(t.sign);
      }
    if (ps.na == 0 || ps.nb == 0) continue;
    fp->src[live.size()] = ps;
    live.push_back(r);
  }
  int grid = 0;
  if (st == FMM_OK && !live.empty()) st = fill_common(fp->c, pl, prods, live, m, n, alpha, C, ldc, dev, opt, grid);
  if (st != FMM_OK || live.empty()) {
    delete fp;
    return st;
  }
  cudaError_t e;
  if (pl.scaled) {
    // FP16: per (product, panel) the largest |operand sum|, one pass over each operand that
    // forms the sums without storing them; the kernel's transform and epilogue read the row of
    // the product's basis index
    unsigned* maxbits = static_cast<unsigned*>(ws);
    e = cudaMemsetAsync(maxbits, 0, pl.scale_bytes, s);
    if (e != cudaSuccess) {
      delete fp;
      return cuda_fail(e, "clearing the panel maxima");
    }
    SumParams ma;
    std::memset(&ma, 0, sizeof ma);
    ma.X = A;
    ma.ldx = lda;
    ma.rows = m;
    ma.cols = k;
    ma.hr = pl.hm;
    ma.hc = pl.hk;
    ma.terms = 1;
    ma.chunk = -1;
    ma.vec_ok = 1;  // 16-byte aligned base and rows (validate_core)
    ma.maxbits = maxbits;
    ma.npanels = static_cast<int32_t>(pl.panels_a);
    ma.panel_w = kBM;
    ma.scale_rows = 1;
    SumParams mb = ma;
    mb.X = B;
    mb.ldx = ldb;
    mb.rows = k;
    mb.cols = n;
    mb.hr = pl.hk;
    mb.hc = pl.hn;
    mb.maxbits = maxbits + static_cast<int64_t>(pl.R) * pl.panels_a;
    mb.npanels = static_cast<int32_t>(pl.panels_b);
    mb.panel_w = pl.tile_n;
    mb.scale_rows = 0;
    {
      PhaseScope ps(kPhasePack, s, 2);
      e = launch_operand_maxima_f16(ma, pl.L, false, dev.sms, s);
      if (e == cudaSuccess) e = launch_operand_maxima_f16(mb, pl.L, true, dev.sms, s);
    }
    if (e != cudaSuccess) {
      delete fp;
      return cuda_fail(e, "panel maxima of the operand sums");
    }
    fp->c.maxbits_a = ma.maxbits;
    fp->c.maxbits_b = mb.maxbits;
    fp->c.panels_a = static_cast<int32_t>(pl.panels_a);
    fp->c.panels_b = static_cast<int32_t>(pl.panels_b);
    for (size_t i = 0; i < live.size(); ++i) fp->c.prod[i].sum_index = static_cast<int32_t>(live[i]);
  }
  {
    PhaseScope ps(kPhaseTensor, s);
    e = pl.fused_ts ? launch_fused_ts(*fp, pl.terms, pl.a_mn, pl.b_mn, pl.scaled, s16, grid, s)
                    : launch_fused(*fp, pl.terms, kFusedTransformWarps, pl.pair, grid, s);
  }
  delete fp;
  if (e != cudaSuccess) return cuda_fail(e, "fused tensor-core pass");
  return FMM_OK;
}


fmm_status encode_f32_2d(CUtensorMap* map, const float* base, int64_t cols, int64_t rows, int64_t ld,
                         uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle swz) {
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld * 4)};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult cr = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(FMM_ERR_CUDA, "cuTensorMapEncodeTiled (FP32 source) failed");
  return FMM_OK;
}

// Hybrid two-level path (Section 3.4): the seven top-level operand sums of A and of B are
// materialised in FP32 in the workspace (blocks of 2h_m x 2h_k and 2h_k x 2h_n, zero-padded);
// the 49 bottom-level products are then formed on chip by the fused kernel from the quadrants
// of those sums, and each is added into its composite destinations
// W[q1, r1] * W[q2, r2] directly in C (no product ever reaches memory).
fmm_status gemm_hybrid(const Plan& pl, int64_t m, int64_t n, int64_t k, float alpha, const void* A,
                       int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, void* ws,
                       const DeviceInfo& dev, const fmm_options* opt, cudaStream_t s) {
  const int64_t h1m = 2 * pl.hm, h1k = 2 * pl.hk, h1n = 2 * pl.hn;
  float* P = static_cast<float*>(ws);
  float* Q = reinterpret_cast<float*>(static_cast<uint8_t*>(ws) + pl.a_bytes);
  SumParams sa;
  std::memset(&sa, 0, sizeof sa);
  sa.X = A;
  sa.ldx = lda;
  sa.rows = m;
  sa.cols = k;
  sa.hr = h1m;
  sa.hc = h1k;
  sa.ld_out = h1k;
  sa.prod_stride = h1m * h1k;
  sa.out_f32 = P;
  sa.terms = 0;
  sa.chunk = -1;
  sa.vec_ok = (reinterpret_cast<uintptr_t>(A) % 16 == 0 && lda % 4 == 0) ? 1 : 0;
  cudaError_t e;
  {
    PhaseScope ps(kPhasePack, s);
    e = launch_operand_sums(sa, 1, false, false, pl.in_type, 0, dev.sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "top-level operand sums (A)");
  SumParams sb = sa;
  sb.X = B;
  sb.ldx = ldb;
  sb.rows = k;
  sb.cols = n;
  sb.hr = h1k;
  sb.hc = h1n;
  sb.ld_out = h1n;
  sb.prod_stride = h1k * h1n;
  sb.out_f32 = Q;
  sb.vec_ok = (reinterpret_cast<uintptr_t>(B) % 16 == 0 && ldb % 4 == 0) ? 1 : 0;
  {
    PhaseScope ps(kPhasePack, s);
    e = launch_operand_sums(sb, 1, true, false, pl.in_type, 0, dev.sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "top-level operand sums (B)");

  // FP16: panel maxima of the 49 bottom-level operand sums, one pass over each top-level sum
  unsigned* maxbits = pl.scaled ? reinterpret_cast<unsigned*>(static_cast<uint8_t*>(ws) + pl.a_bytes + pl.b_bytes)
                                : nullptr;
  if (maxbits) {
    e = cudaMemsetAsync(maxbits, 0, pl.scale_bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the panel maxima");
    for (int r1 = 0; r1 < 7; ++r1) {
      SumParams ma;
      std::memset(&ma, 0, sizeof ma);
      ma.X = P + r1 * h1m * h1k;
      ma.ldx = h1k;
      ma.rows = h1m;
      ma.cols = h1k;
      ma.hr = pl.hm;
      ma.hc = pl.hk;
      ma.terms = 1;
      ma.chunk = -1;
      ma.vec_ok = 1;
      ma.maxbits = maxbits + static_cast<int64_t>(r1) * 7 * pl.panels_a;
      ma.npanels = static_cast<int32_t>(pl.panels_a);
      ma.panel_w = kBM;
      ma.scale_rows = 1;
      SumParams mb = ma;
      mb.X = Q + r1 * h1k * h1n;
      mb.ldx = h1n;
      mb.rows = h1k;
      mb.cols = h1n;
      mb.hr = pl.hk;
      mb.hc = pl.hn;
      mb.maxbits = maxbits + 49 * pl.panels_a + static_cast<int64_t>(r1) * 7 * pl.panels_b;
      mb.npanels = static_cast<int32_t>(pl.panels_b);
      mb.panel_w = pl.tile_n;
      mb.scale_rows = 0;
      PhaseScope ps(kPhasePack, s, 2);
      e = launch_operand_maxima(ma, false, dev.sms, s);
      if (e == cudaSuccess) e = launch_operand_maxima(mb, true, dev.sms, s);
      if (e != cudaSuccess) return cuda_fail(e, "panel maxima of the bottom-level sums");
    }
  }
  FusedParams* fp = new FusedParams;
  std::memset(fp, 0, sizeof(FusedParams));
  fmm_status st = FMM_OK;
  for (int r1 = 0; r1 < 7 && st == FMM_OK; ++r1) {
    for (int q2 = 0; q2 < 4 && st == FMM_OK; ++q2) {
      const int i2 = q2 / 2, j2 = q2 % 2;
      st = encode_f32_2d(&fp->tmSA[r1 * 4 + q2], P + r1 * h1m * h1k + i2 * pl.hm * h1k + j2 * pl.hk,
                         pl.hk, pl.hm, h1k, 32, kBM, CU_TENSOR_MAP_SWIZZLE_128B);
      if (st == FMM_OK)
        st = encode_f32_2d(&fp->tmSB[r1 * 4 + q2], Q + r1 * h1k * h1n + i2 * pl.hk * h1n + j2 * pl.hn,
                           pl.hn, pl.hk, h1n, kFusedTileN, 32, CU_TENSOR_MAP_SWIZZLE_NONE);
    }
  }
  const std::vector<Product> prods = make_products(2);
  std::vector<int> live(49);
  for (int r = 0; r < 49; ++r) {
    live[r] = r;
    const int r1 = r / 7, r2 = r % 7;
    ProductSrc& ps = fp->src[r];
    for (int q2 = 0; q2 < 4; ++q2) {
      if (const int c = strassen_u(r2, q2)) {
        ps.a_block[ps.na] = static_cast<int8_t>(r1 * 4 + q2);
        if (c < 0) ps.a_neg |= static_cast<uint8_t>(1u << ps.na);
        ps.a_sign[ps.na++] = static_cast<int8_t>(c);
      }
      if (const int c = strassen_v(r2, q2)) {
        ps.b_block[ps.nb] = static_cast<int8_t>(r1 * 4 + q2);
        if (c < 0) ps.b_neg |= static_cast<uint8_t>(1u << ps.nb);
        ps.b_sign[ps.nb++] = static_cast<int8_t>(c);
      }
    }
  }
  int grid = 0;
  if (st == FMM_OK) st = fill_common(fp->c, pl, prods, live, m, n, alpha, C, ldc, dev, opt, grid);
  if (st != FMM_OK) {
    delete fp;
    return st;
  }
  if (maxbits) {
    fp->c.maxbits_a = maxbits;
    fp->c.maxbits_b = maxbits + 49 * pl.panels_a;
    fp->c.panels_a = static_cast<int32_t>(pl.panels_a);
    fp->c.panels_b = static_cast<int32_t>(pl.panels_b);
  }
  {
    PhaseScope ps(kPhaseTensor, s);
    e = pl.fused_ts ? launch_fused_ts(*fp, pl.terms, pl.a_mn, pl.b_mn, pl.scaled, false, grid, s)
                    : launch_fused(*fp, pl.terms, kFusedTransformWarps, pl.pair, grid, s);
  }
  delete fp;
  if (e != cudaSuccess) return cuda_fail(e, "hybrid tensor-core pass");
  return FMM_OK;
}

// Argument checks of one product (no CUDA calls).
// TMA can read this operand in place: 16-byte aligned base and rows.
bool tma_addressable(const Operand& o) {
  return reinterpret_cast<uintptr_t>(o.X) % 16 == 0 && o.ld % 8 == 0;
}

// Operand "sums" of a classical product of 16-bit operands are the operands themselves; the
// tensor-core kernel reads an operand in place when TMA can address it (prepare_packed), and
// when both are read in place the product needs no workspace at all.
bool in_place_operand(const Plan& pl, const Operand& o) {
  return pl.algo == FMM_ALGO_PACKED && pl.L == 0 && pl.terms == 1 && o.type != kInF32 && !pl.outer_scaling &&
         tma_addressable(o);
}

fmm_status validate_core(const Plan& pl, int64_t m, int64_t n, int64_t k, Operand a, Operand b,
                         float* C, int64_t ldc, void* ws, size_t ws_bytes) {
  const int64_t a_rows = pl.a_mn ? k : m, a_cols = pl.a_mn ? m : k;
  const int64_t b_rows = pl.b_mn ? k : n, b_cols = pl.b_mn ? n : k;
  if (a.ld < std::max<int64_t>(1, a_cols) || b.ld < std::max<int64_t>(1, b_cols) ||
      ldc < std::max<int64_t>(1, n))
    return fail(FMM_ERR_ARG, "leading dimension smaller than the row length");
  if (m == 0 || n == 0) return FMM_OK;
  if (!C) return fail(FMM_ERR_ARG, "C is NULL");
  if (k > 0 && (!a.X || !b.X)) return fail(FMM_ERR_ARG, "an input operand is NULL");
  const size_t c_bytes = static_cast<size_t>(((m - 1) * ldc + n) * 4);
  if (k > 0) {
    const size_t a_span = static_cast<size_t>(((a_rows - 1) * a.ld + a_cols) * elem_bytes(a.type));
    const size_t b_span = static_cast<size_t>(((b_rows - 1) * b.ld + b_cols) * elem_bytes(b.type));
    if (overlaps(C, c_bytes, a.X, a_span) || overlaps(C, c_bytes, b.X, b_span))
      return fail(FMM_ERR_ARG, "C overlaps an input operand");
  }
  const size_t need = (in_place_operand(pl, a) && in_place_operand(pl, b)) ? 0 : pl.ws;
  if (need > 0) {
    if (!ws || ws_bytes < need)
      return fail(FMM_ERR_WORKSPACE, "workspace of " + std::to_string(need) + " bytes required");
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(FMM_ERR_ALIGN, "workspace must be 256-byte aligned");
    if (overlaps(C, c_bytes, ws, need)) return fail(FMM_ERR_ARG, "C overlaps the workspace");
  }
  if (pl.algo == FMM_ALGO_FUSED && k > 0 &&
      (reinterpret_cast<uintptr_t>(a.X) % 16 != 0 || reinterpret_cast<uintptr_t>(b.X) % 16 != 0 ||
       (a.ld * elem_bytes(a.type)) % 16 != 0 || (b.ld * elem_bytes(b.type)) % 16 != 0))
    return fail(FMM_ERR_ALIGN,
                "the fused algorithm needs 16-byte aligned A and B and rows of a multiple of 16 bytes "
                "(lda, ldb multiples of 4 for FP32, of 8 for 16-bit operands)");
  return FMM_OK;
}

// Everything one packed product launches, prepared on the host: the beta pass, the two
// operand-sum passes and the tensor-core kernel's parameter block.
struct PackedJob {
  Plan pl;
  int64_t m = 0, n = 0, k = 0, ldc = 0;
  float alpha = 1.f, beta = 0.f;
  float* C = nullptr;
  int a_type = kInF32, b_type = kInF32;
  SumParams sa, sb;
  TableSumParams ta, tb;  // bases other than Strassen's: sums formed from the product table
  // classical products of 16-bit operands: the tensor-core kernel reads the operand straight
  // from the caller's buffer (no sum pass)
  bool direct_a = false, direct_b = false;
  unsigned* maxbits = nullptr;
  int grid = 0;
  bool has_work = false;  // k > 0 and alpha != 0
  PackedParams params;
  // pipelined plans: one parameter block per top-level product (its 7^(L-1) products)
  std::vector<PackedParams> chunks;
  // store-first plans (beta = 0): one parameter block per launch phase; C is not zeroed
  std::vector<PackedParams> phases;
  // store-first in the ownership mode (one launch; each tile position's products run in order
  // on one worker, each item's C updates complete before the next item's): C is not zeroed
  bool owned_store = false;
};

// Launch phases in which, with beta = 0, the first update of every C block is a store: no
// zeroing pass before the products and no read of C by the first update of each block.  A
// product joins the current phase unless one of its destination blocks is being stored by a
// product already in it; it stores into each of its blocks that no earlier phase has written
// and adds into the others.  Phases run as separate launches in stream order, so every store
// has landed before any addition into its block.  Sets DestEntry::store; returns the product
// lists of the phases (Strassen: 1 + 4 + 2 products at one level, 1 + 12 + 24 + 12 at two).
std::vector<std::vector<int>> plan_store_phases(CommonParams& c) {
  const int R = c.num_products;
  std::vector<int> phase_of(R, -1);
  bool written[kMaxSources] = {};
  std::vector<std::vector<int>> phases;
  int left = R;
  while (left > 0) {
    bool storing[kMaxSources] = {};
    std::vector<int> ph;
    for (int r = 0; r < R; ++r) {
      if (phase_of[r] >= 0) continue;
      bool ok = true;
      for (int d = 0; d < c.prod[r].count; ++d) ok = ok && !storing[c.prod[r].d[d].block];
      if (!ok) continue;
      phase_of[r] = static_cast<int>(phases.size());
      ph.push_back(r);
      --left;
      for (int d = 0; d < c.prod[r].count; ++d) {
        DestEntry& de = c.prod[r].d[d];
        de.store = written[de.block] ? 0 : 1;
        if (de.store) storing[de.block] = true;
      }
    }
    for (int b = 0; b < kMaxSources; ++b) written[b] = written[b] || storing[b];
    phases.push_back(ph);
  }
  return phases;
}

// batched = true: the job joins a batched launch, which never pipelines.
fmm_status prepare_packed(const Plan& plan, int64_t m, int64_t n, int64_t k, float alpha, Operand a,
                          Operand b, float beta, float* C, int64_t ldc, void* ws, const DeviceInfo& dev,
                          const fmm_options* opt, PackedJob& job, bool batched = false) {
  Plan pl = plan;
  // Automatic ownership order (measured on GB300, split3, m = n = 16384): with beta = 0 and
  // short one-level products (h_k <= 512) each tile position's seven products run in order on
  // one worker, so the first product to update a C block stores it and the later updates find
  // the block in L2 (k = 512: 303 against 258 effective TFLOPS with launch phases; k = 1024:
  // 506 against 467).  From h_k = 768 on, and at two levels (49 products per tile position,
  // padded rounds), the launch phases are faster; with the Winograd form (two C updates per
  // product) already at h_k = 512 (8192^2 x 1024: 383 against 411).  Strassen's basis only,
  // the options at their defaults and C rows that TMA addresses; the results are then
  // bitwise reproducible as well.
  const int sf_opt = opt ? opt->store_first : 0;
  const int pipe_opt = opt ? opt->pipeline : 0;
  const int det_opt = opt ? opt->deterministic : 0;
  const int sched_opt = opt ? opt->schedule : 0;
  const int rt_opt = opt ? opt->round_tiles : 0;
  if (!batched && !pl.deterministic && det_opt == 0 && sf_opt == 0 && pipe_opt == 0 && sched_opt == 0 &&
      rt_opt == 0 && beta == 0.0f && pl.algo == FMM_ALGO_PACKED && pl.L == 1 && pl.basis == kBasisStrassen &&
      pl.hk <= 512 &&
      !pl.outer_scaling && reinterpret_cast<uintptr_t>(C) % 16 == 0 && ldc % 4 == 0) {
    pl.deterministic = true;
    pl.schedule = kSchedTileRounds;
  }
  job.pl = pl;
  job.m = m; job.n = n; job.k = k; job.ldc = ldc;
  job.alpha = alpha; job.beta = beta; job.C = C;
  job.a_type = a.type; job.b_type = b.type;
  job.has_work = m > 0 && n > 0 && k > 0 && alpha != 0.0f;
  std::memset(&job.sa, 0, sizeof job.sa);
  std::memset(&job.sb, 0, sizeof job.sb);
  std::memset(&job.ta, 0, sizeof job.ta);
  std::memset(&job.tb, 0, sizeof job.tb);
  std::memset(&job.params, 0, sizeof job.params);
  if (!job.has_work) return FMM_OK;
  const int64_t a_rows = pl.a_mn ? k : m, a_cols = pl.a_mn ? m : k;
  const int64_t b_rows = pl.b_mn ? k : n, b_cols = pl.b_mn ? n : k;
  // (no workspace at all when both operands are read in place: every region stays null)
  uint8_t* wsb = static_cast<uint8_t*>(ws);
  uint16_t* a_hi = wsb ? reinterpret_cast<uint16_t*>(wsb) : nullptr;
  uint16_t* b_hi = wsb ? reinterpret_cast<uint16_t*>(wsb + pl.a_bytes) : nullptr;
  uint16_t* a_lo = wsb && pl.terms == 3 ? reinterpret_cast<uint16_t*>(wsb + pl.a_bytes + pl.b_bytes) : nullptr;
  uint16_t* b_lo = wsb && pl.terms == 3 ? reinterpret_cast<uint16_t*>(wsb + 2 * pl.a_bytes + pl.b_bytes) : nullptr;
  job.maxbits = wsb && pl.scaled ? reinterpret_cast<unsigned*>(wsb + pl.a_bytes + pl.b_bytes) : nullptr;
  // With one product and no sums, the "sum" of a 16-bit operand is the operand itself: the
  // kernel's TMA reads it in place wherever TMA can address it (16-byte aligned base and
  // rows).  Exact FP16 values need no power-of-two panel scaling (their products are exact in
  // the FP32 accumulator), so the scaled variant drops its scaling when both operands are read
  // in place, and reads neither in place otherwise.
  job.direct_a = in_place_operand(pl, a);
  job.direct_b = in_place_operand(pl, b);
  if (pl.scaled && !(job.direct_a && job.direct_b)) job.direct_a = job.direct_b = false;
  if (job.direct_a && job.direct_b) job.maxbits = nullptr;

  SumParams& sa = job.sa;
  sa.X = a.X;
  sa.ldx = a.ld;
  sa.rows = a_rows;
  sa.cols = a_cols;
  sa.hr = pl.a_mn ? pl.hk : pl.hm;
  sa.hc = pl.a_mn ? pl.hm : pl.hk;
  sa.ld_out = pl.lda_w;
  sa.prod_stride = sa.hr * pl.lda_w;
  sa.out_hi = a_hi;
  sa.out_lo = a_lo;
  sa.terms = pl.terms;
  sa.chunk = -1;  // every product (the pipelined path sets one top-level product per pass)
  unsigned* outer_rows = pl.outer_scaling ? reinterpret_cast<unsigned*>(wsb + pl.outer_off) : nullptr;
  sa.row_maxbits = outer_rows;  // rows of A
  sa.vec_ok = (reinterpret_cast<uintptr_t>(a.X) % 16 == 0 && a.ld % 4 == 0) ? 1 : 0;
  SumParams& sb = job.sb;
  sb = sa;
  sb.X = b.X;
  sb.ldx = b.ld;
  sb.rows = b_rows;
  sb.cols = b_cols;
  sb.hr = pl.b_mn ? pl.hk : pl.hn;
  sb.hc = pl.b_mn ? pl.hn : pl.hk;
  sb.ld_out = pl.ldb_w;
  sb.prod_stride = sb.hr * pl.ldb_w;
  sb.out_hi = b_hi;
  sb.out_lo = b_lo;
  sb.row_maxbits = nullptr;
  sb.col_maxbits = outer_rows ? outer_rows + m : nullptr;  // columns of B (and of C)
  sb.vec_ok = (reinterpret_cast<uintptr_t>(b.X) % 16 == 0 && b.ld % 4 == 0) ? 1 : 0;
  if (job.maxbits) {
    sa.maxbits = job.maxbits;
    sa.npanels = static_cast<int32_t>(pl.panels_a);
    sa.panel_w = kBM;
    sa.scale_rows = 1;
    sb.maxbits = job.maxbits + pl.R * pl.panels_a;
    sb.npanels = static_cast<int32_t>(pl.panels_b);
    sb.panel_w = pl.tile_n;
    sb.scale_rows = 0;
  }
  if (pl.basis != kBasisStrassen) {
    // stored block s of the source (row-major in its grid) is operand block (bi, bj), or
    // (bj, bi) when the source holds the operand transposed; its coefficient in product r
    // is that block's entry of U (A) or V (B)
    const std::vector<Product> tprods = make_products(pl.L, pl.basis);
    auto fill_table = [&](TableSumParams& tp, const SumParams& sp, bool is_b, bool transq) -> bool {
      tp.p = sp;
      const int orows = is_b ? pl.gk : pl.gm, ocols = is_b ? pl.gn : pl.gk;
      tp.grid_r = transq ? ocols : orows;
      tp.grid_c = transq ? orows : ocols;
      tp.nprod = pl.R;
      if (tp.grid_r * tp.grid_c > kMaxTableBlocks || pl.R > kMaxTableRank) return false;
      for (int r = 0; r < pl.R; ++r)
        for (const Term& t : is_b ? tprods[r].b : tprods[r].a) {
          const int oi = t.block / ocols, oj = t.block % ocols;
          const int sblk = transq ? oj * tp.grid_c + oi : oi * tp.grid_c + oj;
          tp.coef[sblk][r] = static_cast<int8_t>(t.sign);
        }
      return true;
    };
    if (!fill_table(job.ta, sa, false, pl.a_mn) || !fill_table(job.tb, sb, true, !pl.b_mn))
      return fail(FMM_ERR_UNSUPPORTED, "basis table too large for the table pass");
  }

  PackedParams* pp = &job.params;
  fmm_status st = FMM_OK;
  const int nb = pl.terms == 3 ? 2 : 1;
  // K-major tiles: BK-deep rows, 128-byte swizzle (BK 64) or 64-byte swizzle (BK 32);
  // MN-major tiles: boxes of 64 (m or n) x BK (k), 128-byte swizzle.  Maps over products
  // prod0 .. prod0 + nprod - 1 (the z coordinate counts from prod0).
  const CUtensorMapSwizzle kswz = pl.bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  auto encode_maps = [&](PackedParams* q, int prod0, int nprod) -> fmm_status {
    fmm_status es = FMM_OK;
    for (int t = 0; t < nb && es == FMM_OK; ++t) {
      // in place (L = 0, one product): the caller's buffer and row stride
      void* ab = job.direct_a ? const_cast<void*>(a.X) : (t ? a_lo : a_hi) + prod0 * sa.prod_stride;
      void* bb = job.direct_b ? const_cast<void*>(b.X) : (t ? b_lo : b_hi) + prod0 * sb.prod_stride;
      const int64_t lda_m = job.direct_a ? a.ld : pl.lda_w;
      const int64_t ldb_m = job.direct_b ? b.ld : pl.ldb_w;
      if (pl.a_mn)
        es = encode_3d(&q->tmA[t], ab, pl.hm, pl.hk, nprod, lda_m, 64, pl.bk);
      else
        es = encode_3d(&q->tmA[t], ab, pl.hk, pl.hm, nprod, lda_m, pl.bk, kBM, kswz);
      if (es != FMM_OK) break;
      if (pl.b_mn)
        es = encode_3d(&q->tmB[t], bb, pl.hn, pl.hk, nprod, ldb_m, 64, pl.bk);
      else
        es = encode_3d(&q->tmB[t], bb, pl.hk, pl.hn, nprod, ldb_m, pl.bk,
                       pl.pair ? pl.tile_n / 2 : pl.tile_n, kswz);
    }
    return es;
  };
  st = encode_maps(pp, 0, pl.R);
  const std::vector<Product> prods = make_products(pl.L, pl.basis);
  std::vector<int> live(pl.R);
  for (int r = 0; r < pl.R; ++r) live[r] = r;
  if (st == FMM_OK) st = fill_common(pp->c, pl, prods, live, m, n, alpha, C, ldc, dev, opt, job.grid);
  if (st != FMM_OK) return st;
  // a classical product with beta = 0 writes every element of C exactly once: store it
  pp->c.c_store = (pl.R == 1 && beta == 0.0f) ? 1 : 0;
  if (job.maxbits) {
    pp->c.maxbits_a = job.maxbits;
    pp->c.maxbits_b = job.maxbits + pl.R * pl.panels_a;
    pp->c.panels_a = static_cast<int32_t>(pl.panels_a);
    pp->c.panels_b = static_cast<int32_t>(pl.panels_b);
  }
  // Automatic pipelining (measured on GB300): only for two-level products whose C rows are
  // not 16-byte aligned, with inner blocks of 512..1536 and a large C.  Each launch then adds
  // into 1-2 of C's four quadrants, which eases the contention of the element-wise
  // reductions (+18 % for 30001 x 29999 x 4097); with aligned C it gains nothing (+2 % to
  // -15 % on square and rank-k shapes: seven launches and their ramps cost what the hidden
  // sum passes save).
  if (pl.pipeline_mode == 0 && pl.algo == FMM_ALGO_PACKED && pl.L == 2 && !pp->c.c_tma && !pl.outer_scaling &&
      pl.hk >= 512 &&
      pl.hk <= 1536 && pl.hm >= 2048 && pl.hn >= 2048)
    job.pl.pipeline = true;
  if (batched) job.pl.pipeline = false;
  job.chunks.clear();
  job.phases.clear();
  job.owned_store = false;
  const int sf = opt ? opt->store_first : 0;
  if ((sf == 0 || sf == 2) && beta == 0.0f && pl.R > 1 && !batched && !job.pl.pipeline && pl.deterministic &&
      !pl.outer_scaling && pl.algo == FMM_ALGO_PACKED) {
    // ownership order: the first product (in product order) to update a block stores it
    bool written[kMaxSources] = {};
    for (int r = 0; r < pp->c.num_products; ++r)
      for (int d = 0; d < pp->c.prod[r].count; ++d) {
        DestEntry& de = pp->c.prod[r].d[d];
        de.store = written[de.block] ? 0 : 1;
        written[de.block] = true;
      }
    job.owned_store = true;
  }
  if (sf == 0 || sf == 2) {
    if (beta == 0.0f && pl.R > 1 && !batched && !job.pl.pipeline && !pl.deterministic && !pl.outer_scaling &&
        pl.algo == FMM_ALGO_PACKED) {
      const std::vector<std::vector<int>> ph = plan_store_phases(pp->c);
      const int64_t tiles = static_cast<int64_t>(pp->c.tiles_m) * pp->c.tiles_n;
      job.phases.resize(ph.size(), *pp);
      for (size_t i = 0; i < ph.size(); ++i) {
        PackedParams& q = job.phases[i];
        const int P = static_cast<int>(ph[i].size());
        for (int j = 0; j < kMaxProducts; ++j) q.c.prod[j] = j < P ? pp->c.prod[ph[i][j]] : ProductDests{};
        q.c.num_products = P;
        q.c.num_items = static_cast<int32_t>(P * tiles);
      }
    }
  }
  if (job.pl.pipeline) {
    // top-level product c: products c * P .. c * P + P - 1 (P = 7^(L-1)), kernel-local 0 .. P-1
    const int P = pl.R / 7;
    job.chunks.resize(7, *pp);
    for (int c = 0; c < 7 && st == FMM_OK; ++c) {
      PackedParams& q = job.chunks[c];
      st = encode_maps(&q, c * P, P);
      for (int j = 0; j < kMaxProducts; ++j) {
        q.c.prod[j] = j < P ? pp->c.prod[c * P + j] : ProductDests{};
        q.c.prod[j].sum_index = j;  // this launch's maps start at top-level product c's sums
      }
      q.c.num_products = P;
      const int64_t tiles = static_cast<int64_t>(pp->c.tiles_m) * pp->c.tiles_n;
      q.c.num_items = static_cast<int32_t>(
          pp->c.deterministic ? (tiles + pp->c.round_tiles - 1) / pp->c.round_tiles * pp->c.round_tiles * P
                              : P * tiles);
      if (job.maxbits) {
        q.c.maxbits_a = pp->c.maxbits_a + static_cast<int64_t>(c) * P * pl.panels_a;
        q.c.maxbits_b = pp->c.maxbits_b + static_cast<int64_t>(c) * P * pl.panels_b;
      }
    }
  }
  return st;
}

// Operand-sum passes (A, then B) of one top-level product of a pipelined job on stream s.
fmm_status launch_chunk_sums(const PackedJob& job, int c, const DeviceInfo& dev, cudaStream_t s) {
  const Plan& pl = job.pl;
  SumParams sa = job.sa, sb = job.sb;
  sa.chunk = sb.chunk = c;
  for (int q = 0; q < 4; ++q) {
    // the source of A' stored transposed (a_mn) swaps quadrants (i, j) and (j, i); likewise
    // a K-major B' (stored n x k)
    const int qa = pl.a_mn ? 2 * (q % 2) + q / 2 : q;
    const int qb = !pl.b_mn ? 2 * (q % 2) + q / 2 : q;
    sa.c1[q] = static_cast<int8_t>(basis_u(pl.basis, c, qa));
    sb.c1[q] = static_cast<int8_t>(basis_v(pl.basis, c, qb));
  }
  PhaseScope ps(kPhasePack, s, 2);
  cudaError_t e = launch_operand_sums(sa, pl.L, false, pl.a_mn, job.a_type, pl.bf16 ? 0 : 1, dev.sms, s);
  if (e != cudaSuccess) return cuda_fail(e, "operand-sum pass (A)");
  e = launch_operand_sums(sb, pl.L, true, !pl.b_mn, job.b_type, pl.bf16 ? 0 : 1, dev.sms, s);
  if (e != cudaSuccess) return cuda_fail(e, "operand-sum pass (B)");
  return FMM_OK;
}

// Internal stream and events of the pipelined path, one set per device, created on first use.
// Enqueueing holds g_pipe_mu so that concurrent callers do not interleave their records and
// waits on the shared events.
struct PipeResources {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr;
  cudaEvent_t ready[7] = {};
};
std::mutex g_pipe_mu;
PipeResources g_pipe[64];

fmm_status pipe_resources(int device, PipeResources*& out) {
  if (device < 0 || device >= 64) return fail(FMM_ERR_CUDA, "device index out of range");
  PipeResources& r = g_pipe[device];
  if (!r.side) {
    cudaError_t e = cudaStreamCreateWithFlags(&r.side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming);
    for (int c = 0; c < 7 && e == cudaSuccess; ++c) e = cudaEventCreateWithFlags(&r.ready[c], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      r.side = nullptr;
      return cuda_fail(e, "creating the pipeline stream and events");
    }
  }
  out = &r;
  return FMM_OK;
}

// Pipelined job: beta and the sums of top-level product 0 on s; the sums of products 1..6 on
// the side stream (after everything enqueued on s so far); the tensor-core kernel of each
// top-level product on s once its sums exist.  The last wait joins the side stream into s.
fmm_status launch_pipelined(const PackedJob& job, const DeviceInfo& dev, cudaStream_t s) {
  const Plan& pl = job.pl;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  PipeResources* res = nullptr;
  fmm_status st = pipe_resources(device, res);
  if (st != FMM_OK) return st;
  if (job.beta != 1.0f) {
    PhaseScope ps(kPhaseBeta, s);
    e = launch_beta(job.C, job.m, job.n, job.ldc, job.beta, dev.sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "beta pass");
  }
  if (job.maxbits) {
    e = cudaMemsetAsync(job.maxbits, 0, pl.scale_bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the panel maxima");
  }
  e = cudaEventRecord(res->fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(res->side, res->fork, 0);
  if (e != cudaSuccess) return cuda_fail(e, "forking the pipeline stream");
  st = launch_chunk_sums(job, 0, dev, s);
  for (int c = 1; c < 7 && st == FMM_OK; ++c) {
    st = launch_chunk_sums(job, c, dev, res->side);
    if (st == FMM_OK && (e = cudaEventRecord(res->ready[c], res->side)) != cudaSuccess)
      st = cuda_fail(e, "recording a pipeline event");
  }
  if (st != FMM_OK) return st;
  KernelArgs* ka = new KernelArgs;
  std::memset(ka, 0, sizeof(KernelArgs));
  {
    PhaseScope ps(kPhaseTensor, s, 7);
    for (int c = 0; c < 7 && st == FMM_OK; ++c) {
      if (c > 0 && (e = cudaStreamWaitEvent(s, res->ready[c], 0)) != cudaSuccess) {
        st = cuda_fail(e, "waiting for a pipeline event");
        break;
      }
      ka->one = job.chunks[c];
      e = launch_packed(*ka, pl.tile_n, pl.terms, pl.bf16, pl.a_mn, pl.b_mn, pl.bk, pl.pair, job.grid, s);
      if (e != cudaSuccess) st = cuda_fail(e, "tensor-core pass");
    }
  }
  delete ka;
  return st;
}

// The beta pass and the operand-sum passes of a prepared job (everything before the
// tensor-core kernel).
fmm_status launch_passes(const PackedJob& job, const DeviceInfo& dev, cudaStream_t s) {
  if (job.m == 0 || job.n == 0) return FMM_OK;
  const Plan& pl = job.pl;
  const bool outer = pl.outer_scaling && job.has_work;
  if (outer) {
    // maxima of the rows of A and columns of B, then beta * C into the scaled problem
    PhaseScope ps(kPhaseBeta, s, 3);
    cudaError_t e = launch_outer_maxbits(job.sa.X, job.m, job.k, job.sa.ldx, job.sb.X, job.n, job.sb.ldx,
                                         job.a_type, const_cast<unsigned*>(job.sa.row_maxbits),
                                         const_cast<unsigned*>(job.sb.col_maxbits), dev.sms, s);
    if (e == cudaSuccess && !(job.beta == 0.0f && job.params.c.c_store))
      e = job.beta == 0.0f ? launch_beta(job.C, job.m, job.n, job.ldc, 0.0f, dev.sms, s)
                           : launch_outer_rescale(job.C, job.m, job.n, job.ldc, job.sa.row_maxbits,
                                                  job.sb.col_maxbits, -1, job.beta, dev.sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "outside-scaling passes");
  } else if (job.beta != 1.0f &&
             !(job.has_work && (job.params.c.c_store || !job.phases.empty() || job.owned_store))) {
    PhaseScope ps(kPhaseBeta, s);
    cudaError_t e = launch_beta(job.C, job.m, job.n, job.ldc, job.beta, dev.sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "beta pass");
  }
  if (!job.has_work) return FMM_OK;
  if (job.maxbits) {
    cudaError_t e = cudaMemsetAsync(job.maxbits, 0, pl.scale_bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the panel maxima");
  }
  if (pl.basis != kBasisStrassen) {
    // the sum kernel's full pass carries Strassen's tables; other bases form every product's
    // sums in one pass per operand from the product table
    cudaError_t e;
    {
      PhaseScope ps(kPhasePack, s);
      e = launch_table_sums(job.ta, job.a_type, pl.bf16 ? 0 : 1, dev.sms, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "operand-sum pass (A, basis table)");
    {
      PhaseScope ps(kPhasePack, s);
      e = launch_table_sums(job.tb, job.b_type, pl.bf16 ? 0 : 1, dev.sms, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "operand-sum pass (B, basis table)");
    return FMM_OK;
  }
  cudaError_t e = cudaSuccess;
  if (!job.direct_a) {
    PhaseScope ps(kPhasePack, s);
    e = launch_operand_sums(job.sa, pl.L, false, pl.a_mn, job.a_type, pl.bf16 ? 0 : 1, dev.sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "operand-sum pass (A)");
  if (!job.direct_b) {
    PhaseScope ps(kPhasePack, s);
    e = launch_operand_sums(job.sb, pl.L, true, !pl.b_mn, job.b_type, pl.bf16 ? 0 : 1, dev.sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "operand-sum pass (B)");
  return FMM_OK;
}

// C (m x n) = alpha * A' B' + beta * C with the operand layouts of `pl`.  `a` stores A' as
// m x k (K-major) or k x m (pl.a_mn); `b` stores B' as k x n (pl.b_mn) or n x k.
fmm_status gemm_core(const Plan& pl, int64_t m, int64_t n, int64_t k, float alpha, Operand a,
                     Operand b, float beta, float* C, int64_t ldc, void* ws, size_t ws_bytes,
                     void* stream, const fmm_options* opt) {
  fmm_status st = validate_core(pl, m, n, k, a, b, C, ldc, ws, ws_bytes);
  if (st != FMM_OK || m == 0 || n == 0) return st;
  DeviceInfo dev;
  st = device_info(dev);
  if (st != FMM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  if (pl.algo == FMM_ALGO_FUSED || pl.algo == FMM_ALGO_HYBRID) {
    // beta first: C <- beta * C (beta == 0: C is not read)
    if (beta != 1.0f) {
      PhaseScope ps(kPhaseBeta, s);
      cudaError_t e = launch_beta(C, m, n, ldc, beta, dev.sms, s);
      if (e != cudaSuccess) return cuda_fail(e, "beta pass");
    }
    if (k == 0 || alpha == 0.0f) return FMM_OK;
    if (pl.algo == FMM_ALGO_FUSED) return gemm_fused(pl, m, n, k, alpha, a.X, a.ld, b.X, b.ld, C, ldc, ws, dev, opt, s);
    return gemm_hybrid(pl, m, n, k, alpha, a.X, a.ld, b.X, b.ld, C, ldc, ws, dev, opt, s);
  }

  KernelArgs* ka = new KernelArgs;
  std::memset(ka, 0, sizeof(KernelArgs));
  PackedJob* job = new PackedJob;
  st = prepare_packed(pl, m, n, k, alpha, a, b, beta, C, ldc, ws, dev, opt, *job);
  if (st == FMM_OK && job->pl.pipeline && job->has_work && !job->chunks.empty()) {
    st = launch_pipelined(*job, dev, s);
    delete job;
    delete ka;
    return st;
  }
  if (st == FMM_OK) st = launch_passes(*job, dev, s);
  if (st == FMM_OK && job->has_work) {
    cudaError_t e = cudaSuccess;
    if (job->phases.empty()) {
      ka->one = job->params;
      PhaseScope ps(kPhaseTensor, s);
      e = launch_packed(*ka, pl.tile_n, pl.terms, pl.bf16, pl.a_mn, pl.b_mn, pl.bk, pl.pair, job->grid, s);
    } else {
      // store-first phases, in stream order (each phase's stores land before the next adds)
      PhaseScope ps(kPhaseTensor, s, static_cast<int>(job->phases.size()));
      for (size_t i = 0; i < job->phases.size() && e == cudaSuccess; ++i) {
        ka->one = job->phases[i];
        e = launch_packed(*ka, pl.tile_n, pl.terms, pl.bf16, pl.a_mn, pl.b_mn, pl.bk, pl.pair, job->grid, s);
      }
    }
    if (e != cudaSuccess) st = cuda_fail(e, "tensor-core pass");
    if (st == FMM_OK && pl.outer_scaling) {
      // C out of the scaled problem: exact powers of two per row and column
      PhaseScope ps(kPhaseBeta, s);
      e = launch_outer_rescale(C, m, n, ldc, job->sa.row_maxbits, job->sb.col_maxbits, +1, 1.0f, dev.sms, s);
      if (e != cudaSuccess) st = cuda_fail(e, "outside-scaling pass (C)");
    }
  }
  delete job;
  delete ka;
  return st;
}

}  // namespace

void set_last_error(const std::string& msg) { g_last_error = msg; }

}  // namespace fmm

// Host side of a batched plan: every problem's prepared passes, and per tile width the
// arguments of one batched tensor-core launch whose parameter blocks live in the workspace.
struct fmm_batched_plan {
  struct Group {
    int tile_n = 128;
    int bk = 64;
    bool pair = false;
    int grid = 0;
    fmm::KernelArgs* args = nullptr;
  };
  int device = 0;
  int terms = 3;
  bool bf16 = true;
  fmm::DeviceInfo dev;
  std::vector<fmm::PackedJob*> jobs;
  std::vector<Group> groups;
  ~fmm_batched_plan() {
    for (auto* j : jobs) delete j;
    for (auto& g : groups) delete g.args;
  }
};

using namespace fmm;

namespace fmm {
namespace {

// Dynamic peeling (Section 3.5 names it beside padding): the core m_e x n_e x k_e, each the
// largest multiple of 8 * 2^L not above the size, splits evenly at every level, so its
// Strassen product needs no padding; the strips around it are classical products.
struct PeelPart {
  int64_t r0, c0, k0;  // first row of C / A, first column of C / B, first k of A-columns / B-rows
  int64_t m, n, k;
  int levels;
  bool accumulate;     // beta = 1 (adds to what an earlier part wrote)
};

std::vector<PeelPart> peel_parts(int64_t m, int64_t n, int64_t k, int levels, const fmm_options* opt) {
  // core sizes: multiples of 8 times the basis's block grid in each dimension
  BasisShape sh;
  if (!basis_shape(levels, opt ? opt->basis : 0, sh)) sh = {1 << levels, 1 << levels, 1 << levels, 0};
  const int64_t qm = 8 * sh.gm, qn = 8 * sh.gn, qk = 8 * sh.gk;
  const int64_t me = m / qm * qm, ne = n / qn * qn, ke = k / qk * qk;
  std::vector<PeelPart> parts;
  if (me == 0 || ne == 0 || ke == 0) {  // no core: one classical product
    parts.push_back({0, 0, 0, m, n, k, 0, false});
    return parts;
  }
  parts.push_back({0, 0, 0, me, ne, ke, levels, false});        // Strassen core
  if (ke < k) parts.push_back({0, 0, ke, me, ne, k - ke, 0, true});  // k strip into the core
  if (me < m) parts.push_back({me, 0, 0, m - me, n, k, 0, false});   // bottom rows, full width
  if (ne < n) parts.push_back({0, ne, 0, me, n - ne, k, 0, false});  // right columns of the core rows
  return parts;
}

fmm_options no_fringe(const fmm_options* opt) {
  fmm_options o;
  std::memset(&o, 0, sizeof o);
  if (opt) o = *opt;
  o.fringe = 0;
  return o;
}

}  // namespace
}  // namespace fmm

extern "C" {

size_t fmm_workspace_size_ex(int64_t m, int64_t n, int64_t k, int levels, int variant,
                             const fmm_options* opt) {
  if (opt && opt->fringe == 1 && levels >= 1) {
    const fmm_options o = no_fringe(opt);
    size_t ws = 0;
    for (const PeelPart& pp : peel_parts(m, n, k, levels, &o)) {
      Plan pl;
      if (make_plan(pp.m, pp.n, pp.k, pp.levels, variant, &o, false, true, pl) != FMM_OK)
        return static_cast<size_t>(-1);
      ws = std::max(ws, pl.ws);
    }
    return ws;
  }
  Plan pl;
  if (make_plan(m, n, k, levels, variant, opt, false, true, pl) != FMM_OK) return static_cast<size_t>(-1);
  return pl.ws;
}

size_t fmm_workspace_size(int64_t m, int64_t n, int64_t k, int levels, int variant) {
  return fmm_workspace_size_ex(m, n, k, levels, variant, nullptr);
}

fmm_status fmm_gemm_ex(int64_t m, int64_t n, int64_t k, float alpha, const void* A, int64_t lda,
                       const void* B, int64_t ldb, float beta, float* C, int64_t ldc, int levels,
                       int variant, void* workspace, size_t ws_bytes, void* stream,
                       const fmm_options* opt) {
  g_last_error.clear();
  if (opt && (opt->fringe < 0 || opt->fringe > 1)) return fail(FMM_ERR_ARG, "fringe must be 0 or 1");
  if (opt && opt->fringe == 1 && levels >= 1 && m > 0 && n > 0) {
    // peeled: every part is an ordinary call on sub-views, in order on `stream` (they share
    // the workspace); the parts cover C exactly once, and the k strip adds into the core
    const fmm_options o = no_fringe(opt);
    const std::vector<PeelPart> parts = peel_parts(m, n, k, levels, &o);
    Plan first;
    fmm_status st = make_plan(m, n, k, levels, variant, &o, false, true, first);
    if (st != FMM_OK) return st;
    const size_t eb = elem_bytes(first.in_type);
    for (const PeelPart& pp : parts) {
      Plan pl;
      st = make_plan(pp.m, pp.n, pp.k, pp.levels, variant, &o, false, true, pl);
      if (st != FMM_OK) return st;
      const void* Ap = static_cast<const uint8_t*>(A) + (pp.r0 * lda + pp.k0) * eb;
      const void* Bp = static_cast<const uint8_t*>(B) + (pp.k0 * ldb + pp.c0) * eb;
      float* Cp = C + pp.r0 * ldc + pp.c0;
      st = gemm_core(pl, pp.m, pp.n, pp.k, alpha, Operand{Ap, lda, pl.in_type}, Operand{Bp, ldb, pl.in_type},
                     pp.accumulate ? 1.0f : beta, Cp, ldc, workspace, ws_bytes, stream, &o);
      if (st != FMM_OK) return st;
    }
    return FMM_OK;
  }
  Plan pl;
  fmm_status st = make_plan(m, n, k, levels, variant, opt, false, true, pl);
  if (st != FMM_OK) return st;
  return gemm_core(pl, m, n, k, alpha, Operand{A, lda, pl.in_type}, Operand{B, ldb, pl.in_type}, beta, C,
                   ldc, workspace, ws_bytes, stream, opt);
}

fmm_status fmm_gemm(int64_t m, int64_t n, int64_t k, float alpha, const void* A, int64_t lda,
                    const void* B, int64_t ldb, float beta, float* C, int64_t ldc, int levels,
                    int variant, void* workspace, size_t ws_bytes, void* stream) {
  return fmm_gemm_ex(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, levels, variant, workspace,
                     ws_bytes, stream, nullptr);
}

size_t fmm_workspace_size_backward_ex(int64_t m, int64_t n, int64_t k, int levels, int variant,
                                      const fmm_options* opt) {
  Plan pa, pb;
  if (make_plan(m, k, n, levels, variant, opt, false, false, pa) != FMM_OK ||
      make_plan(k, n, m, levels, variant, opt, true, true, pb) != FMM_OK)
    return static_cast<size_t>(-1);
  return std::max(pa.ws, pb.ws);
}

size_t fmm_workspace_size_backward(int64_t m, int64_t n, int64_t k, int levels, int variant) {
  return fmm_workspace_size_backward_ex(m, n, k, levels, variant, nullptr);
}

fmm_status fmm_gemm_backward_ex(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda,
                                const void* B, int64_t ldb, const float* dC, int64_t lddc, float* dA,
                                int64_t ldda, float* dB, int64_t lddb, int levels, int variant,
                                void* workspace, size_t ws_bytes, void* stream, const fmm_options* opt) {
  g_last_error.clear();
  // dA (m x k) = dC (m x n) B^T: A' = dC stored m x n (K-major), B' = B^T stored as B, k x n
  // (K-major, quadrants transposed).
  if (dA) {
    Plan pl;
    fmm_status st = make_plan(m, k, n, levels, variant, opt, false, false, pl);
    if (st != FMM_OK) return st;
    st = gemm_core(pl, m, k, n, 1.0f, Operand{dC, lddc, kInF32}, Operand{B, ldb, pl.in_type}, 0.0f, dA,
                   ldda, workspace, ws_bytes, stream, opt);
    if (st != FMM_OK) return st;
  }
  // dB (k x n) = A^T dC: A' = A^T stored as A, m x k (MN-major, quadrants transposed),
  // B' = dC stored m x n (MN-major).
  if (dB) {
    Plan pl;
    fmm_status st = make_plan(k, n, m, levels, variant, opt, true, true, pl);
    if (st != FMM_OK) return st;
    st = gemm_core(pl, k, n, m, 1.0f, Operand{A, lda, pl.in_type}, Operand{dC, lddc, kInF32}, 0.0f, dB,
                   lddb, workspace, ws_bytes, stream, opt);
    if (st != FMM_OK) return st;
  }
  return FMM_OK;
}

fmm_status fmm_gemm_backward(int64_t m, int64_t n, int64_t k, const void* A, int64_t lda,
                             const void* B, int64_t ldb, const float* dC, int64_t lddc, float* dA,
                             int64_t ldda, float* dB, int64_t lddb, int levels, int variant,
                             void* workspace, size_t ws_bytes, void* stream) {
  return fmm_gemm_backward_ex(m, n, k, A, lda, B, ldb, dC, lddc, dA, ldda, dB, lddb, levels, variant,
                              workspace, ws_bytes, stream, nullptr);
}

void fmm_tune_default(fmm_tune_table* out) {
  if (!out) return;
  std::memset(out, 0, sizeof *out);
  // measured on GB300, split-BF16 arithmetic, square problems: one level wins from 4096,
  // two levels from 16384 (see the benchmark records)
  out->count = 3;
  out->max_dim[0] = 3072;
  out->levels[0] = 0;
  out->max_dim[1] = 12288;
  out->levels[1] = 1;
  out->max_dim[2] = INT64_MAX;
  out->levels[2] = 2;
}

void fmm_tune_default_ex(int variant, fmm_tune_table* out) {
  if (!out) return;
  if (variant == FMM_BF16 || variant == FMM_F16_SCALED) {
    // 16-bit operands: the classical product reads them in place (no pass at all), while
    // every Strassen level adds operand-sum passes; measured on GB300 over 1024..8192 (and
    // the 256 uneven FP16 products of 1024..8192), classical wins every class
    std::memset(out, 0, sizeof *out);
    out->count = 1;
    out->max_dim[0] = INT64_MAX;
    out->levels[0] = 0;
    return;
  }
  fmm_tune_default(out);
}

fmm_status fmm_tune_select(const fmm_tune_table* tune, int64_t m, int64_t n, int64_t k, int* levels,
                           int* tile_n) {
  fmm_tune_table def;
  if (!tune) {
    fmm_tune_default(&def);
    tune = &def;
  }
  if (tune->count < 1 || tune->count > 8) return fail(FMM_ERR_ARG, "tune table: count must be 1..8");
  const int64_t d = std::min(m, std::min(n, k));
  int i = 0;
  while (i < tune->count - 1 && d > tune->max_dim[i]) ++i;
  if (tune->levels[i] < 0 || tune->levels[i] > 2) return fail(FMM_ERR_ARG, "tune table: levels must be 0..2");
  if (tune->tile_n[i] != 0 && tune->tile_n[i] != 128 && tune->tile_n[i] != 256)
    return fail(FMM_ERR_ARG, "tune table: tile_n must be 0, 128 or 256");
  if (levels) *levels = tune->levels[i];
  if (tile_n) *tile_n = tune->tile_n[i];
  return FMM_OK;
}

}  // extern "C"

namespace fmm {
namespace {

// Per-problem plans of a batch, workspace regions laid out as
// [parameter blocks + work-list offsets per tile width | operand sums of problem 0 | ...].
struct BatchLayout {
  std::vector<Plan> plans;
  std::vector<size_t> ws_off;  // offset of each problem's operand-sum region
  size_t desc_bytes = 0;
  size_t total = 0;
};

fmm_status batch_layout(int count, const int64_t* m, const int64_t* n, const int64_t* k, int variant,
                        const fmm_tune_table* tune, BatchLayout& lay) {
  if (count < 0 || (count > 0 && (!m || !n || !k))) return fail(FMM_ERR_ARG, "bad batch arrays");
  fmm_tune_table def;
  if (!tune) {  // the built-in table of this variant
    fmm_tune_default_ex(variant, &def);
    tune = &def;
  }
  lay.plans.resize(count);
  lay.ws_off.resize(count);
  // parameter blocks (at most two tile-width groups) and item offsets
  lay.desc_bytes = static_cast<size_t>(round_up(static_cast<int64_t>(count) * sizeof(PackedParams), 256)) +
                   2 * static_cast<size_t>(round_up((count + 1) * 4, 256));
  size_t off = lay.desc_bytes;
  for (int p = 0; p < count; ++p) {
    int levels = 0, tile_n = 0;
    fmm_status st = fmm_tune_select(tune, m[p], n[p], k[p], &levels, &tile_n);
    if (st != FMM_OK) return st;
    fmm_options opt;
    std::memset(&opt, 0, sizeof opt);
    opt.algo = FMM_ALGO_PACKED;
    opt.tile_n = tile_n;
    opt.schedule = 1;  // product-major inside each problem
    st = make_plan(m[p], n[p], k[p], levels, variant, &opt, false, true, lay.plans[p]);
    if (st != FMM_OK) return st;
    lay.ws_off[p] = off;
    off += static_cast<size_t>(round_up(static_cast<int64_t>(lay.plans[p].ws), 256));
  }
  lay.total = off;
  return FMM_OK;
}

}  // namespace
}  // namespace fmm

extern "C" {

size_t fmm_batched_workspace_size(int count, const int64_t* m, const int64_t* n, const int64_t* k,
                                  int variant, const fmm_tune_table* tune) {
  BatchLayout lay;
  if (batch_layout(count, m, n, k, variant, tune, lay) != FMM_OK) return static_cast<size_t>(-1);
  return lay.total;
}

fmm_status fmm_batched_plan_create(int count, const int64_t* m, const int64_t* n, const int64_t* k,
                                   const float* alpha, const void* const* A, const int64_t* lda,
                                   const void* const* B, const int64_t* ldb, const float* beta,
                                   float* const* C, const int64_t* ldc, int variant,
                                   const fmm_tune_table* tune, void* workspace, size_t ws_bytes,
                                   fmm_batched_plan** plan_out) {
  g_last_error.clear();
  if (!plan_out) return fail(FMM_ERR_ARG, "plan pointer is NULL");
  *plan_out = nullptr;
  if (count > 0 && (!alpha || !A || !lda || !B || !ldb || !beta || !C || !ldc))
    return fail(FMM_ERR_ARG, "a batch array is NULL");
  BatchLayout lay;
  fmm_status st = batch_layout(count, m, n, k, variant, tune, lay);
  if (st != FMM_OK) return st;
  if (lay.total > 0 && (!workspace || ws_bytes < lay.total))
    return fail(FMM_ERR_WORKSPACE, "batched workspace of " + std::to_string(lay.total) + " bytes required");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(FMM_ERR_ALIGN, "workspace must be 256-byte aligned");
  DeviceInfo dev;
  st = device_info(dev);
  if (st != FMM_OK) return st;
  fmm_batched_plan* plan = new fmm_batched_plan;
  plan->dev = dev;
  cudaGetDevice(&plan->device);
  uint8_t* wsb = static_cast<uint8_t*>(workspace);
  for (int p = 0; p < count && st == FMM_OK; ++p) {
    const Plan& pl = lay.plans[p];
    plan->terms = pl.terms;
    plan->bf16 = pl.bf16;
    const Operand a{A[p], lda[p], pl.in_type}, b{B[p], ldb[p], pl.in_type};
    void* ws = wsb + lay.ws_off[p];
    st = validate_core(pl, m[p], n[p], k[p], a, b, C[p], ldc[p], ws, pl.ws);
    if (st != FMM_OK) break;
    PackedJob* job = new PackedJob;
    plan->jobs.push_back(job);
    st = prepare_packed(pl, m[p], n[p], k[p], alpha[p], a, b, beta[p], C[p], ldc[p], ws, dev, nullptr, *job,
                        /*batched=*/true);
  }
  // one batched tensor-core launch per tile width: upload parameter blocks and item offsets
  // (every problem of a batch has the same CTA-pair setting: the automatic one)
  size_t desc_off = 0;
  const size_t item_off0 = static_cast<size_t>(round_up(static_cast<int64_t>(count) * sizeof(PackedParams), 256));
  for (int tn : {128, 256}) {
    if (st != FMM_OK) break;
    std::vector<PackedParams> descs;
    std::vector<int32_t> begin;
    int64_t items = 0;
    bool pair = false;
    for (PackedJob* job : plan->jobs) {
      if (!job->has_work || job->pl.tile_n != tn) continue;
      pair = job->pl.pair;
      begin.push_back(static_cast<int32_t>(items));
      descs.push_back(job->params);
      items += job->params.c.num_items;
    }
    if (descs.empty()) continue;
    if (items >= (int64_t(1) << 31)) {
      st = fail(FMM_ERR_ARG, "batch has too many work items");
      break;
    }
    begin.push_back(static_cast<int32_t>(items));
    PackedParams* d_desc = reinterpret_cast<PackedParams*>(wsb + desc_off);
    int32_t* d_begin = reinterpret_cast<int32_t*>(wsb + item_off0 + (tn == 128 ? 0 : round_up((count + 1) * 4, 256)));
    cudaError_t e = cudaMemcpy(d_desc, descs.data(), descs.size() * sizeof(PackedParams), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_begin, begin.data(), begin.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "uploading the batched parameter blocks");
      break;
    }
    desc_off += descs.size() * sizeof(PackedParams);
    fmm_batched_plan::Group g;
    g.tile_n = tn;
    for (PackedJob* job : plan->jobs)
      if (job->has_work && job->pl.tile_n == tn) g.bk = job->pl.bk;
    g.args = new KernelArgs;
    std::memset(g.args, 0, sizeof(KernelArgs));
    g.args->many = d_desc;
    g.args->item_begin = d_begin;
    g.args->count = static_cast<int32_t>(descs.size());
    g.args->batched = 1;
    g.args->total_items = static_cast<int32_t>(items);
    g.args->one.c.err = dev.err;
    g.args->one.c.timeout_ns = g_timeout_ns.load();
    g.pair = pair;
    g.grid = pair ? 2 * static_cast<int>(std::min<int64_t>(items, dev.sms / 2))
                  : static_cast<int>(std::min<int64_t>(items, dev.sms));
    plan->groups.push_back(g);
  }
  if (st != FMM_OK) {
    delete plan;
    return st;
  }
  *plan_out = plan;
  return FMM_OK;
}

fmm_status fmm_batched_plan_execute(const fmm_batched_plan* plan, void* stream) {
  g_last_error.clear();
  if (!plan) return fail(FMM_ERR_ARG, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (const PackedJob* job : plan->jobs) {
    fmm_status st = launch_passes(*job, plan->dev, s);
    if (st != FMM_OK) return st;
  }
  for (const auto& g : plan->groups) {
    cudaError_t e;
    {
      PhaseScope ps(kPhaseTensor, s);
      e = launch_packed(*g.args, g.tile_n, plan->terms, plan->bf16, false, true, g.bk, g.pair, g.grid, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batched tensor-core pass");
  }
  return FMM_OK;
}

void fmm_batched_plan_destroy(fmm_batched_plan* plan) { delete plan; }

fmm_status fmm_gemm_batched(int count, const int64_t* m, const int64_t* n, const int64_t* k,
                            const float* alpha, const void* const* A, const int64_t* lda,
                            const void* const* B, const int64_t* ldb, const float* beta,
                            float* const* C, const int64_t* ldc, int variant,
                            const fmm_tune_table* tune, void* workspace, size_t ws_bytes, void* stream) {
  fmm_batched_plan* plan = nullptr;
  fmm_status st = fmm_batched_plan_create(count, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, variant,
                                          tune, workspace, ws_bytes, &plan);
  if (st != FMM_OK) return st;
  st = fmm_batched_plan_execute(plan, stream);
  fmm_batched_plan_destroy(plan);
  return st;
}

const char* fmm_last_error(void) { return g_last_error.c_str(); }

fmm_status fmm_device_status(void* stream) {
  DeviceInfo dev;
  fmm_status st = device_info(dev);
  if (st != FMM_OK) return st;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  unsigned rec[4] = {0, 0, 0, 0};
  e = cudaMemcpy(rec, dev.err, sizeof rec, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
  const unsigned word = rec[0];
  if (word != 0 || rec[1] != 0) {
    const unsigned zero[4] = {0, 0, 0, 0};
    e = cudaMemcpy(dev.err, zero, sizeof zero, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the device error word");
    char buf[320];
    if (word & (kErrPairTmem | kErrBadParams)) {
      std::snprintf(buf, sizeof buf, "device-side check failed: %s (error bits 0x%x)",
                    (word & kErrPairTmem) ? "CTA pair holds different TMEM columns"
                                          : "parameter block names a tensor map outside its table",
                    word);
      return fail(FMM_ERR_CUDA, buf);
    }
    static const char* const kSites[] = {"none", "producer: source slot", "producer: operand stage",
                                         "MMA: accumulator", "MMA: operand stage", "epilogue: accumulator",
                                         "transform: source slot", "transform: operand stage", "teardown"};
    if (rec[1] != 0 && rec[1] < sizeof kSites / sizeof kSites[0])
      std::snprintf(buf, sizeof buf,
                    "device-side wait timed out (error bits 0x%x; first: %s, item %d, k-step %u, block %u)", word,
                    kSites[rec[1]], static_cast<int>(rec[2]), rec[3] & 0xffffu, rec[3] >> 16);
    else
      std::snprintf(buf, sizeof buf, "device-side wait timed out (error bits 0x%x)", word);
    return fail(FMM_ERR_TIMEOUT, buf);
  }
  return FMM_OK;
}

void fmm_set_wait_timeout_ns(uint64_t ns) { g_timeout_ns.store(ns); }

fmm_status fmm_debug_wait_timeout(void* stream) {
  DeviceInfo dev;
  fmm_status st = device_info(dev);
  if (st != FMM_OK) return st;
  cudaError_t e = launch_debug_wait(dev.err, g_timeout_ns.load(), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "debug wait kernel");
  return FMM_OK;
}

// Exports the level-L product table in the layout U[(bi*2^L + bj) * 7^L + r] (likewise V, W),
// so that host-side tests can check it against the Brent equations without a GPU.
int fmm_product_table(int levels, int8_t* U, int8_t* V, int8_t* W) {
  return fmm_product_table_ex(levels, kBasisStrassen, U, V, W);
}

int fmm_basis_shape(int levels, int basis, int* dims) {
  BasisShape sh;
  if (!dims || !basis_shape(levels, basis, sh)) return -1;
  dims[0] = sh.gm;
  dims[1] = sh.gk;
  dims[2] = sh.gn;
  dims[3] = sh.R;
  return 0;
}

int fmm_product_table_ex(int levels, int basis, int8_t* U, int8_t* V, int8_t* W) {
  BasisShape sh;
  if (!U || !V || !W || !basis_shape(levels, basis, sh)) return -1;
  const int R = sh.R;
  std::memset(U, 0, static_cast<size_t>(R) * sh.gm * sh.gk);
  std::memset(V, 0, static_cast<size_t>(R) * sh.gk * sh.gn);
  std::memset(W, 0, static_cast<size_t>(R) * sh.gm * sh.gn);
  const std::vector<Product> prods = make_products(levels, basis);
  for (int r = 0; r < R; ++r) {
    for (const Term& t : prods[r].a) U[t.block * R + r] = static_cast<int8_t>(t.sign);
    for (const Term& t : prods[r].b) V[t.block * R + r] = static_cast<int8_t>(t.sign);
    for (const Term& t : prods[r].c) W[t.block * R + r] = static_cast<int8_t>(t.sign);
  }
  return R;
}

int fmm_store_phases(int levels, int basis, int* phase_of, int8_t* store) {
  BasisShape sh;
  if (!phase_of || !store || levels < 1 || !basis_shape(levels, basis, sh)) return -1;
  const int R = sh.R, nblocks = sh.gm * sh.gn;
  if (R > kMaxProducts || nblocks > kMaxSources) return -1;
  const std::vector<Product> prods = make_products(levels, basis);
  std::unique_ptr<CommonParams> c(new CommonParams);
  std::memset(c.get(), 0, sizeof(CommonParams));
  c->num_products = R;
  for (int r = 0; r < R; ++r) {
    int cnt = 0;
    for (const Term& t : prods[r].c) c->prod[r].d[cnt++].block = t.block;
    c->prod[r].count = cnt;
  }
  const std::vector<std::vector<int>> ph = plan_store_phases(*c);
  std::memset(store, 0, static_cast<size_t>(R) * nblocks);
  for (size_t i = 0; i < ph.size(); ++i)
    for (int r : ph[i]) phase_of[r] = static_cast<int>(i);
  for (int r = 0; r < R; ++r)
    for (int d = 0; d < c->prod[r].count; ++d)
      store[c->prod[r].d[d].block * R + r] = static_cast<int8_t>(c->prod[r].d[d].store);
  return static_cast<int>(ph.size());
}

fmm_status fmm_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return FMM_OK;
}

fmm_status fmm_profile_read(double* ms, int64_t* launches) {
  std::vector<EventPair> recorded;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    recorded.swap(g_prof_pool);
  }
  for (int i = 0; i < kNumPhases; ++i) {
    if (ms) ms[i] = 0.0;
    if (launches) launches[i] = 0;
  }
  fmm_status st = FMM_OK;
  for (EventPair& ev : recorded) {
    cudaError_t e = cudaEventSynchronize(ev.b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev.a, ev.b);
    if (e != cudaSuccess) st = cuda_fail(e, "reading profile events");
    if (ms) ms[ev.phase] += t;
    if (launches) launches[ev.phase] += ev.launches;
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_free.insert(g_prof_free.end(), recorded.begin(), recorded.end());
  return st;
}

const char* fmm_version(void) { return "fmm-gb300 0.1 (sm_103a)"; }

}  // extern "C"
