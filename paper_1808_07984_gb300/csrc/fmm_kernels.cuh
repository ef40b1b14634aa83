// fmm_kernels.cuh -- parameter blocks and device kernels of the Strassen GEMM library.
//
// Two persistent, warp-specialised tcgen05 kernels run every Strassen product ("instance"
// in Section 3.2) of one GEMM call.  A work item is (product r, 128 x BN output tile of the
// h_m x h_n block grid).  Both kernels share the MMA and epilogue roles below:
//
//   MMA role (warp 1)        TMEM allocator and single-thread UMMA issuer: 1 or 3
//                            tcgen05.mma per 16-wide k-slice into a double-buffered FP32
//                            TMEM accumulator;
//   epilogue role (warps 4-7) tcgen05.ld of the finished accumulator, then, for every C
//                            block the product feeds, C_block += alpha * W[c, r] * M_r (the
//                            multi-destination write-back of Section 3.1) by TMA reductions
//                            (or element-wise reductions when C rows are not 16-byte
//                            aligned), clipped at each block's real extent.
//
// They differ in where the operand sums come from:
//   fmm_packed_kernel  the sums were formed by a streaming pass and are TMA-loaded as BF16;
//   fmm_fused_kernel   (fmm_fused.cuh) TMA stages the FP32 source tiles of every block a
//                      product's operands combine, and transform warps add them with their
//                      signs and split/round them into the MMA operand tiles on chip
//                      (Section 3.1: the sums are formed while the tiles are packed).
//
// Every C update is a reduction, so items of different products that feed the same C block
// may run on different SMs at the same time without a race (the atomic-update scheme of
// Section 3.3); beta is applied to C by a separate pass before the products start.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include "ptx.cuh"

namespace fmm {

constexpr int kBM = 128;          // rows of an output tile (UMMA M)
constexpr int kBK = 64;           // k-elements per stage of the fused kernel and the default packed stage
constexpr int kMaxProducts = 49;  // 7^2
constexpr int kMaxDest = 4;       // W_C <= 4 at two levels
constexpr int kMaxSources = 16;   // 4^2 blocks per operand at two levels
constexpr int kThreads = 256;
constexpr int kFusedTileN = 128;  // output tile width of the fused kernel

// Eq. (3), Section 3: the seven products of one-level Strassen.  Quadrant q = 2*row + col
// (Eq. 2).  strassen_u(r, q): coefficient of A_q in the A-operand of product r; strassen_v:
// of B_q in its B-operand; strassen_w: coefficient with which M_r is added into C_q.
__host__ __device__ constexpr int strassen_u(int r, int q) {
  constexpr int8_t t[7][4] = {{1, 0, 0, 1}, {0, 0, 1, 1},  {1, 0, 0, 0}, {0, 0, 0, 1},
                              {1, 1, 0, 0}, {-1, 0, 1, 0}, {0, 1, 0, -1}};
  return t[r][q];
}
__host__ __device__ constexpr int strassen_v(int r, int q) {
  constexpr int8_t t[7][4] = {{1, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, -1}, {-1, 0, 1, 0},
                              {0, 0, 0, 1}, {1, 1, 0, 0}, {0, 0, 1, 1}};
  return t[r][q];
}
__host__ __device__ constexpr int strassen_w(int r, int q) {
  constexpr int8_t t[7][4] = {{1, 0, 0, 1},  {0, 0, 1, -1}, {0, 1, 0, 1}, {1, 0, 1, 0},
                              {-1, 1, 0, 0}, {0, 0, 0, 1},  {1, 0, 0, 0}};
  return t[r][q];
}

// The Strassen-Winograd variant (named among the fast-matmul algorithms the primitive can
// carry, Section 6), written per product: each operand and each C update taken directly from
// the quadrants (14 nonzeros in each table; its usual form shares partial sums instead).
__host__ __device__ constexpr int winograd_u(int r, int q) {
  constexpr int8_t t[7][4] = {{1, 0, 0, 0}, {0, 1, 0, 0},  {1, 1, -1, -1}, {0, 0, 0, 1},
                              {0, 0, 1, 1}, {-1, 0, 1, 1}, {1, 0, -1, 0}};
  return t[r][q];
}
__host__ __device__ constexpr int winograd_v(int r, int q) {
  constexpr int8_t t[7][4] = {{1, 0, 0, 0},   {0, 0, 1, 0},   {0, 0, 0, 1}, {1, -1, -1, 1},
                              {-1, 1, 0, 0}, {1, -1, 0, 1}, {0, -1, 0, 1}};
  return t[r][q];
}
__host__ __device__ constexpr int winograd_w(int r, int q) {
  constexpr int8_t t[7][4] = {{1, 1, 1, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, -1, 0},
                              {0, 1, 0, 1}, {0, 1, 1, 1}, {0, 0, 1, 1}};
  return t[r][q];
}
enum Basis : int { kBasisStrassen = 0, kBasisWinograd = 1 };
__host__ __device__ constexpr int basis_u(int basis, int r, int q) {
  return basis == kBasisWinograd ? winograd_u(r, q) : strassen_u(r, q);
}
__host__ __device__ constexpr int basis_v(int basis, int r, int q) {
  return basis == kBasisWinograd ? winograd_v(r, q) : strassen_v(r, q);
}
__host__ __device__ constexpr int basis_w(int basis, int r, int q) {
  return basis == kBasisWinograd ? winograd_w(r, q) : strassen_w(r, q);
}

enum ErrBits : unsigned {
  kErrProducerWait = 1u,
  kErrMmaWait = 2u,
  kErrEpilogueWait = 4u,
  kErrDebugWait = 8u,
  kErrTransformWait = 16u,
  kErrPairTmem = 32u,   // the two CTAs of a pair were given different TMEM columns
  kErrBadParams = 64u,  // a parameter block named a tensor map outside its table
};

// Where a bounded wait gave up first.  The device error record is four words: [0] the error
// bits above, [1] the site of the first wait that gave up (0 = none), [2] its work item,
// [3] its k-step (low 16 bits) and block index (high 16 bits); fmm_device_status reports it.
enum WaitSite : unsigned {
  kSiteProducerSlot = 1,    // producer: a source slot (or operand stage) to become free
  kSiteProducerStage = 2,
  kSiteMmaAcc = 3,          // MMA issuer: the accumulator to be drained by the epilogue
  kSiteMmaStage = 4,        // MMA issuer: an operand stage to be filled
  kSiteEpilogueAcc = 5,     // epilogue: an accumulator to be finished
  kSiteTransformSlot = 6,   // transform: a source slot to be loaded
  kSiteTransformStage = 7,  // transform: an operand stage to be released by the UMMAs
  kSiteTeardown = 8,        // final waits before the CTA retires
};
__device__ __forceinline__ void record_wait_failure(unsigned int* err, unsigned site, int item, int kb) {
  if (atomicCAS(err + 1, 0u, site) == 0u) {
    err[2] = static_cast<unsigned>(item);
    err[3] = (static_cast<unsigned>(kb) & 0xffffu) | (blockIdx.x << 16);
  }
}

struct DestEntry {
  int64_t offset;  // element offset of the destination block's origin inside C
  int32_t rows;    // rows of that block that exist in C (<= h_m)
  int32_t cols;    // columns of that block that exist in C (<= h_n)
  float coef;      // alpha * W[c, r]
  int32_t block;   // destination block index bi * 2^L + bj (selects its tensor map)
  int32_t store;   // 1: this is the block's first update (beta = 0): store, do not add
  int32_t pad;
};

struct ProductDests {
  int32_t count;
  int32_t sum_index;  // index of the product's operand sums (3-D tensor maps, panel maxima)
  DestEntry d[kMaxDest];
};

// Kernel parameters of the packed-operand path (operand sums already formed).
enum Schedule : int32_t {
  kSchedProductMajor = 0,  // all tiles of product 0, then product 1, ... (operand reuse)
  kSchedTileRounds = 1,    // each CTA runs every product of one tile in turn (C stays in L2)
};

// Part of the kernel parameters shared by both kernels: work list, destinations, C maps.
struct CommonParams {
  CUtensorMap tmC[kMaxSources];  // one f32 map per destination block, clipped to its extent
  float* C;
  int64_t ldc;
  unsigned int* err;
  uint64_t timeout_ns;
  float alpha;
  int32_t tiles_m, tiles_n, nk, num_items;
  int32_t num_products;
  int32_t schedule;     // Schedule
  int32_t round_tiles;  // kSchedTileRounds: tiles per round (0 = one per worker)
  // ownership: every round holds G tiles (the last one padded with empty items), so worker
  // b applies all R products of its tile, and its epilogue lets an item's C updates complete
  // before the next item's: the C sums come out in one fixed order (bitwise reproducible)
  int32_t deterministic;
  int32_t c_tma;     // write-back by TMA reductions through tmC (C rows 16-byte aligned)
  int32_t c_vec4;    // element-wise path: C rows are 16-byte aligned, vector reductions allowed
  // one product and beta = 0: every output tile has exactly one item, whose write-back stores
  // C instead of adding into it (no beta pass, no read of C)
  int32_t c_store;
  // power-of-two scaling of the operand sums (FP16 variant), else null: panel maxima of the
  // A-operand sums per (product, tile row) and of the B-operand sums per (product, tile column)
  const unsigned int* maxbits_a;
  const unsigned int* maxbits_b;
  int32_t panels_a, panels_b;
  ProductDests prod[kMaxProducts];
};

// Kernel parameters of the packed-operand path (operand sums already formed).
struct PackedParams {
  CUtensorMap tmA[2];  // A-operand sums, hi / lo: 3-D {k, m, product} (MN-major: {m, k, product})
  CUtensorMap tmB[2];  // B-operand sums, hi / lo: 3-D {n, k, product} (K-major: {k, n, product})
  CommonParams c;
};

// Source blocks of one product's operands (fused path).
// Kernels read whole 32-bit words of it: kSrcWordHeader = {na, nb, a_neg, b_neg},
// kSrcWordABlock = a_block[0..3], kSrcWordBBlock = b_block[0..3].
struct alignas(4) ProductSrc {
  int8_t na, nb;         // W_A, W_B (only blocks that exist in A / B are listed)
  uint8_t a_neg, b_neg;  // bit w set: term w enters with coefficient -1
  int8_t a_block[kMaxDest], a_sign[kMaxDest];
  int8_t b_block[kMaxDest], b_sign[kMaxDest];
};
constexpr int kSrcWordHeader = 0, kSrcWordABlock = 1, kSrcWordBBlock = 3;
static_assert(offsetof(ProductSrc, a_neg) == 2 && offsetof(ProductSrc, b_neg) == 3, "ProductSrc header word");
static_assert(offsetof(ProductSrc, a_block) == 4 * kSrcWordABlock, "ProductSrc a_block word");
static_assert(offsetof(ProductSrc, b_block) == 4 * kSrcWordBBlock, "ProductSrc b_block word");

// Kernel parameters of the fused path (operand sums formed on chip).
constexpr int kMaxFusedSources = 28;  // hybrid two-level: 7 top-level sums x 4 quadrants

struct FusedParams {
  CUtensorMap tmSA[kMaxFusedSources];  // FP32 source blocks of A: 2-D {k, m}, box 32 x 128, 128B swizzle
  CUtensorMap tmSB[kMaxFusedSources];  // FP32 source blocks of B: 2-D {n, k}, box 128 x 32, no swizzle
  ProductSrc src[kMaxProducts];
  CommonParams c;
};

// Parameters of the operand-sum pass over one operand (A or B), row-major in and out.
struct SumParams {
  const void* X;       // source matrix, row-major
  int64_t ldx;
  int64_t rows, cols;  // extent of X
  int64_t hr, hc;      // block size along rows / cols of X
  int64_t ld_out;      // row stride of the output (elements, multiple of 8)
  int64_t prod_stride; // elements between consecutive products in the output
  uint16_t* out_hi;
  uint16_t* out_lo;
  float* out_f32;      // terms == 0: the sums are stored unrounded in FP32 here
  int32_t terms;       // 3: split hi/lo, 1: single rounding, 0: FP32
  int32_t vec_ok;      // X base and ldx allow vector loads
  // power-of-two scaling (FP16 operands): per (product, panel) maximum |sum| as float bits;
  // panels are panel_w stored rows (scale_rows) or panel_w stored columns
  unsigned int* maxbits;
  int32_t npanels;
  int32_t panel_w;
  int32_t scale_rows;
  // chunk >= 0 (levels >= 1): form only the products whose top-level index is `chunk`, with
  // top-level coefficients c1[q] (already mapped through the transposed-source rule)
  int32_t chunk;
  int8_t c1[4];
  // outside power-of-two scaling (or null): float bits of max |x| per source row / column;
  // each element is multiplied by 2^-e of its row (row_maxbits) or column (col_maxbits)
  const unsigned int* row_maxbits;
  const unsigned int* col_maxbits;
};

// Exponent e of a row's or column's largest magnitude (float bits): max in [2^e, 2^(e+1)),
// e = 0 for an all-zero (or non-finite) vector; subnormal maxima count as 2^-126.
__host__ __device__ inline int outer_exp(unsigned int maxbits) {
  if (maxbits == 0) return 0;
  const int f = static_cast<int>((maxbits >> 23) & 0xffu);
  if (f == 0xff) return 0;
  return (f == 0 ? 1 : f) - 127;
}

// Shift s of a panel whose largest |sum| has float bits `maxbits`: the sums are stored as
// sum * 2^-s, which puts the panel maximum in [2^14, 2^15) (FP16 normal range, no overflow);
// s = 0 for an all-zero panel.  The epilogue multiplies by 2^(s_A + s_B) exactly.
__host__ __device__ inline int panel_shift(unsigned int maxbits) {
  if (maxbits == 0) return 0;
  int e = static_cast<int>((maxbits >> 23) & 0xffu);
  if (e == 0) e = 1;          // subnormal maximum: treat as 2^-126
  if (e == 0xff) return 0;    // Inf / NaN: leave unscaled
  return (e - 127) - 14;
}

// Grouped raster of the tile grid: 8 tile-rows at a time, column-major inside the group, so
// that concurrently running CTAs share operand panels in L2.
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int& tm, int& tn) {
  constexpr int G = 8;
  const int group_size = G * tiles_n;
  const int g = t / group_size;
  const int first_m = g * G;
  const int gm = min(tiles_m - first_m, G);
  const int in_g = t - g * group_size;
  tm = first_m + in_g % gm;
  tn = in_g / gm;
}

// Work item -> (product r, tile row tm, tile column tn).  Worker b runs items b, b + W, ...
// (W = number of workers).  kSchedProductMajor: item = r * tiles + t.  kSchedTileRounds: tiles
// are taken G at a time (G = round_tiles, or W); within a round the item index is
// r * G + (t - round start), so the workers run all R products of G tiles before the next
// round (with G = W, worker b runs products 0..R-1 of one tile back to back), and the C
// blocks of a round can stay in L2; the last, partial round is spread product by product.
// `workers` is the number of independent item streams: CTAs, or CTA pairs of the pair kernel.
__device__ __forceinline__ bool decode_item(int item, const CommonParams& p, int& r, int& tm, int& tn,
                                            int workers) {
  const int tiles = p.tiles_m * p.tiles_n;
  int t;
  if (p.schedule == kSchedTileRounds) {
    const int G = p.round_tiles > 0 ? p.round_tiles : workers, R = p.num_products;
    // ownership: every round is full (items past the last tile are empty)
    const int full = p.deterministic ? (tiles + G - 1) / G : tiles / G;
    const int items_full = full * G * R;
    if (item < items_full) {
      const int j = item / (G * R);
      const int w = item - j * G * R;
      r = w / G;
      t = j * G + (w - r * G);
    } else {
      const int i2 = item - items_full;
      const int rem = tiles - full * G;
      r = i2 / rem;
      t = full * G + (i2 - r * rem);
    }
  } else {
    r = item / tiles;
    t = item - r * tiles;
  }
  if (t >= tiles) return false;  // padding of an ownership round
  tile_coords(t, p.tiles_m, p.tiles_n, tm, tn);
  return true;
}


// Kernel arguments of the packed path: one problem held in parameter space, or a batch of
// problems whose parameter blocks live in global memory (uploaded by the host before the
// launch), with item_begin[p] the first global work item of problem p.
struct KernelArgs {
  PackedParams one;
  const PackedParams* many;
  const int32_t* item_begin;  // count + 1 entries
  int32_t count;
  int32_t batched;
  int32_t total_items;
};

__device__ __forceinline__ const PackedParams& problem_of(const KernelArgs& a, int item, int& local) {
  if (!a.batched) {
    local = item;
    return a.one;
  }
  int lo = 0, hi = a.count - 1;  // last problem whose first item is <= item
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.item_begin[mid] <= item) lo = mid; else hi = mid - 1;
  }
  local = item - a.item_begin[lo];
  return a.many[lo];
}

// Work-list views used by the shared roles: the number of global items and, for one item,
// its problem's CommonParams and the item's index inside that problem.
struct OneProblem {
  const CommonParams* c;
  __device__ int num_items() const { return c->num_items; }
  __device__ const CommonParams& get(int item, int& local) const {
    local = item;
    return *c;
  }
};
struct PackedWork {
  const KernelArgs* a;
  __device__ int num_items() const { return a->batched ? a->total_items : a->one.c.num_items; }
  __device__ const CommonParams& get(int item, int& local) const { return problem_of(*a, item, local).c; }
};

// Byte layout of one operand stage (both kernels): [A hi | B hi | A lo | B lo].  A tile:
// 128 (m) x 64 (k) K-major, or (MN-major) two 64 (m) x 64 (k) boxes; B tile: 64 (k) x BNL
// MN-major as BNL/64 boxes of 64 (n) x 64 (k), or BNL x 64 K-major; 128-byte swizzle.  BNL
// is the tile width BN, or BN / 2 for one CTA of a CTA pair (which holds half of B).
template <int BN, int TERMS, int BK = kBK, int BNL = BN>
struct StageLayout {
  static_assert(BK == 64 || BK == 32, "k-step of 64 (128-byte swizzle) or 32 (64-byte swizzle)");
  static constexpr uint32_t kABytes = kBM * BK * 2;
  static constexpr uint32_t kBBytes = BNL * BK * 2;
  static constexpr uint32_t kBytes = (TERMS == 3 ? 2u : 1u) * (kABytes + kBBytes);
  static constexpr uint32_t kAHi = 0, kBHi = kABytes, kALo = kABytes + kBBytes,
                            kBLo = 2 * kABytes + kBBytes;
};

constexpr uint32_t kEpiBytes = 4 * 2 * 4096;  // epilogue staging: 4 warps x 2 x (32 x 32 FP32)

// ------------------------------------------------------------------- MMA role
// Single thread.  For each item: wait for a free accumulator, then for each k-step wait for
// the operand stage, issue 4 k16 slices x (1 or 3) UMMAs, and release the stage; finally
// signal the epilogue.  Returns false if a wait gave up.
// K-major descriptor of a tile with BK-deep rows (128-byte swizzle for 64, 64-byte for 32).
template <int BK>
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t addr) {
  return BK == 64 ? make_sdesc_kmajor_sw128(addr) : make_sdesc_kmajor_sw64(addr);
}

//
// PAIR: the thread runs in the even CTA of a CTA pair and issues 256-row pair UMMAs (each
// CTA contributes 128 rows of A and half of B, and receives its 128 rows of the accumulator);
// its commits arrive on the barriers of both CTAs, and the accumulator is free again once the
// epilogues of both CTAs have released it.
template <int BN, int TERMS, int STAGES, bool BF16, bool A_MN, bool B_MN, class Work, int BK = kBK,
          bool PAIR = false>
__device__ __forceinline__ bool mma_role(const Work& work, uint8_t* smem, uint64_t* full,
                                         uint64_t* empty, uint64_t* acc_full, uint64_t* acc_empty,
                                         uint32_t tmem_base, volatile int* abort_flag,
                                         uint64_t timeout_ns) {
  using SL = StageLayout<BN, TERMS, BK, PAIR ? BN / 2 : BN>;
  constexpr uint32_t kMnAtom = BK * 128;  // MN-major: bytes between 64-wide atoms along M / N
  constexpr uint32_t idesc = make_idesc_f16(PAIR ? 2 * kBM : kBM, BN, BF16, A_MN, B_MN);
  int stage = 0;
  uint32_t phase = 0;
  int it = 0;
  const int total = work.num_items();
  const int first = PAIR ? static_cast<int>(blockIdx.x >> 1) : static_cast<int>(blockIdx.x);
  const int stride = PAIR ? static_cast<int>(gridDim.x >> 1) : static_cast<int>(gridDim.x);
  auto acc_free = [&](int j) {
    const uint32_t bar = smem_u32(&acc_empty[j & 1]);
    const uint32_t par = ((j >> 1) & 1) ^ 1u;
    return PAIR ? mbar_wait_cluster(bar, par, timeout_ns, abort_flag) : mbar_wait(bar, par, timeout_ns, abort_flag);
  };
  for (int item = first; item < total; item += stride) {
    int local;
    const CommonParams& p = work.get(item, local);
    int r_, tm_, tn_;
    if (!decode_item(local, p, r_, tm_, tn_, stride)) continue;  // empty item
    const int acc = it & 1;
    if (!acc_free(it)) return false;
    tc_fence_after();
    const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * BN);
    for (int kb = 0; kb < p.nk; ++kb) {
      if (!mbar_wait(smem_u32(&full[stage]), phase, timeout_ns, abort_flag)) return false;
      tc_fence_after();
      uint8_t* st = smem + stage * SL::kBytes;
      const uint64_t da_hi = A_MN ? make_sdesc_mnmajor_sw128(smem_u32(st + SL::kAHi), kMnAtom, 1024)
                                  : kmajor_desc<BK>(smem_u32(st + SL::kAHi));
      const uint64_t da_lo = A_MN ? make_sdesc_mnmajor_sw128(smem_u32(st + SL::kALo), kMnAtom, 1024)
                                  : kmajor_desc<BK>(smem_u32(st + SL::kALo));
      const uint64_t db_hi = B_MN ? make_sdesc_mnmajor_sw128(smem_u32(st + SL::kBHi), kMnAtom, 1024)
                                  : kmajor_desc<BK>(smem_u32(st + SL::kBHi));
      const uint64_t db_lo = B_MN ? make_sdesc_mnmajor_sw128(smem_u32(st + SL::kBLo), kMnAtom, 1024)
                                  : kmajor_desc<BK>(smem_u32(st + SL::kBLo));
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        // K-major: 16 elements = 32 bytes inside the swizzle row; MN-major: 16 k-rows = two
        // 1024-byte atoms.  Descriptor start addresses are encoded >> 4.
        const uint64_t ka = A_MN ? static_cast<uint64_t>(kk * 128) : static_cast<uint64_t>(kk * 2);
        const uint64_t kb16 = B_MN ? static_cast<uint64_t>(kk * 128) : static_cast<uint64_t>(kk * 2);
        if (PAIR) {
          umma_f16_ss_pair(d_tmem, da_hi + ka, db_hi + kb16, idesc, (kb | kk) != 0 ? 1u : 0u);
          if (TERMS == 3) {
            umma_f16_ss_pair(d_tmem, da_hi + ka, db_lo + kb16, idesc, 1u);
            umma_f16_ss_pair(d_tmem, da_lo + ka, db_hi + kb16, idesc, 1u);
          }
        } else {
          umma_f16_ss(d_tmem, da_hi + ka, db_hi + kb16, idesc, (kb | kk) != 0 ? 1u : 0u);
          if (TERMS == 3) {
            umma_f16_ss(d_tmem, da_hi + ka, db_lo + kb16, idesc, 1u);
            umma_f16_ss(d_tmem, da_lo + ka, db_hi + kb16, idesc, 1u);
          }
        }
      }
      if (PAIR)
        umma_commit_pair(smem_u32(&empty[stage]), 3);
      else
        umma_commit(smem_u32(&empty[stage]));
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1u;
      }
    }
    if (PAIR)
      umma_commit_pair(smem_u32(&acc_full[acc]), 3);
    else
      umma_commit(smem_u32(&acc_full[acc]));
    ++it;
  }
  // pair: both epilogues have released both accumulators before the CTAs may retire
  if (PAIR && (!acc_free(it) || !acc_free(it + 1))) return false;
  return true;
}

// -------------------------------------------------------------- epilogue role
// Warps 4..7.  Each warp owns TMEM lanes 32q..32q+31 (rows of the tile) and two 4 KB
// staging buffers: a 32 x 32 FP32 block is written there in the 128-byte swizzled layout and
// added into every destination block by TMA reductions.  Returns false if a wait gave up.
//
// PAIR: the CTA with rank `rank` of a pair owns rows 128 * rank .. + 127 of each 256-row pair
// tile; each warp releases the accumulator with one arrival on the even CTA's barrier.
// NACC: accumulators in TMEM (2: double-buffered at columns acc * BN; 1: one at column 0).
template <int BN, class Work, bool PAIR = false, int NACC = 2>
__device__ __forceinline__ bool epilogue_role(const Work& work, uint8_t* epi_smem,
                                              uint64_t* acc_full, uint64_t* acc_empty,
                                              uint32_t tmem_base, volatile int* abort_flag,
                                              uint64_t timeout_ns, int warp, int lane, int rank = 0) {
  const int q = warp & 3;  // TMEM lane quarter this warp may access
  const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
  uint8_t* stage_base = epi_smem + q * 8192;
  int buf = 0;
  int it = 0;
  bool ok = true;
  const int total = work.num_items();
  const int first = PAIR ? static_cast<int>(blockIdx.x >> 1) : static_cast<int>(blockIdx.x);
  const int stride = PAIR ? static_cast<int>(gridDim.x >> 1) : static_cast<int>(gridDim.x);
  for (int item = first; item < total; item += stride) {
    int local;
    const CommonParams& p = work.get(item, local);
    int r, tm, tn;
    if (!decode_item(local, p, r, tm, tn, stride)) continue;  // empty item
    const int acc = NACC == 2 ? (it & 1) : 0;
    const uint32_t acc_par = NACC == 2 ? ((it >> 1) & 1) : (it & 1);
    ++it;
    if (!mbar_wait(smem_u32(&acc_full[acc]), acc_par, timeout_ns, abort_flag)) {
      if (lane == 0) record_wait_failure(p.err, kSiteEpilogueAcc, item, 0);
      ok = false;
      break;
    }
    tc_fence_after();
    // Registers for everything the write-back loops read: `p` may live in global memory
    // (batched launch), so the compiler would reload it after every global reduction.
    const ProductDests pd = p.prod[r];
    const CUtensorMap* const tmC = p.tmC;
    float* const Cm = p.C;
    const int64_t ldc = p.ldc;
    const bool c_tma = p.c_tma != 0;
    const bool c_store = p.c_store != 0;
    const float alpha = p.alpha;
    const int tm_cta = PAIR ? 2 * tm + rank : tm;  // 128-row tile of this CTA
    const int row0 = tm_cta * kBM + q * 32;
    // undo the operand scaling of this (product, tile) exactly: 2^(s_A + s_B); rows past the
    // last A panel (odd CTA of a last, half-empty pair tile) are zero and need none
    const int shift = (p.maxbits_a && tm_cta < p.panels_a)
                          ? panel_shift(p.maxbits_a[pd.sum_index * p.panels_a + tm_cta]) +
                                panel_shift(p.maxbits_b[pd.sum_index * p.panels_b + tn])
                          : 0;
    // destinations are grouped by the sign of W[c, r] (coef = alpha * W[c, r])
    auto wneg = [&](const DestEntry& de) { return ((de.coef < 0.f) != (alpha < 0.f)) ? 1 : 0; };
    bool has_sign[2] = {false, false};
#pragma unroll
    for (int d = 0; d < kMaxDest; ++d)
      if (d < pd.count) has_sign[wneg(pd.d[d])] = true;
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
      float v[32];
      tmem_ld_32x32b_x32(tmem_base + lane_off + static_cast<uint32_t>(acc * BN + c), v);
      if (c + 32 == BN) {
        // every TMEM read of this accumulator is complete: hand it back to the MMA warp
        tc_fence_before();
        if (PAIR) {
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(mapa_shared(smem_u32(&acc_empty[acc]), 0));
        } else {
          mbar_arrive(smem_u32(&acc_empty[acc]));
        }
      }
      const int col0 = tn * BN + c;
#pragma unroll 1
      for (int sg = 0; sg < 2; ++sg) {
        if (!has_sign[sg]) continue;
        const float cf = ldexpf(sg ? -alpha : alpha, shift);
        uint8_t* sb = stage_base + buf * 4096;
        if (lane == 0) bulk_wait_group_read<1>();  // this buffer's previous reductions read it
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 val = make_float4(cf * v[4 * j], cf * v[4 * j + 1], cf * v[4 * j + 2],
                                         cf * v[4 * j + 3]);
          *reinterpret_cast<float4*>(sb + lane * 128 + ((j ^ (lane & 7)) << 4)) = val;
        }
        if (c_tma) {
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
#pragma unroll
            for (int d = 0; d < kMaxDest; ++d) {
              const DestEntry& de = pd.d[d];
              if (d >= pd.count || wneg(de) != sg) continue;
              if (c_store || de.store)
                tma_store_2d(&tmC[de.block], smem_u32(sb), col0, row0);
              else
                tma_reduce_add_2d(&tmC[de.block], smem_u32(sb), col0, row0);
            }
            bulk_commit_group();
          }
        } else {
          // C rows not 16-byte aligned: read the staged 32 x 32 block back transposed, so
          // that lane j adds column col0 + j and every instruction covers 32 consecutive
          // floats of one row.
          __syncwarp();
#pragma unroll
          for (int d = 0; d < kMaxDest; ++d) {
            const DestEntry de = pd.d[d];
            if (d >= pd.count || wneg(de) != sg) continue;
            if (col0 + lane >= de.cols) continue;
            float* dst = Cm + de.offset + static_cast<int64_t>(row0) * ldc + col0 + lane;
            const int nrows = min(32, de.rows - row0);
            // two loops, not one with the branch inside: the reduction loop is the hot one
            // (Strassen destinations), and a branch in it slows it measurably
            if (c_store || de.store) {
#pragma unroll 4
              for (int i = 0; i < nrows; ++i) {
                const float x = *reinterpret_cast<const float*>(sb + i * 128 + (((lane >> 2) ^ (i & 7)) << 4) +
                                                                ((lane & 3) << 2));
                dst[static_cast<int64_t>(i) * ldc] = x;
              }
            } else {
#pragma unroll 4
              for (int i = 0; i < nrows; ++i) {
                const float x = *reinterpret_cast<const float*>(sb + i * 128 + (((lane >> 2) ^ (i & 7)) << 4) +
                                                                ((lane & 3) << 2));
                red_add_global_f32(dst + static_cast<int64_t>(i) * ldc, x);
              }
            }
          }
        }
        buf ^= 1;
      }
    }
    // ownership: this item's reductions land before the next item's (same C tiles)
    if (p.deterministic && lane == 0) bulk_wait_group<0>();
  }
  if (lane == 0) bulk_wait_group<0>();  // reductions complete before the CTA retires
  return ok;
}

// Spin for about `ns` nanoseconds (used after a wait gave up, so that copies and UMMAs
// already in flight finish before shared memory and TMEM are released).
__device__ __forceinline__ void drain_pause(uint64_t ns) {
  const uint64_t t0 = globaltimer_ns();
  while (globaltimer_ns() - t0 < ns) {
  }
}

// ------------------------------------------------------------ packed kernel
template <int BN, int TERMS, int STAGES, int BK = kBK, bool PAIR = false>
struct PackedCfg {
  using SL = StageLayout<BN, TERMS, BK, PAIR ? BN / 2 : BN>;
  static constexpr uint32_t kStageBytes = SL::kBytes;
  static constexpr uint32_t kEpiOffset = STAGES * kStageBytes;
  static constexpr uint32_t kBarOffset = kEpiOffset + kEpiBytes;
  static constexpr uint32_t kSmemBytes = kBarOffset + 256 + 1024;  // + barriers + alignment slack
  static constexpr uint32_t kTmemCols = 2 * BN;
};

// PAIR: launched in clusters of two CTAs (a CTA pair).  A work item is then a 256 x BN pair
// tile: the even CTA loads A rows 0..127 and B columns 0..BN/2-1 of it, the odd CTA rows
// 128..255 and columns BN/2..BN-1; both CTAs' loads complete on the even CTA's stage barrier,
// the even CTA's MMA thread issues the pair UMMAs, and each CTA's epilogue writes back its own
// 128 rows.
template <int BN, int TERMS, int STAGES, bool BF16, bool A_MN, bool B_MN, int BK, bool PAIR>
__global__ void __launch_bounds__(kThreads, 1) fmm_packed_kernel(const __grid_constant__ KernelArgs args) {
  constexpr int BNL = PAIR ? BN / 2 : BN;  // columns of the B tile held by this CTA
  using Cfg = PackedCfg<BN, TERMS, STAGES, BK, PAIR>;
  using SL = StageLayout<BN, TERMS, BK, BNL>;
  constexpr uint32_t kMnAtom = BK * 128;
  static_assert(BN % 64 == 0 && BN <= 256 && BNL % 64 == 0, "UMMA N");
  static_assert(Cfg::kTmemCols >= 32 && Cfg::kTmemCols <= 512, "TMEM columns");
  const PackedWork work{&args};
  const uint64_t timeout_ns = args.one.c.timeout_ns;
  unsigned int* err = args.one.c.err;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::kBarOffset);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* acc_full = bars + 2 * STAGES;
  uint64_t* acc_empty = bars + 2 * STAGES + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int rank = PAIR ? static_cast<int>(cluster_ctarank()) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&acc_full[a]), 1);
      // one arrival per epilogue thread, or (pair) per epilogue warp of both CTAs
      mbar_init(smem_u32(&acc_empty[a]), PAIR ? 2 * 4 : 4 * 32);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0 && !args.batched) {
    tma_prefetch_desc(&args.one.tmA[0]);
    tma_prefetch_desc(&args.one.tmB[0]);
    if (TERMS == 3) {
      tma_prefetch_desc(&args.one.tmA[1]);
      tma_prefetch_desc(&args.one.tmB[1]);
    }
  }
  if (warp == 1) {
    __syncwarp();
    if (PAIR) {
      tmem_alloc_pair(smem_u32(tmem_holder), Cfg::kTmemCols);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_holder), Cfg::kTmemCols);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // the peer's barriers are initialised before anyone signals them
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const int first = PAIR ? static_cast<int>(blockIdx.x >> 1) : static_cast<int>(blockIdx.x);
  const int stride = PAIR ? static_cast<int>(gridDim.x >> 1) : static_cast<int>(gridDim.x);
  if (PAIR) {
    // the pair UMMAs write the same TMEM columns in both CTAs: check that both hold them
    if (threadIdx.x == 0 &&
        ld_shared_cluster_u32(mapa_shared(smem_u32(tmem_holder), static_cast<uint32_t>(rank ^ 1))) != tmem_base) {
      atomicOr(err, kErrPairTmem);
      *abort_flag = 1;
    }
    __syncthreads();
  }
  const bool run = !PAIR || *abort_flag == 0;  // the same in both CTAs of a pair

  if (!run) {
    // nothing issued: fall through to the teardown
  } else if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      const int total = work.num_items();
      for (int item = first; ok && item < total; item += stride) {
        int local;
        const PackedParams& pp = problem_of(args, item, local);
        const CommonParams& p = pp.c;
        int r, tm, tn;
        if (!decode_item(local, p, r, tm, tn, stride)) continue;  // empty item
        const int a_row = (PAIR ? 2 * tm + rank : tm) * kBM;  // first A row of this CTA
        const int b_col = tn * BN + rank * BNL;               // first B column of this CTA
        const int z = p.prod[r].sum_index;                    // the product's operand sums
        for (int kb = 0; kb < p.nk; ++kb) {
          if (!mbar_wait(smem_u32(&empty[stage]), phase ^ 1u, timeout_ns, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + stage * Cfg::kStageBytes;
          const uint32_t fb_local = smem_u32(&full[stage]);
          // pair: both CTAs' bytes complete on the even CTA's barrier, which expects them all
          const uint32_t fb = PAIR ? mapa_shared(fb_local, 0) : fb_local;
          if (rank == 0) mbar_arrive_expect_tx(fb_local, (PAIR ? 2 : 1) * Cfg::kStageBytes);
          auto load = [&](uint32_t dst, const CUtensorMap* map, int c0, int c1) {
            if (PAIR)
              tma_load_3d_pair(dst, map, fb, c0, c1, z);
            else
              tma_load_3d(dst, map, fb, c0, c1, z);
          };
          if (A_MN) {
            // A operand sums stored k-rows x m-cols: two boxes of 64 (m) x BK (k)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              load(smem_u32(st + SL::kAHi + j * kMnAtom), &pp.tmA[0], a_row + 64 * j, kb * BK);
              if (TERMS == 3) load(smem_u32(st + SL::kALo + j * kMnAtom), &pp.tmA[1], a_row + 64 * j, kb * BK);
            }
          } else {
            load(smem_u32(st + SL::kAHi), &pp.tmA[0], kb * BK, a_row);
            if (TERMS == 3) load(smem_u32(st + SL::kALo), &pp.tmA[1], kb * BK, a_row);
          }
          if (B_MN) {
            // B operand sums stored k-rows x n-cols: BNL/64 boxes of 64 (n) x BK (k)
#pragma unroll
            for (int j = 0; j < BNL / 64; ++j) {
              load(smem_u32(st + SL::kBHi + j * kMnAtom), &pp.tmB[0], b_col + 64 * j, kb * BK);
              if (TERMS == 3) load(smem_u32(st + SL::kBLo + j * kMnAtom), &pp.tmB[1], b_col + 64 * j, kb * BK);
            }
          } else {
            load(smem_u32(st + SL::kBHi), &pp.tmB[0], kb * BK, b_col);
            if (TERMS == 3) load(smem_u32(st + SL::kBLo), &pp.tmB[1], kb * BK, b_col);
          }
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // pair: every stage release of the peer's MMA thread has arrived before the CTA retires
      for (int i = 0; PAIR && ok && i < STAGES; ++i) {
        ok = mbar_wait(smem_u32(&empty[stage]), phase ^ 1u, timeout_ns, abort_flag);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) {
        atomicOr(err, kErrProducerWait);
        *abort_flag = 1;
        drain_pause(2000000ull);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      if (!mma_role<BN, TERMS, STAGES, BF16, A_MN, B_MN, PackedWork, BK, PAIR>(
              work, smem, full, empty, acc_full, acc_empty, tmem_base, abort_flag, timeout_ns)) {
        atomicOr(err, kErrMmaWait);
        *abort_flag = 1;
        drain_pause(2000000ull);
      }
    }
  } else if (warp >= 4) {
    if (!epilogue_role<BN, PackedWork, PAIR>(work, smem + Cfg::kEpiOffset, acc_full, acc_empty, tmem_base,
                                             abort_flag, timeout_ns, warp, lane, rank)) {
      if (lane == 0) atomicOr(err, kErrEpilogueWait);
      *abort_flag = 1;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // neither CTA retires while the other may still signal it
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    if (PAIR)
      tmem_dealloc_pair(tmem_base, Cfg::kTmemCols);
    else
      tmem_dealloc(tmem_base, Cfg::kTmemCols);
  }
}

}  // namespace fmm
