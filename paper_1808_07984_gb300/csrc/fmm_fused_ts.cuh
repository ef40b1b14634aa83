// fmm_fused_ts.cuh -- Strassen products with the operand sums formed on chip (Section 3.1),
// the A-operand sums held in tensor memory.
//
// Forming the sums on chip moves every source tile through shared memory (TMA write, then the
// transform's read) and, in fmm_fused_kernel, writes both operands' BF16 sums back into shared
// memory for the UMMAs to read again.  Here the A-operand sums never enter shared memory: the
// transform threads store them into tensor memory with tcgen05.st, and the UMMAs take A from
// TMEM (the ".kind::f16 [d], [a_tmem], b_desc" form).  Per CTA and 64-deep k-step that removes
// the A-sum writes (32 KB for split3) and the UMMAs' A reads (48 KB) from shared memory.
//
// CTA pairs (clusters of two CTAs) on 256 x 256 output tiles:
//   warps 0, 2  producers (fused_producer, lane 0 of each; warp 0 loads k half 0, warp 2 half
//               1): one FP32 tile per source block and 32-deep k half into the half's ring of
//               16 KB slots;
//   warps 8-15  transform.  Warps 8-11 form k half 0 of every k-step, warps 12-15 half 1, each
//               group reading the slots of its own ring (the producer loads half h into ring
//               h).  Thread (lane quarter q = warp % 4, lane l) owns A row 32q + l: it adds that row of each A source slot with its
//               sign, splits the 32 sums into BF16 hi / lo and stores them into its CTA's TMEM
//               at the stage's A columns (32 k per half = 16 columns per term).  It also adds
//               8 k-rows x 4 columns of each B source slot and writes the split B sums into the
//               stage's MN-major, 128-byte swizzled B tile in shared memory;
//   warp 1      (even CTA) issues the cta_group::2 UMMAs: A from TMEM (each CTA's 128 rows),
//               B from shared memory (each CTA's 128 columns);
//   warps 4-7   multi-destination write-back (epilogue_role) of the accumulator.
// Transposed sources (the backward products dA = dC B^T and dB = A^T dC, Section 3 on the
// transposed operands): A_MN -- the A operand is stored K-major by rows of k (its source tile
// is 32 k-rows x 128 m, 512-byte rows, loaded like a B tile); each thread gathers its row's 32
// k-values from one column of the tile (conflict-free: a warp reads 32 consecutive words).
// B_KM -- the B operand is stored with n rows of k (its source tile is 128 n-rows x 32 k,
// 128-byte swizzle, loaded like an A tile); thread tb owns n-row tb, adds its row like an A row
// and writes the B-operand tile K-major (128-byte swizzle) for a K-major UMMA descriptor.
// S16 (forward products, one term): the source blocks are the caller's BF16 (or, with F16, FP16)
// operands; a tile of 128 rows x 32 k (64-byte swizzle) or 32 k-rows x 128 n takes half a slot,
// and the transform converts each value to FP32 (exactly) before adding it.
// F16 (one term): FP16 operands with power-of-two scaling -- each product's A-operand sums of
// this CTA's 128-row panel and B-operand sums of the tile's columns are multiplied by 2^-s
// (the panel maxima, p.maxbits_a / maxbits_b, were found by a pass before this kernel) before
// the FP16 rounding, and the epilogue multiplies by 2^(s_A + s_B) exactly.
// TMEM (512 columns): the 256-column accumulator, then kStages A stages of 32 columns per term.
// The accumulator is single-buffered (the A stages take the other half of TMEM): the UMMAs of
// an item start once both epilogues have read the previous item's accumulator out.
#pragma once
#include "fmm_fused.cuh"

namespace fmm {

template <int TERMS>
struct FusedTsCfg {
  static constexpr int kTileN = 2 * kFusedBN;  // UMMA N of the pair tile
  // Shared memory goes to the source slots first: each k half's ring must hold enough bytes in
  // flight to cover the latency of its TMA loads (measured: with three 16 KB slots per half the
  // transform waits on its loads, shared memory at 30 % of its throughput).
  static constexpr int kStages = 2;            // operand stages (A in TMEM, B in shared memory)
  static constexpr int kSlots = 8;             // FP32 source slots: two rings of four, one per k half
  static constexpr uint32_t kBTermBytes = kBK * kFusedBN * 2;  // 64 k x 128 n BF16 per term
  static constexpr uint32_t kStageBytes = (TERMS == 3 ? 2u : 1u) * kBTermBytes;
  static constexpr uint32_t kSlotOffset = kStages * kStageBytes;
  static constexpr uint32_t kEpiOffset = kSlotOffset + kSlots * kSlotBytes;
  static constexpr uint32_t kBarOffset = kEpiOffset + kEpiBytes;
  static constexpr uint32_t kSmemBytes = kBarOffset + 512 + 1024;
  static constexpr uint32_t kTmemCols = 512;
  static constexpr uint32_t kTermCols = kBK / 2;                 // 64 BF16 per row = 32 columns
  static constexpr uint32_t kAStageCols = (TERMS == 3 ? 2u : 1u) * kTermCols;
  static constexpr uint32_t kACol0 = kTileN;                     // A stages after the accumulator
  static_assert(kACol0 + kStages * kAStageCols <= kTmemCols, "TMEM columns");
};

// UMMA issue of the TS kernel (one thread of the even CTA).  Returns false if a wait gave up.
template <int TERMS, bool B_KM, bool F16 = false>
__device__ __forceinline__ bool mma_role_ts(const CommonParams& p, uint8_t* smem, uint64_t* op_full,
                                            uint64_t* op_empty, uint64_t* acc_full, uint64_t* acc_empty,
                                            uint32_t tmem_base, volatile int* abort_flag) {
  using Cfg = FusedTsCfg<TERMS>;
  constexpr int S = Cfg::kStages;
  constexpr uint32_t idesc = make_idesc_f16(2 * kBM, Cfg::kTileN, !F16, false, !B_KM);
  constexpr uint32_t kMnAtom = kBK * 128;  // bytes between 64-wide n atoms of a B tile
  const int first = static_cast<int>(blockIdx.x >> 1), stride = static_cast<int>(gridDim.x >> 1);
  int o = 0;
  uint32_t oph = 0;
  int it = 0;
  for (int item = first; item < p.num_items; item += stride) {
    int r, tm, tn;
    if (!decode_item(item, p, r, tm, tn, stride)) continue;  // empty item
    // one accumulator: both epilogues have read the previous item's out of TMEM
    if (!mbar_wait_cluster(smem_u32(&acc_empty[0]), (it & 1) ^ 1u, p.timeout_ns, abort_flag)) {
      record_wait_failure(p.err, kSiteMmaAcc, item, 0);
      return false;
    }
    tc_fence_after();
    for (int kb = 0; kb < p.nk; ++kb) {
      if (!mbar_wait_cluster(smem_u32(&op_full[o]), oph, p.timeout_ns, abort_flag)) {
        record_wait_failure(p.err, kSiteMmaStage, item, kb);
        return false;
      }
      tc_fence_after();
      uint8_t* st = smem + o * Cfg::kStageBytes;
      // B tile: MN-major (two 64-wide n atoms of 64 k-rows) or K-major (128 n-rows of 64 k)
      const uint64_t db_hi = B_KM ? make_sdesc_kmajor_sw128(smem_u32(st))
                                  : make_sdesc_mnmajor_sw128(smem_u32(st), kMnAtom, 1024);
      const uint64_t db_lo = B_KM ? make_sdesc_kmajor_sw128(smem_u32(st + Cfg::kBTermBytes))
                                  : make_sdesc_mnmajor_sw128(smem_u32(st + Cfg::kBTermBytes), kMnAtom, 1024);
      const uint32_t a_hi = tmem_base + Cfg::kACol0 + static_cast<uint32_t>(o) * Cfg::kAStageCols;
      const uint32_t a_lo = a_hi + Cfg::kTermCols;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        // k16 slice: 8 TMEM columns of A; of B 16 k-rows (two 1024-byte atoms, MN-major) or 32
        // bytes inside the 128-byte rows (K-major), >> 4 encoded
        const uint32_t ka = static_cast<uint32_t>(8 * kk);
        const uint64_t kb16 = static_cast<uint64_t>(B_KM ? kk * 2 : kk * 128);
        umma_f16_ts_pair(tmem_base, a_hi + ka, db_hi + kb16, idesc, (kb | kk) != 0 ? 1u : 0u);
        if (TERMS == 3) {
          umma_f16_ts_pair(tmem_base, a_hi + ka, db_lo + kb16, idesc, 1u);
          umma_f16_ts_pair(tmem_base, a_lo + ka, db_hi + kb16, idesc, 1u);
        }
      }
      umma_commit_pair(smem_u32(&op_empty[o]), 3);
      if (++o == S) {
        o = 0;
        oph ^= 1u;
      }
    }
    umma_commit_pair(smem_u32(&acc_full[0]), 3);
    ++it;
  }
  // both epilogues have read the last accumulator before the CTAs may retire
  if (it > 0 && !mbar_wait_cluster(smem_u32(&acc_empty[0]), (it & 1) ^ 1u, p.timeout_ns, abort_flag)) {
    record_wait_failure(p.err, kSiteTeardown, -1, 0);
    return false;
  }
  return true;
}

// Two 16-bit values of a 32-bit word (the lower address in the low half) as floats: BF16, or FP16
// when F16.  Both conversions are exact.
template <bool F16>
__device__ __forceinline__ void unpack16(uint32_t w, float& lo, float& hi) {
  if (F16) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w));
    lo = f.x;
    hi = f.y;
  } else {
    lo = __uint_as_float(w << 16);
    hi = __uint_as_float(w & 0xFFFF0000u);
  }
}

template <int TERMS, bool A_MN = false, bool B_KM = false, bool F16 = false, bool S16 = false>
__global__ void __launch_bounds__(fused_threads<8>(), 1) fmm_fused_ts_kernel(const __grid_constant__ FusedParams fp) {
  static_assert(!F16 || TERMS == 1, "FP16 operands: one term");
  static_assert(!S16 || (TERMS == 1 && !A_MN && !B_KM), "16-bit source tiles: forward products, one term");
  using Cfg = FusedTsCfg<TERMS>;
  constexpr int S = Cfg::kStages;
  constexpr int NS = Cfg::kSlots;
  const CommonParams& p = fp.c;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::kBarOffset);
  uint64_t* slot_full = bars;
  uint64_t* slot_empty = bars + NS;
  uint64_t* op_full = bars + 2 * NS;
  uint64_t* op_empty = bars + 2 * NS + S;
  uint64_t* acc_full = bars + 2 * NS + 2 * S;
  uint64_t* acc_empty = bars + 2 * NS + 2 * S + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * NS + 2 * S + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  uint8_t* slots = smem + Cfg::kSlotOffset;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int rank = static_cast<int>(cluster_ctarank());

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&slot_full[s]), 1);
      mbar_init(smem_u32(&slot_empty[s]), 4);  // the four transform warps of the ring's k half
    }
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&op_full[s]), 2 * 8);  // the transform warps of both CTAs
      mbar_init(smem_u32(&op_empty[s]), 1);
    }
    mbar_init(smem_u32(&acc_full[0]), 1);
    mbar_init(smem_u32(&acc_empty[0]), 2 * 4);  // the epilogue warps of both CTAs
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    __syncwarp();
    tmem_alloc_pair(smem_u32(tmem_holder), Cfg::kTmemCols);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // the peer's barriers are initialised before anyone signals them
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const int first = static_cast<int>(blockIdx.x >> 1);
  const int stride = static_cast<int>(gridDim.x >> 1);
  // the pair UMMAs use the same TMEM columns in both CTAs: check that both hold them
  if (threadIdx.x == 0 &&
      ld_shared_cluster_u32(mapa_shared(smem_u32(tmem_holder), static_cast<uint32_t>(rank ^ 1))) != tmem_base) {
    atomicOr(p.err, kErrPairTmem);
    *abort_flag = 1;
  }
  __syncthreads();
  const bool run = *abort_flag == 0;  // the same in both CTAs of a pair

  if (!run) {
    // nothing issued: fall through to the teardown
  } else if (warp == 0 || (kFusedTsProducers > 1 && warp == 2)) {
    if (lane == 0 &&
        !fused_producer<NS, true, 2, A_MN, B_KM, kFusedTsProducers, S16 ? kSlotBytes / 2 : kSlotBytes>(
            fp, slots, slot_full, slot_empty, rank, first, stride, abort_flag, warp >> 1)) {
      atomicOr(p.err, kErrProducerWait);
      *abort_flag = 1;
      drain_pause(2000000ull);
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      if (!mma_role_ts<TERMS, B_KM, F16>(p, smem, op_full, op_empty, acc_full, acc_empty, tmem_base, abort_flag)) {
        atomicOr(p.err, kErrMmaWait);
        *abort_flag = 1;
        drain_pause(2000000ull);
      }
    }
  } else if (warp >= 4 && warp < 8) {
    if (!epilogue_role<Cfg::kTileN, OneProblem, true, 1>(OneProblem{&p}, smem + Cfg::kEpiOffset, acc_full,
                                                        acc_empty, tmem_base, abort_flag, p.timeout_ns, warp,
                                                        lane, rank)) {
      if (lane == 0) atomicOr(p.err, kErrEpilogueWait);
      *abort_flag = 1;
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ transform
    const int tw = warp - 8;
    const int g = tw >> 2;             // k half this warp forms
    const int q = tw & 3;              // TMEM lane quarter (= warp % 4)
    const int arow = 32 * q + lane;    // A row of the tile (TMEM lane)
    const int tb = (threadIdx.x - 256) & 127;  // thread within the half's group
    const int bk0 = tb >> 5;           // first B k-row (of 32) of the half: bk0 + 4v, v < 8
    const int nq = tb & 31;            // B columns 4 nq .. 4 nq + 3
    const uint32_t lane_bits = static_cast<uint32_t>(32 * q) << 16;
    constexpr int NPR = NS / 2;        // slots of this half's ring
    int slot = 0;
    uint32_t sph = 0;
    int o = 0;
    uint32_t oph = 0;
    bool ok = true;
    for (int item = first; ok && item < p.num_items; item += stride) {
      int r, tm, tn;
      if (!decode_item(item, p, r, tm, tn, stride)) continue;  // empty item
      const uint32_t hdr = reinterpret_cast<const uint32_t*>(&fp.src[r])[kSrcWordHeader];
      const int na = hdr & 0xff, nb = (hdr >> 8) & 0xff;
      const uint32_t a_neg = (hdr >> 16) & 0xff, b_neg = hdr >> 24;
      // FP16: the shifts of this item's A panel (this CTA's 128 rows) and B panel (tile column)
      int sh_a = 0, sh_b = 0;
      if (F16) {
        const int tm_cta = 2 * tm + rank;
        const int z = p.prod[r].sum_index;  // the product's row of panel maxima
        if (tm_cta < p.panels_a) sh_a = panel_shift(p.maxbits_a[z * p.panels_a + tm_cta]);
        sh_b = panel_shift(p.maxbits_b[z * p.panels_b + tn]);
      }
      for (int kb = 0; ok && kb < p.nk; ++kb) {
        float aA[32];
        float aB[8][4];
#pragma unroll
        for (int e = 0; e < 32; ++e) aA[e] = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v)
#pragma unroll
          for (int e = 0; e < 4; ++e) aB[v][e] = 0.f;
        // this half's slots of the k-step (its own ring): A sources, then B sources
        for (int w = 0; ok && w < na + nb; ++w) {
          const int sidx = g * NPR + slot;
          ok = mbar_wait(smem_u32(&slot_full[sidx]), sph, p.timeout_ns, abort_flag);
          if (!ok) {
            if (lane == 0) record_wait_failure(p.err, kSiteTransformSlot, item, kb);
            break;
          }
          const uint8_t* sl = slots + sidx * kSlotBytes;
          if (w < na) {
            const float sg = ((a_neg >> w) & 1u) ? -1.f : 1.f;
            if (S16) {
              // 128 rows x 32 k of 16-bit values, 64-byte rows, 64-byte swizzle: 16-byte chunk
              // c of the row sits at chunk c ^ ((row >> 1) & 3)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const uint4 x = *reinterpret_cast<const uint4*>(sl + arow * 64 + ((c ^ ((arow >> 1) & 3)) << 4));
                const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  float lo, hi;
                  unpack16<F16>(w[j], lo, hi);
                  aA[8 * c + 2 * j] = fmaf(sg, lo, aA[8 * c + 2 * j]);
                  aA[8 * c + 2 * j + 1] = fmaf(sg, hi, aA[8 * c + 2 * j + 1]);
                }
              }
            } else if (A_MN) {
              // 32 k-rows x 128 m: this row's k-values are one column of the tile
#pragma unroll
              for (int kk = 0; kk < 32; ++kk)
                aA[kk] = fmaf(sg, *reinterpret_cast<const float*>(sl + kk * 512 + arow * 4), aA[kk]);
            } else {
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                const float4 x = *reinterpret_cast<const float4*>(sl + arow * 128 + ((c ^ (arow & 7)) << 4));
                aA[4 * c] = fmaf(sg, x.x, aA[4 * c]);
                aA[4 * c + 1] = fmaf(sg, x.y, aA[4 * c + 1]);
                aA[4 * c + 2] = fmaf(sg, x.z, aA[4 * c + 2]);
                aA[4 * c + 3] = fmaf(sg, x.w, aA[4 * c + 3]);
              }
            }
          } else {
            const float sg = ((b_neg >> (w - na)) & 1u) ? -1.f : 1.f;
            if (B_KM) {
              // 128 n-rows x 32 k, 128-byte swizzle: n-row tb, 32 k-values (aB as 8 x 4 in k order)
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                const float4 x = *reinterpret_cast<const float4*>(sl + tb * 128 + ((c ^ (tb & 7)) << 4));
                aB[c][0] = fmaf(sg, x.x, aB[c][0]);
                aB[c][1] = fmaf(sg, x.y, aB[c][1]);
                aB[c][2] = fmaf(sg, x.z, aB[c][2]);
                aB[c][3] = fmaf(sg, x.w, aB[c][3]);
              }
            } else if (S16) {
              // 32 k-rows x 128 n of 16-bit values, 256-byte rows, unswizzled
#pragma unroll
              for (int v = 0; v < 8; ++v) {
                const uint2 x = *reinterpret_cast<const uint2*>(sl + (bk0 + 4 * v) * 256 + nq * 8);
                float b0, b1, b2, b3;
                unpack16<F16>(x.x, b0, b1);
                unpack16<F16>(x.y, b2, b3);
                aB[v][0] = fmaf(sg, b0, aB[v][0]);
                aB[v][1] = fmaf(sg, b1, aB[v][1]);
                aB[v][2] = fmaf(sg, b2, aB[v][2]);
                aB[v][3] = fmaf(sg, b3, aB[v][3]);
              }
            } else {
#pragma unroll
              for (int v = 0; v < 8; ++v) {
                const float4 x = *reinterpret_cast<const float4*>(sl + (bk0 + 4 * v) * 512 + nq * 16);
                aB[v][0] = fmaf(sg, x.x, aB[v][0]);
                aB[v][1] = fmaf(sg, x.y, aB[v][1]);
                aB[v][2] = fmaf(sg, x.z, aB[v][2]);
                aB[v][3] = fmaf(sg, x.w, aB[v][3]);
              }
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&slot_empty[sidx]));
          if (++slot == NPR) {
            slot = 0;
            sph ^= 1u;
          }
        }
        if (!ok) break;
        // the stage's previous UMMAs (A in TMEM, B in shared memory) have completed
        if (!mbar_wait(smem_u32(&op_empty[o]), oph ^ 1u, p.timeout_ns, abort_flag)) {
          if (lane == 0) record_wait_failure(p.err, kSiteTransformStage, item, kb);
          ok = false;
          break;
        }
        // A sums: k = 32 g .. 32 g + 31 of row arow -> 16 columns per term
        {
          uint32_t hi[16], lo[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (TERMS == 3)
              split2(aA[2 * i], aA[2 * i + 1], hi[i], lo[i]);
            else if (F16)
              hi[i] = pack_f16x2(ldexpf(aA[2 * i], -sh_a), ldexpf(aA[2 * i + 1], -sh_a));
            else
              hi[i] = pack_bf16x2(aA[2 * i], aA[2 * i + 1]);
          }
          const uint32_t ta = tmem_base + lane_bits + Cfg::kACol0 + static_cast<uint32_t>(o) * Cfg::kAStageCols +
                              static_cast<uint32_t>(16 * g);
          tmem_st_32x32b_x16(ta, hi);
          if (TERMS == 3) tmem_st_32x32b_x16(ta + Cfg::kTermCols, lo);
        }
        uint8_t* st = smem + o * Cfg::kStageBytes;
        if (B_KM) {
          // B sums of n-row tb, k = 32 g .. 32 g + 31: 16-byte chunks 4 g .. 4 g + 3 of the
          // row's 128 bytes, K-major 128-byte swizzle
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint32_t off = tb * 128 + (((4 * g + j) ^ (tb & 7)) << 4);
            if (TERMS == 3) {
              uint4 hv, lv;
              split2(aB[2 * j][0], aB[2 * j][1], hv.x, lv.x);
              split2(aB[2 * j][2], aB[2 * j][3], hv.y, lv.y);
              split2(aB[2 * j + 1][0], aB[2 * j + 1][1], hv.z, lv.z);
              split2(aB[2 * j + 1][2], aB[2 * j + 1][3], hv.w, lv.w);
              *reinterpret_cast<uint4*>(st + off) = hv;
              *reinterpret_cast<uint4*>(st + Cfg::kBTermBytes + off) = lv;
            } else {
              uint4 hv;
              hv.x = pack_bf16x2(aB[2 * j][0], aB[2 * j][1]);
              hv.y = pack_bf16x2(aB[2 * j][2], aB[2 * j][3]);
              hv.z = pack_bf16x2(aB[2 * j + 1][0], aB[2 * j + 1][1]);
              hv.w = pack_bf16x2(aB[2 * j + 1][2], aB[2 * j + 1][3]);
              *reinterpret_cast<uint4*>(st + off) = hv;
            }
          }
        }
        // B sums: k-rows 32 g + bk0 + 4 v, columns 4 nq .. + 3, MN-major swizzled
#pragma unroll
        for (int v = 0; !B_KM && v < 8; ++v) {
          const int kk = 32 * g + bk0 + 4 * v;
          const int c = (nq & 15) >> 1;  // 8-wide chunk inside the 64-wide n atom
          const uint32_t off = (nq >> 4) * 8192 + (kk >> 3) * 1024 + (kk & 7) * 128 +
                               ((c ^ (kk & 7)) << 4) + (nq & 1) * 8;
          if (TERMS == 3) {
            uint2 hv, lv;
            split2(aB[v][0], aB[v][1], hv.x, lv.x);
            split2(aB[v][2], aB[v][3], hv.y, lv.y);
            *reinterpret_cast<uint2*>(st + off) = hv;
            *reinterpret_cast<uint2*>(st + Cfg::kBTermBytes + off) = lv;
          } else if (F16) {
            uint2 hv;
            hv.x = pack_f16x2(ldexpf(aB[v][0], -sh_b), ldexpf(aB[v][1], -sh_b));
            hv.y = pack_f16x2(ldexpf(aB[v][2], -sh_b), ldexpf(aB[v][3], -sh_b));
            *reinterpret_cast<uint2*>(st + off) = hv;
          } else {
            uint2 hv;
            hv.x = pack_bf16x2(aB[v][0], aB[v][1]);
            hv.y = pack_bf16x2(aB[v][2], aB[v][3]);
            *reinterpret_cast<uint2*>(st + off) = hv;
          }
        }
        fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
        tmem_wait_st();            // this thread's TMEM stores have completed
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(mapa_shared(smem_u32(&op_full[o]), 0));
        if (++o == S) {
          o = 0;
          oph ^= 1u;
        }
      }
    }
    // every operand-stage release of the even CTA's MMA thread has arrived before the CTA retires
    for (int i = 0; ok && i < S; ++i) {
      ok = mbar_wait(smem_u32(&op_empty[o]), oph ^ 1u, p.timeout_ns, abort_flag);
      if (!ok && lane == 0) record_wait_failure(p.err, kSiteTeardown, -1, i);
      if (++o == S) {
        o = 0;
        oph ^= 1u;
      }
    }
    if (!ok) {
      if (lane == 0) atomicOr(p.err, kErrTransformWait);
      *abort_flag = 1;
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync();  // neither CTA retires while the other may still signal it
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, Cfg::kTmemCols);
  }
}

}  // namespace fmm
