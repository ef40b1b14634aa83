// fmm_fused.cuh -- Strassen products with the operand sums formed on chip (Section 3.1).
//
// For product r the A-operand is P = sum_w sign_w * A_block(w) (W_A terms) and the
// B-operand Q = sum_w sign_w * B_block(w) (W_B terms).  Per 64-deep k-step:
//   warps 0, 2  (lane 0 of each) TMA-load, for each k half (32 deep) and each source block, one FP32 tile
//               into a 4-slot shared-memory ring (A: 128 rows x 32 k, 128-byte swizzle;
//               B: 32 k-rows x 128 n, unswizzled) -- the W_A (W_B) submatrix tiles;
//   warps 8-15  (transform) add every slot into FP32 register accumulators with its sign,
//               then split the sums into BF16 hi / lo (or round once) and store them into
//               the MMA operand stage (A K-major, B MN-major, 128-byte swizzle);
//   warp 1      UMMA issue as in the packed kernel (mma_role);
//   warps 4-7   multi-destination write-back (epilogue_role).
// No workspace: the sums never leave the SM.  A and B are FP32, 16-byte aligned, with
// leading dimensions that are multiples of 4.
//
// PAIR: clusters of two CTAs share a 256 x 256 output tile through cta_group::2 UMMAs.  Each
// CTA stages and sums its own 128 rows of the A-operand and its own 128 columns of the
// B-operand (the same per-CTA shared-memory traffic as a 128 x 128 tile, for twice the
// UMMA work); the transform warps of both CTAs arrive on the even CTA's operand barrier.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include "fmm_kernels.cuh"

namespace fmm {

// 256 threads for the producer / MMA / epilogue roles plus TW transform warps
template <int TW>
constexpr int fused_threads() { return 256 + 32 * TW; }
constexpr int kFusedBN = kFusedTileN;  // columns of the B-operand each CTA forms
constexpr uint32_t kSlotBytes = 16384;
// threads issuing the source-tile loads: lane 0 of warps 0 and 2 (one issuing thread per warp:
// lanes of one warp that wait on different slots hold each other up)
constexpr int kFusedProducers = 2;    // fmm_fused_kernel: slots 0, 2 and 1, 3 of its ring
constexpr int kFusedTsProducers = 2;  // fmm_fused_ts_kernel: one per k-half ring

template <int TERMS, bool PAIR>
struct FusedCfg {
  static constexpr int kTileN = PAIR ? 2 * kFusedBN : kFusedBN;  // UMMA N
  using SL = StageLayout<kTileN, TERMS, kBK, kFusedBN>;
  static constexpr int kOpStages = TERMS == 3 ? 2 : 4;
  static constexpr int kSlots = 4;
  static constexpr uint32_t kSlotOffset = kOpStages * SL::kBytes;
  static constexpr uint32_t kEpiOffset = kSlotOffset + kSlots * kSlotBytes;
  static constexpr uint32_t kBarOffset = kEpiOffset + kEpiBytes;
  static constexpr uint32_t kSmemBytes = kBarOffset + 512 + 1024;
  static constexpr uint32_t kTmemCols = 2 * kTileN;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);  // .x = lo_elem
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack_f16x2(float lo_elem, float hi_elem) {
  const __half2 v = __floats2half2_rn(lo_elem, hi_elem);  // .x = lo_elem
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Split 2 FP32 values into packed BF16x2 hi and lo words: hi = bf16(x), lo = bf16(x - hi).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  hi = pack_bf16x2(x0, x1);
  const float h0 = __uint_as_float(hi << 16);
  const float h1 = __uint_as_float(hi & 0xFFFF0000u);
  lo = pack_bf16x2(x0 - h0, x1 - h1);
}

// Producer of the fused kernels (one thread): for every item, k-step and 32-deep k half, one
// FP32 tile per source block of the product's A-operand (128 rows x 32 k, 128-byte swizzle),
// then per source block of its B-operand (32 k x 128 n, this CTA's columns), each into the next
// slot of a ring.  RINGS = 1: one ring of NS slots for both k halves; RINGS = 2: k half h goes
// to ring h (slots h * NS / 2 .. (h + 1) * NS / 2 - 1), so that every slot -- and its pair of
// barriers -- is only ever consumed by the threads that form that half (a slot shared by two
// consumer groups could be awaited by one group while the other's use of it is still a phase
// behind, which the parity of an mbarrier wait cannot tell apart).  A_MN: the A-operand
// blocks are stored by rows of k (their maps are {m, k}, box 128 x 32); B_KM: the B-operand
// blocks are stored by rows of n (maps {k, n}, box 32 x 128, 128-byte swizzle).
// NPROD threads issue the loads, thread `who` of them (0 <= who < NPROD): one thread loads
// every ring; with two rings and more threads, even `who` load ring 0 and odd ones ring 1; the NSUB = NPROD / RINGS threads of a
// ring take its tiles in turn (the c-th tile of the ring, counted in the ring's order, goes to
// thread c % NSUB, into slot c % NPR).  One issuing thread limits this loader (measured on GB300
// with 16 KB tiles that stay in L2: about 28 bytes per SM and cycle from one thread, 46 from
// two, 50 from four).  NSUB divides NPR, so the threads fill disjoint slots.
// Returns false if a wait gave up or a parameter block named a tensor map outside its table
// (error bit set).
// TILE_BYTES: bytes of one source tile (FP32 tiles fill a 16 KB slot, 16-bit tiles half of it).
template <int NS, bool PAIR, int RINGS = 1, bool A_MN = false, bool B_KM = false, int NPROD = 1,
          uint32_t TILE_BYTES = kSlotBytes>
__device__ __forceinline__ bool fused_producer(const FusedParams& fp, uint8_t* slots, uint64_t* slot_full,
                                               uint64_t* slot_empty, int rank, int first, int stride,
                                               volatile int* abort_flag, int who = 0) {
  static_assert(RINGS == 1 || RINGS == 2, "one ring, or one per k half");
  constexpr int NPR = NS / RINGS;  // slots per ring
  constexpr bool ALL_RINGS = NPROD < RINGS;  // a single thread loads both rings
  constexpr int NSUB = ALL_RINGS ? 1 : NPROD / RINGS;
  static_assert(ALL_RINGS ? NPROD == 1 : (NPROD % RINGS == 0 && NPR % NSUB == 0), "issuing threads per ring");
  const CommonParams& p = fp.c;
  constexpr int TN = PAIR ? 2 * kFusedBN : kFusedBN;
  const int my_ring = RINGS == 2 ? (who & 1) : 0;
  const uint32_t sub = static_cast<uint32_t>(ALL_RINGS ? 0 : (RINGS == 2 ? who >> 1 : who));
  uint32_t cnt[2] = {0, 0};  // tiles of each ring so far
  bool ok = true;
  auto issue = [&](int ring, const CUtensorMap* map, int x, int y, int item, int kb) -> bool {
    if (!ALL_RINGS && ring != my_ring) return true;  // the other ring's threads load it
    const uint32_t c = cnt[ring]++;
    if (c % NSUB != sub) return true;  // another thread of this ring loads it
    const int sidx = ring * NPR + static_cast<int>(c % NPR);
    const uint32_t use = c / NPR;  // earlier fills of this slot
    if (!mbar_wait(smem_u32(&slot_empty[sidx]), (use & 1u) ^ 1u, p.timeout_ns, abort_flag)) {
      record_wait_failure(p.err, kSiteProducerSlot, item, kb);
      return false;
    }
    const uint32_t fb = smem_u32(&slot_full[sidx]);
    mbar_arrive_expect_tx(fb, TILE_BYTES);
    tma_load_2d(smem_u32(slots + sidx * kSlotBytes), map, fb, x, y);
    return true;
  };
  for (int item = first; ok && item < p.num_items; item += stride) {
    int r, tm, tn;
    if (!decode_item(item, p, r, tm, tn, stride)) continue;  // empty item
    // the product's source lists, read once into registers (indexed parameter loads in
    // the loops below would each go to the constant cache)
    const uint32_t* psw = reinterpret_cast<const uint32_t*>(&fp.src[r]);
    const uint32_t hdr = psw[kSrcWordHeader], ablk = psw[kSrcWordABlock], bblk = psw[kSrcWordBBlock];
    const int na = hdr & 0xff, nb = (hdr >> 8) & 0xff;
    // every map index must name one of the kMaxFusedSources maps: refuse the item otherwise
    bool maps_ok = na <= kMaxDest && nb <= kMaxDest;
    for (int w = 0; w < na && maps_ok; ++w) maps_ok = ((ablk >> (8 * w)) & 0xff) < kMaxFusedSources;
    for (int w = 0; w < nb && maps_ok; ++w) maps_ok = ((bblk >> (8 * w)) & 0xff) < kMaxFusedSources;
    if (!maps_ok) {
      atomicOr(p.err, kErrBadParams);
      return false;
    }
    const int a_row = (PAIR ? 2 * tm + rank : tm) * kBM;  // this CTA's rows and columns
    const int b_col = tn * TN + rank * kFusedBN;
    for (int kb = 0; ok && kb < p.nk; ++kb) {
      for (int h = 0; ok && h < 2; ++h) {
        const int ring = RINGS == 2 ? h : 0;
        const int kx = kb * kBK + 32 * h;
        for (int w = 0; ok && w < na; ++w)
          ok = A_MN ? issue(ring, &fp.tmSA[(ablk >> (8 * w)) & 0xff], a_row, kx, item, kb)
                    : issue(ring, &fp.tmSA[(ablk >> (8 * w)) & 0xff], kx, a_row, item, kb);
        for (int w = 0; ok && w < nb; ++w)
          ok = B_KM ? issue(ring, &fp.tmSB[(bblk >> (8 * w)) & 0xff], kx, b_col, item, kb)
                    : issue(ring, &fp.tmSB[(bblk >> (8 * w)) & 0xff], b_col, kx, item, kb);
      }
    }
  }
  return ok;
}

template <int TERMS, int TW, bool PAIR>
__global__ void __launch_bounds__(fused_threads<TW>(), 1) fmm_fused_kernel(const __grid_constant__ FusedParams fp) {
  static_assert(TW == 8 || TW == 16, "transform warps");
  constexpr int NT = 32 * TW;            // transform threads
  constexpr int AU = 512 / NT;           // A units (row, 8-wide k chunk) per thread per k half
  constexpr int BU = 1024 / NT;          // B units (k row, 4 n) per thread per k half
  using Cfg = FusedCfg<TERMS, PAIR>;
  using SL = typename Cfg::SL;
  constexpr int S = Cfg::kOpStages;
  constexpr int NS = Cfg::kSlots;
  constexpr int TN = Cfg::kTileN;
  const CommonParams& p = fp.c;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::kBarOffset);
  uint64_t* slot_full = bars;
  uint64_t* slot_empty = bars + NS;
  uint64_t* op_full = bars + 2 * NS;
  uint64_t* op_empty = bars + 2 * NS + S;
  uint64_t* acc_full = bars + 2 * NS + 2 * S;
  uint64_t* acc_empty = bars + 2 * NS + 2 * S + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * NS + 2 * S + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  uint8_t* slots = smem + Cfg::kSlotOffset;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int rank = PAIR ? static_cast<int>(cluster_ctarank()) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&slot_full[s]), 1);
      mbar_init(smem_u32(&slot_empty[s]), TW);  // one arrival per transform warp
    }
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&op_full[s]), PAIR ? 2 * TW : TW);  // pair: transform warps of both CTAs
      mbar_init(smem_u32(&op_empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&acc_full[a]), 1);
      mbar_init(smem_u32(&acc_empty[a]), PAIR ? 2 * 4 : 4 * 32);
    }
    *abort_flag = 0;
    fence_mbar_init();
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
    if (threadIdx.x == 0 &&
        ld_shared_cluster_u32(mapa_shared(smem_u32(tmem_holder), static_cast<uint32_t>(rank ^ 1))) != tmem_base) {
      atomicOr(p.err, kErrPairTmem);
      *abort_flag = 1;
    }
    __syncthreads();
  }
  const bool run = !PAIR || *abort_flag == 0;  // the same in both CTAs of a pair

  if (!run) {
    // nothing issued: fall through to the teardown
  } else if (warp == 0 || (kFusedProducers > 1 && warp == 2)) {
    // ------------------------------------------------------------ producer
    if (lane == 0 &&
        !fused_producer<NS, PAIR, 1, false, false, kFusedProducers>(fp, slots, slot_full, slot_empty, rank, first,
                                                                    stride, abort_flag, warp >> 1)) {
      atomicOr(p.err, kErrProducerWait);
      *abort_flag = 1;
      drain_pause(2000000ull);
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      if (!mma_role<TN, TERMS, S, true, false, true, OneProblem, kBK, PAIR>(
              OneProblem{&p}, smem, op_full, op_empty, acc_full, acc_empty, tmem_base, abort_flag, p.timeout_ns)) {
        atomicOr(p.err, kErrMmaWait);
        *abort_flag = 1;
        drain_pause(2000000ull);
      }
    }
  } else if (warp >= 4 && warp < 8) {
    if (!epilogue_role<TN, OneProblem, PAIR>(OneProblem{&p}, smem + Cfg::kEpiOffset, acc_full, acc_empty,
                                             tmem_base, abort_flag, p.timeout_ns, warp, lane, rank)) {
      if (lane == 0) atomicOr(p.err, kErrEpilogueWait);
      *abort_flag = 1;
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ transform
    // Thread t (0..NT-1).  A: per k half, row t & 127 and AU of the half's four 8-wide k
    // chunks starting at AU * (t >> 7).  B: per k half, units j = t + NT v (v < BU): k-row
    // j >> 5 of the half, n = 4 * (j & 31) .. + 3.  Every warp reads every slot.
    const int t = threadIdx.x - 256;
    const int arow = t & 127;
    const int acc0 = AU * (t >> 7);
    int slot = 0;
    uint32_t sph = 0;
    int o = 0;
    uint32_t oph = 0;
    bool ok = true;
    for (int item = first; ok && item < p.num_items; item += stride) {
      int r, tm, tn;
      if (!decode_item(item, p, r, tm, tn, stride)) continue;  // empty item
      // counts and sign masks of the product's source terms, read once into registers
      const uint32_t hdr = reinterpret_cast<const uint32_t*>(&fp.src[r])[kSrcWordHeader];
      const int na = hdr & 0xff, nb = (hdr >> 8) & 0xff;
      const uint32_t a_neg = (hdr >> 16) & 0xff, b_neg = hdr >> 24;
      for (int kb = 0; ok && kb < p.nk; ++kb) {
        float aA[2][AU][8];
        float aB[2][BU][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
          for (int u = 0; u < AU; ++u)
#pragma unroll
            for (int e = 0; e < 8; ++e) aA[h][u][e] = 0.f;
#pragma unroll
          for (int v = 0; v < BU; ++v)
#pragma unroll
            for (int e = 0; e < 4; ++e) aB[h][v][e] = 0.f;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          for (int w = 0; w < na; ++w) {
            if (ok) ok = mbar_wait(smem_u32(&slot_full[slot]), sph, p.timeout_ns, abort_flag);
            if (ok) {
              const uint8_t* sl = slots + slot * kSlotBytes;
              const float sg = ((a_neg >> w) & 1u) ? -1.f : 1.f;
#pragma unroll
              for (int u = 0; u < AU; ++u) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                  const int ch = 2 * (acc0 + u) + e;  // 16-byte FP32 chunk of the 128-byte row
                  const float4 x =
                      *reinterpret_cast<const float4*>(sl + arow * 128 + ((ch ^ (arow & 7)) << 4));
                  aA[h][u][4 * e] = fmaf(sg, x.x, aA[h][u][4 * e]);
                  aA[h][u][4 * e + 1] = fmaf(sg, x.y, aA[h][u][4 * e + 1]);
                  aA[h][u][4 * e + 2] = fmaf(sg, x.z, aA[h][u][4 * e + 2]);
                  aA[h][u][4 * e + 3] = fmaf(sg, x.w, aA[h][u][4 * e + 3]);
                }
              }
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(&slot_empty[slot]));
            }
            if (++slot == NS) {
              slot = 0;
              sph ^= 1u;
            }
          }
          for (int w = 0; w < nb; ++w) {
            if (ok) ok = mbar_wait(smem_u32(&slot_full[slot]), sph, p.timeout_ns, abort_flag);
            if (ok) {
              const uint8_t* sl = slots + slot * kSlotBytes;
              const float sg = ((b_neg >> w) & 1u) ? -1.f : 1.f;
#pragma unroll
              for (int v = 0; v < BU; ++v) {
                const int j = t + NT * v;
                const float4 x = *reinterpret_cast<const float4*>(sl + (j >> 5) * 512 + (j & 31) * 16);
                aB[h][v][0] = fmaf(sg, x.x, aB[h][v][0]);
                aB[h][v][1] = fmaf(sg, x.y, aB[h][v][1]);
                aB[h][v][2] = fmaf(sg, x.z, aB[h][v][2]);
                aB[h][v][3] = fmaf(sg, x.w, aB[h][v][3]);
              }
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(&slot_empty[slot]));
            }
            if (++slot == NS) {
              slot = 0;
              sph ^= 1u;
            }
          }
        }
        if (!ok) break;
        // the operand stage must have been consumed by the UMMAs of its previous use
        if (!mbar_wait(smem_u32(&op_empty[o]), oph ^ 1u, p.timeout_ns, abort_flag)) {
          ok = false;
          break;
        }
        uint8_t* st = smem + o * SL::kBytes;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
          for (int u = 0; u < AU; ++u) {
            const int c = 4 * h + acc0 + u;  // 8-wide bf16 chunk of the 64-deep row
            const uint32_t off = arow * 128 + ((c ^ (arow & 7)) << 4);
            if (TERMS == 3) {
              uint4 hv, lv;
              split2(aA[h][u][0], aA[h][u][1], hv.x, lv.x);
              split2(aA[h][u][2], aA[h][u][3], hv.y, lv.y);
              split2(aA[h][u][4], aA[h][u][5], hv.z, lv.z);
              split2(aA[h][u][6], aA[h][u][7], hv.w, lv.w);
              *reinterpret_cast<uint4*>(st + SL::kAHi + off) = hv;
              *reinterpret_cast<uint4*>(st + SL::kALo + off) = lv;
            } else {
              uint4 hv;
              hv.x = pack_bf16x2(aA[h][u][0], aA[h][u][1]);
              hv.y = pack_bf16x2(aA[h][u][2], aA[h][u][3]);
              hv.z = pack_bf16x2(aA[h][u][4], aA[h][u][5]);
              hv.w = pack_bf16x2(aA[h][u][6], aA[h][u][7]);
              *reinterpret_cast<uint4*>(st + SL::kAHi + off) = hv;
            }
          }
#pragma unroll
          for (int v = 0; v < BU; ++v) {
            const int j = t + NT * v;
            const int kk = 32 * h + (j >> 5);  // k-row of the 64-deep stage
            const int nq = j & 31;             // n = 4 nq .. 4 nq + 3
            const int c = (nq & 15) >> 1;      // 8-wide chunk inside the 64-wide n atom
            const uint32_t off = (nq >> 4) * 8192 + (kk >> 3) * 1024 + (kk & 7) * 128 +
                                 ((c ^ (kk & 7)) << 4) + (nq & 1) * 8;
            if (TERMS == 3) {
              uint2 hv, lv;
              split2(aB[h][v][0], aB[h][v][1], hv.x, lv.x);
              split2(aB[h][v][2], aB[h][v][3], hv.y, lv.y);
              *reinterpret_cast<uint2*>(st + SL::kBHi + off) = hv;
              *reinterpret_cast<uint2*>(st + SL::kBLo + off) = lv;
            } else {
              uint2 hv;
              hv.x = pack_bf16x2(aB[h][v][0], aB[h][v][1]);
              hv.y = pack_bf16x2(aB[h][v][2], aB[h][v][3]);
              *reinterpret_cast<uint2*>(st + SL::kBHi + off) = hv;
            }
          }
        }
        fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
        __syncwarp();
        if (lane == 0) {
          if (PAIR)
            mbar_arrive_cluster(mapa_shared(smem_u32(&op_full[o]), 0));
          else
            mbar_arrive(smem_u32(&op_full[o]));
        }
        if (++o == S) {
          o = 0;
          oph ^= 1u;
        }
      }
    }
    // pair: every operand-stage release of the even CTA's MMA thread has arrived before the
    // CTA retires
    for (int i = 0; PAIR && ok && i < S; ++i) {
      ok = mbar_wait(smem_u32(&op_empty[o]), oph ^ 1u, p.timeout_ns, abort_flag);
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
