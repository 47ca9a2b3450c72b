// Tensor-core form of the cell update (Eq. 1 accumulate + normalise) on
// tcgen05: per 16x8 cell block b and channel tile of N channels (N = 64, 128
// or 256, a template parameter: the narrowest that holds C), the sums
//     S[cell, c] = sum_k T[cell, k] V[k, c]
// run as dense MMAs over the block's candidate samples k (sorted spatially by
// the plan; 32 per sub-chunk, one sub-chunk per chunk at N >= 128 and two at
// N = 64):  D[128 cells x N ch] (+)= A[128 x 16] * B[16 x N]
// with A = the block's weight tile (built in shared memory from the plan's
// weight entries, which carry their byte offset in the tile) and B = the
// sample values of the chunk (K-major, so each channel row holds the chunk's
// samples).  FP32 accumulation in TMEM.
//
// Precision: values and weights are split into a high and a low FP16 part;
// HEGRID_MODE_TC_SPLIT issues hi*hi + hi*lo + lo*hi (the lo*lo term is below
// FP32 rounding), HEGRID_MODE_TC issues hi*hi.  FP16 holds 11 significant
// bits but only 30 binades, so each channel c is first scaled by an exact
// power of two s_c that puts the channel's largest |v| (over all samples,
// found by a pass over the values before the launch) in [2^14, 2^15): every
// scaled value fits FP16, and a value's split error is at most 2^-22 of
// itself or 2^-25 (the FP16 subnormal step) in scaled units, i.e. 2^-39 of
// its own channel's largest value -- whatever the other channels of the tile
// hold.  The epilogue multiplies by 2^-k again.  FP16-stored values need no
// scale (they are exact); BF16-stored values are scaled and rounded to FP16,
// exactly for every value within 2^32 of the channel's largest.
// The tensor core's FP32 accumulate loses about 2^-22 of the running sum per
// MMA (measured; it grows with the number of MMAs added into one accumulator),
// so a block's sum is built in segments of J.seg sub-chunks (rounded down to
// whole chunks, at least one): segment 0 accumulates
// into a "total" TMEM region, later segments into a "segment" region that the
// drain warps add into the total with FP32 round-to-nearest adds (tcgen05
// ld/st).  Consecutive items swap the two regions' roles, so an item's
// epilogue overlaps the next item's first segment.  Weights enter the A tiles
// scaled by 2^15 (exact), which keeps the low FP16 half of their split a
// normal number; W comes from the plan (compensated sums of the weights) and
// is scaled to match.
//
// Warp roles (one CTA per SM, persistent over work items):
//   warp 17     stages the chunk's sample rows (raw, as stored; eight
//               four-row TMA tensor gathers per sub-chunk) into a ring;
//   warp 22     stages the chunk's weight entries (bulk copies) into a
//               3-deep ring of their own (with dense A tiles, kD: copies the
//               chunk's A tiles whole from the plan's dense weight tiles into
//               the A/B stage instead, and warps 8-15 convert B as well);
//   warps 0-7   convert a staged chunk into the B tiles (row = channel; 16-byte
//               pieces of 8 samples; no barrier among them);
//   warps 8-15  zero the A tiles and store the chunk's weight entries into
//               them at the tile offsets the plan precomputed (one barrier
//               among these 8 warps per chunk), side by side with the
//               converters on the same chunk (2-deep A/B ring);
//   warp 16     allocates TMEM and issues the MMAs (one lane);
//   warps 18-21 drain finished segments into the running total and run the
//               epilogue (TMEM -> registers -> S / W -> global).
// Hand-offs use mbarriers; MMA completion is signalled by tcgen05.commit.
// Every wait is bounded (global timer) and reports a timeout through the
// plan's error word.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "hegrid_internal.cuh"
#include "ptx.cuh"

namespace hg {
namespace {

constexpr int kProducerWarps = 16;
constexpr int kProducers = kProducerWarps * 32;
// The producers split in two groups that work on the same chunk side by side:
// warps 0-7 convert the staged rows into the B tiles, warps 8-15 build the A
// tiles from the weight entries (only they need a barrier, between zeroing
// the tiles and storing the entries).
constexpr int kGroupWarps = kProducerWarps / 2;
constexpr int kGroup = kGroupWarps * 32;
constexpr int kAhead = 8;  // weight entries per A builder loaded ahead of their stores
constexpr int kMmaWarp = kProducerWarps;
constexpr int kTmaWarp = kProducerWarps + 1;
constexpr int kDrainWarp0 = kProducerWarps + 2;  // 4 warps: drains and epilogue
constexpr int kEntWarp = kProducerWarps + 6;     // stages the weight entries
constexpr int kThreads = (kProducerWarps + 7) * 32;
constexpr int kK = 32;                     // candidates per sub-chunk (64-byte rows of 16-bit values)
constexpr int kM = HG_BLOCK_CELLS;         // cells per block
constexpr int kStages = 2;                 // A/B tile ring
constexpr int kDefaultSeg = 16;            // sub-chunks per accumulation segment
constexpr int kDefaultBand = -8;  // work order: bands of 8 block columns, channel tiles fastest
constexpr int kDefaultGroup = 0;  // ... all of a block's channel tiles side by side
// The channel tile kN (64, 128 or 256: the MMA's N) is a template parameter:
// the launcher takes the narrowest tile that holds C (256 above it), so few
// channels do not pay for 256-column tiles.  So is kS, the 32-candidate
// sub-chunks per chunk (the unit that passes through the rings with one set
// of barrier hand-offs): 2 for the 64-channel tile, whose per-chunk hand-offs
// would otherwise outweigh its small B tiles, else 1.  Per shape: candidates
// per chunk, staged row slot bytes (4-byte elements), TMEM columns (two
// accumulator regions), staged entries, 16-byte B-tile pieces per converting
// producer thread and converting threads.
// kD: the A tiles come whole from the plan's dense weight tiles (one bulk
// copy per sub-chunk by the entry stager warp: the tiles are the exact image
// the A builders would assemble) and all 16 producer warps convert B.
template <int kN, int kS, bool kD>
struct TcShape {
  static constexpr int kCK = kK * kS;
  static constexpr int kRawPitch = kN * 4;
  static constexpr uint32_t kTmemCols = 2 * kN;
  // staged-row ring and weight-entry ring depths, entries staged per chunk
  // (more come from global memory): as deep and large as shared memory allows
  // (with dense A tiles the entry ring is not needed and the rows get its room)
  static constexpr int kRawStages = kD ? (kN == 256 ? 3 : 6) : (kN == 256 ? 2 : kN == 128 ? 4 : 3);
  static constexpr int kEntStages = kD ? 1 : 3;
  static constexpr int kEntCap = kD ? 8 : 3584;
  static constexpr int kEntStage = kEntCap - 8;  // leaves room for 16-byte alignment
  static constexpr int kConv = kD ? kProducers : kGroup;  // B-converting threads
  static constexpr int kCPT = kN * (kCK / 8) / kConv;  // 16-byte B pieces per converter
  static_assert(kN * (kCK / 8) % kConv == 0, "B pieces do not divide among the converters");
};

// Where a staged chunk's weight entries are: e_lo is the global index of its
// first entry, n the number of entries (the first n0 belong to its first
// sub-chunk), ns how many were staged; entry i < ns sits at byte ck_off + 2 i
// of eck[] and w_off + 4 i of ew[].
struct EntInfo {
  int64_t e_lo;
  int32_t n, ns, n0;
  uint32_t ck_off, w_off;
};

template <int kN, int kS, bool kD>
struct __align__(512) TcSmem {
  using Sh = TcShape<kN, kS, kD>;
  uint8_t A[kStages][2][kS][kM * 64];  // [stage][hi, lo][sub-chunk]: weights, K-major, 64B swizzle
  uint8_t B[kStages][2][kS][kN * 64];  // [stage][hi, lo][sub-chunk]: values, K-major, 64B swizzle
  uint8_t raw[Sh::kRawStages][Sh::kCK * Sh::kRawPitch];  // staged sample rows as stored
  uint8_t eck[Sh::kEntStages][Sh::kEntCap * 2];  // staged entry tile offsets (16-byte aligned window)
  uint8_t ew[Sh::kEntStages][Sh::kEntCap * 4];   // staged entry weights (16-byte aligned window)
  EntInfo einfo[Sh::kEntStages];
  uint64_t raw_full[Sh::kRawStages], raw_empty[Sh::kRawStages];
  uint64_t ent_full[Sh::kEntStages], ent_empty[Sh::kEntStages];
  uint64_t ab_full[kStages], ab_empty[kStages];
  // MMA -> drains: a segment's MMAs are complete.  Two barriers used by
  // alternate segments: with the regions swapping roles per item the MMA
  // warp can complete up to two segments the drains have not taken yet.
  uint64_t segdone[2];
  uint64_t regfree[2];  // drains -> MMA: an accumulator region may be reused
  uint32_t tmem_base;
};

// Byte offset of 16-byte chunk q (0..3) of row r in a K-major, 64B-swizzled tile.
__device__ __forceinline__ uint32_t sw64(int r, int q) {
  return (uint32_t)(r * 64 + ((q ^ ((r >> 1) & 3)) << 4));
}

__device__ __forceinline__ int find_job(const JobTable& jt, int64_t item) {
  int j = 0;
  while (j + 1 < jt.n_jobs && jt.job[j + 1].item_base <= item) ++j;
  return j;
}

// Work order inside a job: cell blocks in bands of |J.band| block columns, so
// concurrently running CTAs share candidate rows in L2, and the channel tiles
// either slowest (J.band > 0) or in groups of J.group (0: all) run side by
// side (J.band < 0: the tiles of a group share the block's weight entries in
// L2; the groups follow one another over all blocks).
__device__ __forceinline__ void item_coords(const GridJob& J, int64_t local, int64_t& b,
                                            int64_t& ct) {
  const int64_t nb = J.pv.n_blocks;
  int64_t bo;
  if (J.band < 0) {
    const int64_t G = J.group > 0 && J.group < J.n_ctiles ? J.group : J.n_ctiles;
    const int64_t grp = local / (G * nb);  // every group before the last is full
    const int64_t r = local - grp * G * nb;
    const int64_t Gg = min(G, J.n_ctiles - grp * G);
    ct = grp * G + r % Gg;
    bo = r / Gg;
  } else {
    ct = local / nb;
    bo = local - ct * nb;
  }
  const int64_t kBand = J.band < 0 ? -(int64_t)J.band : J.band;
  const int64_t per_band = kBand * J.pv.nby_b;
  const int64_t band = bo / per_band;
  const int64_t t = bo - band * per_band;
  const int64_t bw = min(kBand, (int64_t)J.pv.nbx_b - band * kBand);
  b = (t / bw) * J.pv.nbx_b + band * kBand + (t % bw);
}

// First chunk of block b's sweep.  A block's candidates run through its bin
// window row by row, so the block above another (which runs at the same time
// in the work order) reaches the rows the two share a fraction
// J.rot = (block height) / (window height) of its sweep earlier; starting
// each block's sweep at the fraction frac(-row * J.rot) of its chunks (and
// wrapping around) has the blocks of neighbouring rows read their shared
// sample rows at about the same time, while they are in L2.  J.rot = 0: no
// rotation.  Every role of the CTA computes the same value.
__device__ __forceinline__ int sweep_start(const GridJob& J, int64_t b, int n_chunks) {
  if (J.rot <= 0.0f || n_chunks < 2) return 0;
  float f = -(float)(b / J.pv.nbx_b) * J.rot;
  f -= floorf(f);
  return min((int)(f * (float)n_chunks), n_chunks - 1);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

__device__ __forceinline__ uint32_t ld_shared_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t ld_shared_u16(uint32_t addr) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void st_shared_u16(uint32_t addr, uint16_t v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"(v) : "memory");
}

__device__ __forceinline__ void named_bar_a_builders() {
  asm volatile("bar.sync 1, %0;" ::"r"(kGroup) : "memory");
}

// Per-value 16-bit split of two FP32 values: hi = RN(v), lo = RN(v - hi), in
// FP16 (H16) or BF16, packed two per 32-bit word.
template <bool H16>
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  if (H16) {
    const __half2 h = __float22half2_rn(make_float2(v0, v1));
    const float2 f = __half22float2(h);
    const __half2 l = __float22half2_rn(make_float2(v0 - f.x, v1 - f.y));
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __nv_bfloat162 h = __float22bfloat162_rn(make_float2(v0, v1));
    const float2 f = __bfloat1622float2(h);
    const __nv_bfloat162 l = __float22bfloat162_rn(make_float2(v0 - f.x, v1 - f.y));
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}

__device__ __forceinline__ float bf16_bits_to_float(uint32_t b16) { return __uint_as_float(b16 << 16); }

// Exponent k of the power-of-two scale 2^k of a channel whose largest |v| has
// the float bits `mbits`: the scaled largest value lies in [2^14, 2^15).  All
// zero, or non-finite values present (outside the contract): unscaled.  k is
// kept in [-126, 126] so that 2^k and 2^-k are normal floats (a channel whose
// largest value is below 2^-112 is scaled less than that).
__device__ __forceinline__ int chan_scale_exp(uint32_t mbits) {
  const int e = (int)(mbits >> 23);  // biased exponent (the sign bit is clear)
  if (mbits == 0u || e >= 255) return 0;
  return min(141 - e, 126);  // 14 - (e - 127)
}
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// B converters (warps 0-7) for one work item: for every chunk, the staged
// rows, scaled by each channel's power of two and split into FP16 halves,
// become the B tiles (row = channel, K-major, 64-byte swizzle).  DT is the
// stored value type; SPLIT selects the hi/lo form.  n_sub is the item's count
// of 32-candidate sub-chunks (the last chunk may hold fewer than kS).
// `withhold` (failure tests) skips the first chunk's ab_full arrive.
// Returns false if a bounded wait gave up.
template <int DT, bool SPLIT, int kN, int kS, bool kD>
__device__ __forceinline__ bool convert_item(TcSmem<kN, kS, kD>& S, const GridJob& J, int n_chunks,
                                             int n_sub, int j0, int64_t c0, uint32_t& g,
                                             uint32_t& gr, int32_t* err, uint64_t lim,
                                             bool withhold) {
  using Sh = TcShape<kN, kS, kD>;
  constexpr bool kWide = DT == HEGRID_F32 || DT == HEGRID_BF16X2;  // 4-byte elements
  constexpr bool kVsplit = SPLIT && kWide;
  constexpr int kPitch = kWide ? Sh::kRawPitch : Sh::kRawPitch / 2;  // staged rows are packed
  const int t = threadIdx.x;  // 0 .. Sh::kConv-1
  // B row (channel c0 + row) and first 16-byte piece (8 samples) this thread
  // converts; pieces 4 u .. 4 u + 3 belong to sub-chunk u.
  const int row = t % kN, q0 = (t / kN) * Sh::kCPT;
  // this thread's channel scale (channels past C are staged as zeros)
  float sc = 1.0f;
  if (DT != HEGRID_F16 && J.chmax != nullptr && c0 + row < J.C)
    sc = pow2f(chan_scale_exp(__ldg(J.chmax + c0 + row)));
  for (int j = 0; j < n_chunks; ++j, ++g, ++gr) {
    const int s = g % kStages;
    const int rs = gr % Sh::kRawStages;
    if (!mbar_wait(&S.raw_full[rs], (gr / Sh::kRawStages) & 1u, err, lim)) return false;
    if (g >= kStages && !mbar_wait(&S.ab_empty[s], (g / kStages - 1) & 1u, err, lim)) return false;
    // rows of a sub-chunk that the last chunk lacks are not staged: zeros
    const int pj = j + j0 < n_chunks ? j + j0 : j + j0 - n_chunks;  // chunk of the sweep
    const bool present = kS == 1 || q0 * 8 < (n_sub - pj * kS) * kK;
    const uint32_t rb = smem_u32(S.raw[rs]) + q0 * 8 * kPitch;
    const uint32_t bh = smem_u32(S.B[s][0]), bl = smem_u32(S.B[s][1]);
#pragma unroll
    for (int qq = 0; qq < Sh::kCPT; ++qq) {
      // channel column `row` of 8 consecutive staged rows
      uint32_t x[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t a = rb + (qq * 8 + k) * kPitch;
        x[k] = !present ? 0u : kWide ? ld_shared_u32(a + row * 4) : ld_shared_u16(a + row * 2);
      }
      const int q = (q0 + qq) & 3;
      const uint32_t sub = kS == 1 ? 0u : (uint32_t)((q0 + qq) >> 2) * (uint32_t)(kN * 64);
      uint32_t h2[4], l2[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const uint32_t x0 = x[2 * e], x1 = x[2 * e + 1];
        if (DT == HEGRID_F32) {
          split2<true>(__uint_as_float(x0) * sc, __uint_as_float(x1) * sc, h2[e], l2[e]);
        } else if (DT == HEGRID_BF16X2) {
          const float v0 = bf16_bits_to_float(x0 & 0xffffu) + bf16_bits_to_float(x0 >> 16);
          const float v1 = bf16_bits_to_float(x1 & 0xffffu) + bf16_bits_to_float(x1 >> 16);
          split2<true>(v0 * sc, v1 * sc, h2[e], l2[e]);
        } else if (DT == HEGRID_BF16) {  // exact in BF16: one FP16 part
          const __half2 h = __float22half2_rn(
              make_float2(bf16_bits_to_float(x0) * sc, bf16_bits_to_float(x1) * sc));
          h2[e] = *reinterpret_cast<const uint32_t*>(&h);
          l2[e] = 0u;
        } else {  // F16: as stored
          h2[e] = x0 | (x1 << 16);
          l2[e] = 0u;
        }
      }
      st_shared_v4(bh + sub + sw64(row, q), h2[0], h2[1], h2[2], h2[3]);
      if (kVsplit) st_shared_v4(bl + sub + sw64(row, q), l2[0], l2[1], l2[2], l2[3]);
    }
    // the staged rows are read; the B tiles are written (visible to the MMA)
    __syncwarp();
    if ((t & 31) == 0) mbar_arrive(&S.raw_empty[rs]);
    fence_proxy_async_smem();
    __syncwarp();
    if ((t & 31) == 0 && !(withhold && g == 0)) mbar_arrive(&S.ab_full[s]);
  }
  return true;
}

// A builders (warps 8-15) for one work item: for every chunk, zero the A
// tiles, then store the chunk's weight entries, scaled by kTcWeightScale and
// split into FP16 halves, at the tile offsets the plan precomputed (in the
// second sub-tile from entry n0 on).  Returns false if a bounded wait gave up.
template <bool SPLIT, int kN, int kS>
__device__ __forceinline__ bool build_a_item(TcSmem<kN, kS, false>& S, const GridJob& J, int n_chunks,
                                             uint32_t& g, uint32_t& gr, int32_t* err,
                                             uint64_t lim) {
  using Sh = TcShape<kN, kS, false>;
  constexpr uint32_t kSubTile = kM * 64;       // A[s][h][1] follows A[s][h][0]
  constexpr uint32_t kLoTile = kS * kSubTile;  // A[s][1] follows A[s][0]
  const int t = threadIdx.x - kGroup;  // 0 .. kGroup-1
  const PlanView& pv = J.pv;
  for (int j = 0; j < n_chunks; ++j, ++g, ++gr) {
    const int s = g % kStages;
    const int rs = gr % Sh::kEntStages;
    if (!mbar_wait(&S.ent_full[rs], (gr / Sh::kEntStages) & 1u, err, lim)) return false;
    if (g >= kStages && !mbar_wait(&S.ab_empty[s], (g / kStages - 1) & 1u, err, lim)) return false;
    const uint32_t ah = smem_u32(S.A[s][0]);
    // zero (the stores follow the group's barrier)
#pragma unroll
    for (int i = t; i < kS * kM * 64 / 16; i += kGroup) {
      st_shared_v4(ah + i * 16, 0u, 0u, 0u, 0u);
      if (SPLIT) st_shared_v4(ah + kLoTile + i * 16, 0u, 0u, 0u, 0u);
    }
    // the chunk's weight entries (staged in shared memory by the row stager;
    // any beyond the staging capacity come from global memory).  Each thread
    // takes entries t, t + kGroup, ...; kAhead of them are loaded before the
    // barrier and the rest kAhead at a time, every batch's loads ahead of its
    // stores, so a dense chunk waits for global memory once per batch, not
    // once per entry.
    const EntInfo ei = S.einfo[rs];
    const uint32_t eck = smem_u32(S.eck[rs]) + ei.ck_off, ew = smem_u32(S.ew[rs]) + ei.w_off;
    uint32_t eo[kAhead];
    float ev[kAhead];
    auto load_batch = [&](int i0) {
#pragma unroll
      for (int k = 0; k < kAhead; ++k) {
        const int i = i0 + k * kGroup;
        eo[k] = 0u;
        ev[k] = 0.0f;
        if (i < ei.ns) {
          eo[k] = ld_shared_u16(eck + 2 * i);
          ev[k] = __uint_as_float(ld_shared_u32(ew + 4 * i));
        } else if (i < ei.n) {
          eo[k] = __ldg(pv.ent_ck + ei.e_lo + i);
          ev[k] = __ldg(pv.ent_w + ei.e_lo + i);
        }
      }
    };
    // stores entries i0 + k kGroup (k < kAhead) of the loaded batch: scaled
    // by kTcWeightScale, split into FP16 halves, two at a time
    auto store_batch = [&](int i0) {
#pragma unroll
      for (int k = 0; k < kAhead; k += 2) {
        const int i = i0 + k * kGroup;
        uint32_t p0 = eo[k], p1 = eo[k + 1];
        uint32_t h2, l2;
        split2<true>(ev[k] * kTcWeightScale, ev[k + 1] * kTcWeightScale, h2, l2);
        if (kS > 1) {
          p0 += i >= ei.n0 ? kSubTile : 0u;
          p1 += i + kGroup >= ei.n0 ? kSubTile : 0u;
        }
        if (i < ei.n) {
          st_shared_u16(ah + p0, (uint16_t)(h2 & 0xffffu));
          if (SPLIT) st_shared_u16(ah + kLoTile + p0, (uint16_t)(l2 & 0xffffu));
        }
        if (i + kGroup < ei.n) {
          st_shared_u16(ah + p1, (uint16_t)(h2 >> 16));
          if (SPLIT) st_shared_u16(ah + kLoTile + p1, (uint16_t)(l2 >> 16));
        }
      }
    };
    load_batch(t);
    named_bar_a_builders();
    store_batch(t);
    for (int i0 = t + kAhead * kGroup; i0 < ei.n; i0 += kAhead * kGroup) {
      load_batch(i0);
      store_batch(i0);
    }
    // the entries are read; the A tiles are written (visible to the MMA)
    __syncwarp();
    if ((t & 31) == 0) mbar_arrive(&S.ent_empty[rs]);
    fence_proxy_async_smem();
    __syncwarp();
    if ((t & 31) == 0) mbar_arrive(&S.ab_full[s]);
  }
  return true;
}

template <int kN, int kS, bool kD>
__global__ void __launch_bounds__(kThreads, 1) k_grid_tc(const __grid_constant__ JobTable jt) {
  using Sh = TcShape<kN, kS, kD>;
  extern __shared__ unsigned char smem_raw[];
  // 64B-swizzled tiles need 512-byte alignment (the swizzle atom); offsetting
  // smem_raw (not an integer round trip) keeps the shared address space.
  const uint32_t pad = (512u - (smem_u32(smem_raw) & 511u)) & 511u;
  TcSmem<kN, kS, kD>& S = *reinterpret_cast<TcSmem<kN, kS, kD>*>(smem_raw + pad);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t* err = jt.job[0].pv.err_word;
  const uint64_t lim = jt.wait_ns;  // limit of every bounded wait
  // failure-path test (HEGRID_FAULT=wait:N): producer warp 0 withholds its
  // arrive on the first chunk's ab_full, so the waits behind it run out
  const bool withhold = jt.inject != 0 && warp == 0;

  if (tid == 0) {
    for (int i = 0; i < Sh::kRawStages; ++i) {
      mbar_init(&S.raw_full[i], 1);
      mbar_init(&S.raw_empty[i], Sh::kConv / 32);  // the B converters
    }
    for (int i = 0; i < Sh::kEntStages; ++i) {
      mbar_init(&S.ent_full[i], 1);
      mbar_init(&S.ent_empty[i], kGroupWarps);  // the A builders
    }
    for (int i = 0; i < kStages; ++i) {
      // the producer warps, and with dense A tiles the A-tile copy's arrival
      mbar_init(&S.ab_full[i], kD ? kProducerWarps + 1 : kProducerWarps);
      mbar_init(&S.ab_empty[i], 1);
    }
    mbar_init(&S.segdone[0], 1);
    mbar_init(&S.segdone[1], 1);
    mbar_init(&S.regfree[0], 4);
    mbar_init(&S.regfree[1], 4);
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {
    tmem_alloc(&S.tmem_base, Sh::kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  bool bail = false;
  uint32_t g = 0;     // chunks through the A/B ring so far
  uint32_t gr = 0;    // chunks through the raw ring so far
  uint32_t n_tm = 0;  // items that used TMEM so far
  uint32_t n_sg = 0;  // accumulation segments so far (segdone phases)
  uint32_t uses[2] = {0u, 0u};  // MMA warp: segments accumulated into each region so far

  for (int64_t item = blockIdx.x; item < jt.n_items && !bail; item += gridDim.x) {
    const GridJob& J = jt.job[find_job(jt, item)];
    const PlanView& pv = J.pv;
    int64_t b, ct;
    item_coords(J, item - J.item_base, b, ct);
    const int64_t c0 = ct * kN;
    const int64_t C = J.C;
    const int64_t kb0 = pv.cand_off[b];
    const int n_sub = pv.cand_cnt[b] / kK;  // 32-candidate sub-chunks
    const int n_chunks = (n_sub + kS - 1) / kS;
    // J.seg counts sub-chunks: segments keep (about) that many candidates
    const int kSeg = kS == 1 ? J.seg : max(1, J.seg / kS);
    const int n_seg = (n_chunks + kSeg - 1) / kSeg;
    const bool split = J.mode == HEGRID_MODE_TC_SPLIT;
    const bool vsplit = split && (J.dtype == HEGRID_F32 || J.dtype == HEGRID_BF16X2);
    const int eb = (J.dtype == HEGRID_F32 || J.dtype == HEGRID_BF16X2) ? 4 : 2;

    // the sweep's j-th chunk (sweep_start: the sweep begins at chunk j0 and wraps)
    const int j0 = sweep_start(J, b, n_chunks);
    auto phys = [&](int jl) { return jl + j0 < n_chunks ? jl + j0 : jl + j0 - n_chunks; };

    if (warp == kTmaWarp) {
      // ---------------- row stager ----------------
      // Per chunk: the 32 kS sample rows (8 kS four-row tensor gathers of the
      // channel tile; channels past C arrive as zeros), completing on
      // raw_full.  Candidate indices are loaded two chunks ahead.
      const uint32_t row_bytes = (uint32_t)(kN * eb);
      const void* tmap = &J.rows;
      // this lane's candidate of each sub-chunk of the sweep's chunk j (nA) and j + 1 (nB)
      int32_t nA[kS], nB[kS];
      {
        const int p0 = phys(0), p1 = n_chunks > 1 ? phys(1) : 0;
#pragma unroll
        for (int t = 0; t < kS; ++t) {
          nA[t] = p0 * kS + t < n_sub ? __ldg(pv.cand_idx + kb0 + (int64_t)(p0 * kS + t) * kK + lane) : 0;
          nB[t] = n_chunks > 1 && p1 * kS + t < n_sub
                      ? __ldg(pv.cand_idx + kb0 + (int64_t)(p1 * kS + t) * kK + lane)
                      : 0;
        }
      }
      for (int j = 0; j < n_chunks; ++j, ++gr) {
        const int r = gr % Sh::kRawStages;
        const uint32_t u = gr / Sh::kRawStages;
        const int pj = phys(j);
        const int nsj = min(kS, n_sub - pj * kS);  // sub-chunks in this chunk
        const int p2 = j + 2 < n_chunks ? phys(j + 2) : -1;
        int32_t n[kS];  // this lane's rows
#pragma unroll
        for (int t = 0; t < kS; ++t) {
          n[t] = nA[t];
          nA[t] = nB[t];
          if (p2 >= 0 && p2 * kS + t < n_sub)
            nB[t] = __ldg(pv.cand_idx + kb0 + (int64_t)(p2 * kS + t) * kK + lane);
        }
        if (u >= 1 && !mbar_wait(&S.raw_empty[r], (u - 1) & 1u, err, lim)) {
          bail = true;
          break;
        }
        if (lane == 0) mbar_arrive_expect_tx(&S.raw_full[r], row_bytes * (uint32_t)(kK * nsj));
        __syncwarp();
#pragma unroll
        for (int t = 0; t < kS; ++t) {
          const int q4 = (lane & 7) * 4;
          const int32_t r0 = __shfl_sync(0xffffffffu, n[t], q4);
          const int32_t r1 = __shfl_sync(0xffffffffu, n[t], q4 + 1);
          const int32_t r2 = __shfl_sync(0xffffffffu, n[t], q4 + 2);
          const int32_t r3 = __shfl_sync(0xffffffffu, n[t], q4 + 3);
          if (lane < 8 && t < nsj)
            tma_gather4(&S.raw[r][(t * kK + lane * 4) * row_bytes], tmap, (int32_t)c0, r0, r1, r2,
                        r3, &S.raw_full[r]);
        }
      }
      continue;
    }

    if (kD && warp == kEntWarp) {
      // ---------------- A-tile stager (dense A tiles) ----------------
      // Per chunk: once the A/B stage is free, the chunk's sub-chunks' A
      // tiles (hi, and lo in the split form) straight from the plan's dense
      // weight tiles into the stage, completing on ab_full with one
      // expect_tx arrival.
      const uint8_t* wt = pv.wtiles + (kb0 / kK) * (int64_t)(2 * kM * 64);
      for (int j = 0; j < n_chunks; ++j, ++g) {
        const int s = g % kStages;
        const int pj = phys(j);
        const int nsj = min(kS, n_sub - pj * kS);
        if (g >= kStages && !mbar_wait(&S.ab_empty[s], (g / kStages - 1) & 1u, err, lim)) {
          bail = true;
          break;
        }
        if (lane == 0) {
          const uint32_t half = (uint32_t)(kM * 64);
          mbar_arrive_expect_tx(&S.ab_full[s], half * (split ? 2u : 1u) * (uint32_t)nsj);
          for (int t = 0; t < nsj; ++t) {
            const uint8_t* src = wt + (int64_t)(pj * kS + t) * (2 * kM * 64);
            bulk_g2s(S.A[s][0][t], src, half, &S.ab_full[s]);
            if (split) bulk_g2s(S.A[s][1][t], src + half, half, &S.ab_full[s]);
          }
        }
        __syncwarp();
      }
      continue;
    }

    if (warp == kEntWarp) {
      // ---------------- entry stager ----------------
      // Sub-chunk offsets are loaded 31 / kS chunks at a time (lane i holds
      // the offset of sub-chunk pb kS + i; reloaded where the sweep wraps).
      constexpr int kBatch = 31 / kS;
      const int64_t* __restrict__ so = pv.sub_off + kb0 / kK;
      int64_t sob = 0;
      int pb = 0;  // chunk whose first sub-chunk lane 0's offset belongs to
      for (int j = 0; j < n_chunks; ++j, ++gr) {
        const int r = gr % Sh::kEntStages;
        const uint32_t u = gr / Sh::kEntStages;
        const int pj = phys(j);
        if (j == 0 || pj == 0 || pj - pb >= kBatch) {
          pb = pj;
          sob = pb * kS + lane <= n_sub ? __ldg(so + pb * kS + lane) : 0;
        }
        const int jb = pj - pb;
        const int nsj = min(kS, n_sub - pj * kS);  // sub-chunks in this chunk
        const int64_t e_lo = __shfl_sync(0xffffffffu, sob, jb * kS);
        const int64_t e_mid = kS == 1 ? e_lo : __shfl_sync(0xffffffffu, sob, jb * kS + 1);
        const int64_t e_end = __shfl_sync(0xffffffffu, sob, jb * kS + kS);
        const int64_t e_hi = nsj == kS ? e_end : e_mid;
        if (u >= 1 && !mbar_wait(&S.ent_empty[r], (u - 1) & 1u, err, lim)) {
          bail = true;
          break;
        }
        const int ne = (int)(e_hi - e_lo);
        const int ns = ne < Sh::kEntStage ? ne : Sh::kEntStage;
        const int64_t a0 = (e_lo * 2) & ~(int64_t)15, b0 = (e_lo * 4) & ~(int64_t)15;
        const uint32_t abytes = ns > 0 ? (uint32_t)((((e_lo + ns) * 2 + 15) & ~(int64_t)15) - a0) : 0u;
        const uint32_t wbytes = ns > 0 ? (uint32_t)((((e_lo + ns) * 4 + 15) & ~(int64_t)15) - b0) : 0u;
        if (lane == 0) {
          EntInfo ei;
          ei.e_lo = e_lo;
          ei.n = ne;
          ei.ns = ns;
          ei.n0 = kS == 1 ? ne : (int32_t)(e_mid - e_lo);
          ei.ck_off = (uint32_t)(e_lo * 2 - a0);
          ei.w_off = (uint32_t)(e_lo * 4 - b0);
          S.einfo[r] = ei;
          mbar_arrive_expect_tx(&S.ent_full[r], abytes + wbytes);
        }
        __syncwarp();
        if (lane == 0 && abytes)
          bulk_g2s(S.eck[r], reinterpret_cast<const uint8_t*>(pv.ent_ck) + a0, abytes,
                   &S.ent_full[r]);
        if (lane == 1 && wbytes)
          bulk_g2s(S.ew[r], reinterpret_cast<const uint8_t*>(pv.ent_w) + b0, wbytes,
                   &S.ent_full[r]);
      }
      continue;
    }

    if (warp == kMmaWarp) {
      // ---------------- MMA issuer ----------------
      if (n_chunks == 0) continue;
      const uint32_t idS = idesc_f16(0u, kM, kN);  // FP16 A and B, FP32 accumulate
      // Item n_tm accumulates its total in region rT and later segments in
      // rS; the next item swaps them, so its first segment can run while
      // this item's epilogue still reads rT.
      const uint32_t rT = n_tm & 1u, rS = rT ^ 1u;
      uint32_t dcol = 0;
      for (int j = 0; j < n_chunks && !bail; ++j, ++g) {
        const int s = g % kStages;
        const int q = j / kSeg;
        const bool seg_start = j % kSeg == 0;
        const bool seg_end = j % kSeg == kSeg - 1 || j == n_chunks - 1;
        if (seg_start) {
          // the region is free once the drains released its previous use
          // (a drained segment, or an epilogue that read a total)
          const uint32_t r = q == 0 ? rT : rS;
          if (uses[r] > 0 && !mbar_wait(&S.regfree[r], (uses[r] - 1) & 1u, err, lim)) bail = true;
          ++uses[r];
          dcol = r * (uint32_t)kN;
          tc_fence_after();
          if (bail) break;
        }
        if (!mbar_wait(&S.ab_full[s], (g / kStages) & 1u, err, lim)) {
          bail = true;
          break;
        }
        tc_fence_after();
        if (lane == 0) {
          const uint32_t d = tmem + dcol;
          const int nsj = min(kS, n_sub - phys(j) * kS);
#pragma unroll
          for (int t = 0; t < kS; ++t) {
            if (t >= nsj) break;
            const uint32_t a_hi = smem_u32(S.A[s][0][t]), a_lo = smem_u32(S.A[s][1][t]);
            const uint32_t b_hi = smem_u32(S.B[s][0][t]), b_lo = smem_u32(S.B[s][1][t]);
#pragma unroll
            for (int kk = 0; kk < kK / 16; ++kk) {
              const uint32_t o = kk * 32;
              const uint32_t acc = (!seg_start || t > 0 || kk > 0) ? 1u : 0u;
              tc_mma_f16(d, smem_desc_k_sw64(a_hi + o), smem_desc_k_sw64(b_hi + o), idS, acc);
              if (vsplit)
                tc_mma_f16(d, smem_desc_k_sw64(a_hi + o), smem_desc_k_sw64(b_lo + o), idS, 1u);
              if (split)
                tc_mma_f16(d, smem_desc_k_sw64(a_lo + o), smem_desc_k_sw64(b_hi + o), idS, 1u);
            }
          }
          tc_commit(&S.ab_empty[s]);
          if (seg_end) tc_commit(&S.segdone[n_sg & 1u]);
        }
        __syncwarp();
        if (seg_end) ++n_sg;
      }
      ++n_tm;
      continue;
    }

    if (warp >= kDrainWarp0 && warp < kDrainWarp0 + 4) {
      // ---------------- drains and epilogue ----------------
      const int quarter = warp & 3;  // TMEM lane quarter this warp may access
      const int row = quarter * 32 + lane;
      const int bbx = (int)(b % pv.nbx_b), bby = (int)(b / pv.nbx_b);
      const int ix = bbx * HG_BX + (row % HG_BX), iy = bby * HG_BY + (row / HG_BX);
      const bool active = ix < pv.nx && iy < pv.ny;
      const int64_t m = (int64_t)iy * pv.nx + ix;
      float* out = J.map + m * J.ld_map;
      const float qnan = __int_as_float(0x7fc00000);
      if (n_chunks == 0) {
        if (active) {
          const int64_t cend = c0 + kN < C ? c0 + kN : C;
          for (int64_t cc = c0; cc < cend; ++cc) out[cc] = qnan;
          if (c0 == 0 && J.weight_out) J.weight_out[m] = 0.0f;
        }
        continue;
      }
      const uint32_t lrow = (uint32_t)(quarter * 32) << 16;
      const uint32_t rT = n_tm & 1u, rS = rT ^ 1u;
      const uint32_t tseg = tmem + lrow + rS * (uint32_t)kN, ttot = tmem + lrow + rT * (uint32_t)kN;
      for (int q = 0; q < n_seg; ++q) {
        if (!mbar_wait(&S.segdone[n_sg & 1u], (n_sg >> 1) & 1u, err, lim)) {
          bail = true;
          break;
        }
        ++n_sg;
        tc_fence_after();
        if (q > 0) {
          // total += segment, FP32 round-to-nearest (16-column slices keep
          // the kernel within its register budget without spills)
          uint32_t a[16], t[16];
#pragma unroll 1
          for (int cb = 0; cb < kN / 16; ++cb) {
            tmem_ld_32x32b_x16(tseg + cb * 16, a);
            tmem_ld_32x32b_x16(ttot + cb * 16, t);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i)
              t[i] = __float_as_uint(__fadd_rn(__uint_as_float(t[i]), __uint_as_float(a[i])));
            tmem_st_32x32b_x16(ttot + cb * 16, t);
          }
          tmem_st_wait();
          // the segment region is drained
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.regfree[rS]);
        }
      }
      if (bail) break;
      // epilogue: map = total / W * 2^-k_c, W from the plan's compensated
      // sums: FP32 weights for the split form (the hi+lo split differs from
      // them by at most 2^-22 per weight, at random), FP16-rounded weights for
      // the single form; both x 2^15.  k_c is the channel's scale exponent.
      const float Wm = active ? pv.wsum[(int64_t)(split ? 0 : 1) * pv.M + m] : 0.0f;
      const float W = Wm * kTcWeightScale;
      const bool ok = W > 0.0f;
      // one reciprocal per cell: t * (1/W) * 2^-k is within one ulp of t / W * 2^-k
      const float rW = ok ? __frcp_rn(W) : 0.0f;
      const bool scaled = J.chmax != nullptr && J.dtype != HEGRID_F16;
      // 32 columns per step: each lane writes whole 128-byte lines of its row
      uint32_t t[32];
#pragma unroll 1
      for (int cb = 0; cb < kN / 32; ++cb) {
        tmem_ld_32x32b_x32(ttot + cb * 32, t);
        tmem_ld_wait();
        const int64_t cbase = c0 + cb * 32;
        // lane l holds 2^-k of channel cbase + l; every lane takes them all
        const float inv_l = scaled && cbase + lane < C
                                ? pow2f(-chan_scale_exp(__ldg(J.chmax + cbase + lane)))
                                : 1.0f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          // the second product is exact (a power of two on a normal value)
          const float inv = __shfl_sync(0xffffffffu, inv_l, i);
          t[i] = __float_as_uint(ok ? __fmul_rn(__fmul_rn(__uint_as_float(t[i]), rW), inv) : qnan);
        }
        if (active) {
          if (cbase + 32 <= C && (((uintptr_t)(out + cbase) & 15u) == 0)) {
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              __stcs(reinterpret_cast<float4*>(out + cbase + i),
                     make_float4(__uint_as_float(t[i]), __uint_as_float(t[i + 1]),
                                 __uint_as_float(t[i + 2]), __uint_as_float(t[i + 3])));
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (cbase + i < C) __stcs(out + cbase + i, __uint_as_float(t[i]));
          }
        }
      }
      if (active && c0 == 0 && J.weight_out) J.weight_out[m] = Wm;
      // the total region has been read
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.regfree[rT]);
      ++n_tm;
      continue;
    }

    // ---------------- producers (warps 0-15) ----------------
    if (n_chunks == 0) continue;
    {
      bool ok = true;
      if constexpr (!kD) {
        if (warp >= kGroupWarps) {  // A builders
          ok = split ? build_a_item<true, kN, kS>(S, J, n_chunks, g, gr, err, lim)
                     : build_a_item<false, kN, kS>(S, J, n_chunks, g, gr, err, lim);
          bail = !ok;
          ++n_tm;
          continue;
        }
      }
      if (split) {  // B converters
        switch (J.dtype) {
          case HEGRID_F32: ok = convert_item<HEGRID_F32, true, kN, kS, kD>(S, J, n_chunks, n_sub, j0, c0, g, gr, err, lim, withhold); break;
          case HEGRID_BF16: ok = convert_item<HEGRID_BF16, true, kN, kS, kD>(S, J, n_chunks, n_sub, j0, c0, g, gr, err, lim, withhold); break;
          case HEGRID_F16: ok = convert_item<HEGRID_F16, true, kN, kS, kD>(S, J, n_chunks, n_sub, j0, c0, g, gr, err, lim, withhold); break;
          default: ok = convert_item<HEGRID_BF16X2, true, kN, kS, kD>(S, J, n_chunks, n_sub, j0, c0, g, gr, err, lim, withhold); break;
        }
      } else {
        switch (J.dtype) {
          case HEGRID_F32: ok = convert_item<HEGRID_F32, false, kN, kS, kD>(S, J, n_chunks, n_sub, j0, c0, g, gr, err, lim, withhold); break;
          case HEGRID_BF16: ok = convert_item<HEGRID_BF16, false, kN, kS, kD>(S, J, n_chunks, n_sub, j0, c0, g, gr, err, lim, withhold); break;
          case HEGRID_F16: ok = convert_item<HEGRID_F16, false, kN, kS, kD>(S, J, n_chunks, n_sub, j0, c0, g, gr, err, lim, withhold); break;
          default: ok = convert_item<HEGRID_BF16X2, false, kN, kS, kD>(S, J, n_chunks, n_sub, j0, c0, g, gr, err, lim, withhold); break;
        }
      }
      bail = !ok;
      ++n_tm;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem, Sh::kTmemCols);
}

template <int kN, int kS, bool kD>
hegrid_status launch_tile(const JobTable& jt, cudaStream_t s) {
  static int sms = 0;
  const size_t smem = sizeof(TcSmem<kN, kS, kD>) + 512;
  if (!sms) {
    int dev;
    cudaGetDevice(&dev);
    HG_CUDA_TRY(cudaFuncSetAttribute(k_grid_tc<kN, kS, kD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  int64_t grid = std::min<int64_t>(jt.n_items, (int64_t)sms);
  if (grid < 1) return HEGRID_OK;
  if (fault_hit(kFaultWait)) {
    JobTable t = jt;
    t.inject = 1;
    t.wait_ns = kInjectWaitNs;
    k_grid_tc<kN, kS, kD><<<(unsigned)grid, kThreads, smem, s>>>(t);
  } else {
    k_grid_tc<kN, kS, kD><<<(unsigned)grid, kThreads, smem, s>>>(jt);
  }
  count_launch();
  HG_CUDA_TRY(launch_status());
  return HEGRID_OK;
}

}  // namespace

int tc_channel_tile(int64_t C) { return C <= 64 ? 64 : C <= 128 ? 128 : 256; }
int tc_default_band() { return kDefaultBand; }
int tc_default_seg() { return kDefaultSeg; }
int tc_default_group() { return kDefaultGroup; }

hegrid_status launch_grid_tc(const JobTable& jt, cudaStream_t s, int tile, bool dense_a) {
  switch (tile * 2 + (dense_a ? 1 : 0)) {
    case 128: return launch_tile<64, 2, false>(jt, s);
    case 129: return launch_tile<64, 2, true>(jt, s);
    case 256: return launch_tile<128, 1, false>(jt, s);
    case 257: return launch_tile<128, 1, true>(jt, s);
    case 512: return launch_tile<256, 1, false>(jt, s);
    case 513: return launch_tile<256, 1, true>(jt, s);
    default:
      set_error("unsupported tensor-core channel tile");
      return HEGRID_ERR_UNSUPPORTED;
  }
}

}  // namespace hg
