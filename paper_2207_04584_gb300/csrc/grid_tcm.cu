// Channel-major tensor-core form of the cell update (Eq. 1 accumulate +
// normalise) on tcgen05.  Per 16x8 cell block b and tile of 128 channels the
// sums run transposed,
//     S^T[c, cell] = sum_k V^T[c, k] T^T[k, cell],
// as D[128 ch x 128 cells] (+)= A[128 x 16] * B[16 x 128] over the block's
// candidate samples k (32 per sub-chunk), with
//   A = the values of the sub-chunk's samples, one channel per TMEM lane:
//       the 32 sample rows' 128-channel slices are gathered by TMA into a
//       shared-memory ring, read once by the value warps (one thread per
//       channel, so a warp reads 32 consecutive channels of a row), scaled
//       by the channel's power of two, split into FP16 halves and stored into
//       TMEM (tcgen05.st), where the MMA reads them;
//   B = the sub-chunk's weight tile (cells x candidates, K-major, 64-byte
//       swizzle, FP16 hi and lo halves of the weights x 2^15), built once
//       per plan by k_build_wtiles and brought in by one bulk copy.
// The values are not written back to shared memory as MMA operand tiles and
// no weight tile is built per channel tile: per sub-chunk and 128 channels
// the kernel moves 16 KB of sample rows in and out of shared memory, 16 KB of
// weight tiles in, and the MMAs read 24 KB of them, about 72 KB against the
// cell-major kernel's ~125 KB per 128 channels (staged rows in and out,
// converted B tiles, zeroed and scattered A tiles, entries, operand reads).
// Precision, segments, the per-channel scale and W are those of the
// cell-major kernel (grid_tc.cu): hi*hi + hi*lo (+ lo*hi for 4-byte values)
// in the split form, hi*hi in the single form.
//
// Warp roles (one CTA per SM, persistent over work items):
//   warps 0-7    value warps: warp w serves TMEM lane quarter w & 3 (its
//                32 channels) and candidates 16 (w >> 2) .. +15 of each
//                sub-chunk;
//   warp 8       allocates TMEM and issues the MMAs (one lane);
//   warp 9       bulk-copies each sub-chunk's weight tiles into the ring;
//   warp 14      gathers each sub-chunk's 32 sample rows (eight four-row TMA
//                tensor gathers of the 128-channel slice; channels past C
//                arrive as zeros) into the row ring;
//   warps 10-13  drain finished segments into the running total and run the
//                epilogue (TMEM -> registers -> S / W -> global, one cell per
//                step, a warp's 32 channels of it in one coalesced store).
// Hand-offs use mbarriers; MMA completion is signalled by tcgen05.commit.
// Every wait is bounded (global timer) and reports a timeout through the
// plan's error word.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "hegrid_internal.cuh"
#include "ptx.cuh"
#include "wtile.cuh"

namespace hg {
namespace {

constexpr int kCM = 128;             // channels per item (the MMA's M, TMEM lanes)
constexpr int kCN = HG_BLOCK_CELLS;  // cells per block (the MMA's N)
constexpr int kCK = 32;              // candidates per sub-chunk
// Rings: the value operands in TMEM and the weight tiles in shared memory
// are held in two round slots of kRound stages each (kAStg = kBStg = 2 kRound):
// the MMA warp issues a round's MMAs behind one fence and releases the
// round's stages with one tcgen05.commit.  A round never spans two
// accumulation segments; a short round at a segment's end leaves its slot's
// remaining stages unused (their barriers still complete one phase per
// round).  The sample rows (kRStg stages) are released as soon as the value
// warps have read them.
constexpr int kRound = 4;  // sub-chunks per MMA issue round
constexpr int kAStg = 2 * kRound;
constexpr int kBStg = 2 * kRound;
constexpr int kRStg = 5;
constexpr int kValWarps = 8;
constexpr int kMmaW = 8;
constexpr int kTileW = 9;
constexpr int kDrainW0 = 10;  // 4 warps
constexpr int kRowW = 14;
constexpr int kThreadsCM = 15 * 32;
constexpr uint32_t kHalfTile = kWTileHalfBytes;      // one 16-bit half: 128 rows x 64 bytes
constexpr uint32_t kDCols = kCN;                     // accumulator columns (one per cell)
constexpr uint32_t kACol0 = 2u * kDCols;             // value operands after the two regions
constexpr uint32_t kAStageCols = kCK;                // hi: 16 columns, lo: 16 columns
constexpr uint32_t kTmemColsCM = 512;
static_assert(kACol0 + kAStg * kAStageCols <= kTmemColsCM, "TMEM columns");
constexpr int kDefaultSegCM = 16;
constexpr int kPrefetch = 12;  // weight tiles prefetched into L2 this many sub-chunks ahead


constexpr uint32_t kRawStage = (uint32_t)kCK * kCM * 4u;  // 32 rows x 128 channels x <= 4 bytes

struct __align__(1024) CmSmem {
  uint8_t B[kBStg][kWTileBytes];  // [stage]: hi tile, then lo tile
  uint8_t raw[kRStg][kRawStage];  // [stage]: the sub-chunk's 32 rows, 128 channels each, as stored
  uint64_t raw_full[kRStg];       // row gathers -> value warps
  uint64_t raw_empty[kRStg];      // value warps -> row stager: the stage's rows are read
  uint64_t a_full[kAStg];         // value warps -> MMA: the stage's values are in TMEM
  uint64_t b_full[kBStg];         // bulk copy -> MMA: the stage's weight tiles landed
  uint64_t round_empty[2];        // MMA -> value warps, tile stager: a round slot's MMAs are complete
  uint64_t segdone[2];
  uint64_t regfree[2];
  uint32_t tmem_base;
};

__device__ __forceinline__ int find_job_cm(const JobTable& jt, int64_t item) {
  int j = 0;
  while (j + 1 < jt.n_jobs && jt.job[j + 1].item_base <= item) ++j;
  return j;
}

// Work order as in the cell-major kernel: blocks in bands of |band| block
// columns; channel tiles slowest (band > 0) or side by side in groups of
// `group` (band < 0; 0: all of a block's tiles).
__device__ __forceinline__ void item_coords_cm(const GridJob& J, int64_t local, int64_t& b,
                                               int64_t& ct) {
  const int64_t nb = J.pv.n_blocks;
  int64_t bo;
  if (J.band < 0) {
    const int64_t G = J.group > 0 && J.group < J.n_ctiles ? J.group : J.n_ctiles;
    const int64_t grp = local / (G * nb);
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

// First sub-chunk of block b's sweep (see sweep_start in grid_tc.cu).
__device__ __forceinline__ int sweep_start_cm(const GridJob& J, int64_t b, int n) {
  if (J.rot <= 0.0f || n < 2) return 0;
  float f = -(float)(b / J.pv.nbx_b) * J.rot;
  f -= floorf(f);
  return min((int)(f * (float)n), n - 1);
}

__device__ __forceinline__ int chan_scale_exp_cm(uint32_t mbits) {
  const int e = (int)(mbits >> 23);
  if (mbits == 0u || e >= 255) return 0;
  return min(141 - e, 126);
}
__device__ __forceinline__ float pow2f_cm(int k) { return __int_as_float((127 + k) << 23); }
__device__ __forceinline__ float bf16_to_f(uint32_t b16) { return __uint_as_float(b16 << 16); }

// Two FP32 values -> packed FP16 hi halves and lo halves (hi = RN(v),
// lo = RN(v - hi)); the first value in the low 16 bits.
__device__ __forceinline__ void split_h2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __float22half2_rn(make_float2(v0, v1));
  const float2 f = __half22float2(h);
  const __half2 l = __float22half2_rn(make_float2(v0 - f.x, v1 - f.y));
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// D[tmem] (+)= A[tmem] * B[smem desc], kind::f16 (A from tensor memory).
__device__ __forceinline__ void tc_mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                              uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Prefetch `bytes` (a multiple of 16, 16-byte aligned) of global memory into L2.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tmem_st_x8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
      : "memory");
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t addr) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr) : "memory");
  return v;
}

// Issue rounds: sub-chunk j of an item (segments of kSeg sub-chunks) lies in
// round j / kSeg * ceil(kSeg / kRound) + (j % kSeg) / kRound of the item, at
// slot (j % kSeg) % kRound; an item of n sub-chunks takes
// rounds_of(n, kSeg) rounds.  Round R uses stages (R & 1) kRound + slot.
__device__ __forceinline__ int rounds_per_seg(int kSeg) { return (kSeg + kRound - 1) / kRound; }
__device__ __forceinline__ uint32_t rounds_of(int n, int kSeg) {
  if (n <= 0) return 0u;
  const int full = (n - 1) / kSeg;  // segments before the last
  const int last = n - full * kSeg;
  return (uint32_t)(full * rounds_per_seg(kSeg) + (last + kRound - 1) / kRound);
}

// Value warps for one work item.  Returns false if a bounded wait gave up.
template <int DT, bool SPLIT>
__device__ __forceinline__ bool values_item(CmSmem& S, const GridJob& J, int n_sub, int kSeg,
                                            int64_t c0, uint32_t tmem, uint32_t& gr,
                                            uint32_t R0, int32_t* err, uint64_t lim,
                                            bool withhold) {
  constexpr bool kWide = DT == HEGRID_F32 || DT == HEGRID_BF16X2;
  constexpr bool kVsplit = SPLIT && kWide;
  constexpr uint32_t kEb = kWide ? 4u : 2u;
  constexpr uint32_t kRow = kCM * kEb;  // bytes of a staged row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, h = warp >> 2;
  const int64_t c = c0 + 32 * q + lane;
  float sc = 1.0f;
  if (DT != HEGRID_F16 && J.chmax != nullptr && c < J.C)
    sc = pow2f_cm(chan_scale_exp_cm(__ldg(J.chmax + c)));
  const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
  const int rps = rounds_per_seg(kSeg);
  for (int j = 0; j < n_sub; ++j, ++gr) {
    const int r = (int)(gr % kRStg);
    if (!mbar_wait(&S.raw_full[r], (gr / kRStg) & 1u, err, lim)) return false;
    // this thread's channel in rows 16 h .. 16 h + 15 of the staged sub-chunk
    const uint32_t rb = smem_u32(S.raw[r]) + (uint32_t)(16 * h) * kRow + (uint32_t)(32 * q + lane) * kEb;
    uint32_t v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = kWide ? lds_u32(rb + i * kRow) : lds_u16(rb + i * kRow);
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.raw_empty[r]);
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const uint32_t x0 = v[2 * e], x1 = v[2 * e + 1];
      if (DT == HEGRID_F32) {
        split_h2(__uint_as_float(x0) * sc, __uint_as_float(x1) * sc, hi[e], lo[e]);
      } else if (DT == HEGRID_BF16X2) {
        const float f0 = bf16_to_f(x0 & 0xffffu) + bf16_to_f(x0 >> 16);
        const float f1 = bf16_to_f(x1 & 0xffffu) + bf16_to_f(x1 >> 16);
        split_h2(f0 * sc, f1 * sc, hi[e], lo[e]);
      } else if (DT == HEGRID_BF16) {  // exact in BF16: one FP16 part
        const __half2 hh = __float22half2_rn(make_float2(bf16_to_f(x0) * sc, bf16_to_f(x1) * sc));
        hi[e] = *reinterpret_cast<const uint32_t*>(&hh);
        lo[e] = 0u;
      } else {  // F16 as stored
        hi[e] = x0 | (x1 << 16);
        lo[e] = 0u;
      }
    }
    const int seg = j / kSeg, jj = j - seg * kSeg;
    const uint32_t R = R0 + (uint32_t)(seg * rps + jj / kRound);
    const int s = (int)(R & 1u) * kRound + jj % kRound;
    // the round slot is free once round R - 2's MMAs are complete
    if (jj % kRound == 0 && R >= 2u &&
        !mbar_wait(&S.round_empty[R & 1u], ((R >> 1) - 1u) & 1u, err, lim))
      return false;
    tc_fence_after();
    const uint32_t a = tl + kACol0 + (uint32_t)s * kAStageCols + 8u * (uint32_t)h;
    tmem_st_x8(a, hi);
    if (kVsplit) tmem_st_x8(a + 16u, lo);
    tmem_st_wait();
    tc_fence_before();
    __syncwarp();
    if (lane == 0 && !(withhold && R == 0u && jj == 0)) mbar_arrive(&S.a_full[s]);
    // a round cut short by its segment's end: arrive on the slot's unused
    // stages too, so that every stage completes one phase per round
    const int seg_end = min((seg + 1) * kSeg, n_sub);
    if (j == seg_end - 1 && lane == 0)
      for (int t = jj % kRound + 1; t < kRound; ++t) mbar_arrive(&S.a_full[(int)(R & 1u) * kRound + t]);
  }
  return true;
}

__global__ void __launch_bounds__(kThreadsCM, 1) k_grid_tcm(const __grid_constant__ JobTable jt) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
  CmSmem& S = *reinterpret_cast<CmSmem*>(smem_raw + pad);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t* err = jt.job[0].pv.err_word;
  const uint64_t lim = jt.wait_ns;
  const bool withhold = jt.inject != 0 && warp == 0;

  if (tid == 0) {
    for (int i = 0; i < kRStg; ++i) {
      mbar_init(&S.raw_full[i], 1);
      mbar_init(&S.raw_empty[i], kValWarps);
    }
    for (int i = 0; i < kAStg; ++i) mbar_init(&S.a_full[i], kValWarps);
    for (int i = 0; i < kBStg; ++i) mbar_init(&S.b_full[i], 1);
    mbar_init(&S.round_empty[0], 1);
    mbar_init(&S.round_empty[1], 1);
    mbar_init(&S.segdone[0], 1);
    mbar_init(&S.segdone[1], 1);
    mbar_init(&S.regfree[0], 4);
    mbar_init(&S.regfree[1], 4);
    fence_mbar_init();
  }
  if (warp == kMmaW) {
    tmem_alloc(&S.tmem_base, kTmemColsCM);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  bool bail = false;
  uint32_t gr = 0;    // sub-chunks through the row ring so far
  uint32_t R0 = 0;    // issue rounds so far (before the current item)
  uint32_t n_tm = 0;  // items that used TMEM so far
  uint32_t n_sg = 0;  // accumulation segments so far
  uint32_t uses[2] = {0u, 0u};

  for (int64_t item = blockIdx.x; item < jt.n_items && !bail; item += gridDim.x) {
    const GridJob& J = jt.job[find_job_cm(jt, item)];
    const PlanView& pv = J.pv;
    int64_t b, ct;
    item_coords_cm(J, item - J.item_base, b, ct);
    const int64_t c0 = ct * kCM;
    const int64_t C = J.C;
    const int64_t kb0 = pv.cand_off[b];
    const int n_sub = pv.cand_cnt[b] / kCK;
    const int kSeg = J.seg;
    const int n_seg = (n_sub + kSeg - 1) / kSeg;
    const bool split = J.mode == HEGRID_MODE_TC_SPLIT;
    const bool vsplit = split && (J.dtype == HEGRID_F32 || J.dtype == HEGRID_BF16X2);
    const int j0 = sweep_start_cm(J, b, n_sub);
    const int rps = rounds_per_seg(kSeg);
    const uint32_t Ri = R0;  // the item's first round
    R0 += rounds_of(n_sub, kSeg);

    if (warp == kRowW) {
      // ---------------- row stager ----------------
      // Candidate indices are loaded two sub-chunks ahead.
      const bool wide = J.dtype == HEGRID_F32 || J.dtype == HEGRID_BF16X2;
      const uint32_t row_bytes = (uint32_t)kCM * (wide ? 4u : 2u);
      const void* tmap = &J.rows;
      auto phys = [&](int jl) { return jl + j0 < n_sub ? jl + j0 : jl + j0 - n_sub; };
      auto cand_of = [&](int jl) -> int32_t {
        return __ldg(pv.cand_idx + kb0 + (int64_t)phys(jl) * kCK + lane);
      };
      int32_t nA = n_sub > 0 ? cand_of(0) : 0, nB = n_sub > 1 ? cand_of(1) : 0;
      for (int j = 0; j < n_sub; ++j, ++gr) {
        const int s = (int)(gr % kRStg);
        const int32_t n = nA;
        nA = nB;
        if (j + 2 < n_sub) nB = cand_of(j + 2);
        if (gr >= kRStg && !mbar_wait(&S.raw_empty[s], (gr / kRStg - 1) & 1u, err, lim)) {
          bail = true;
          break;
        }
        if (lane == 0) mbar_arrive_expect_tx(&S.raw_full[s], row_bytes * (uint32_t)kCK);
        __syncwarp();
        const int q4 = (lane & 7) * 4;
        const int32_t r0 = __shfl_sync(0xffffffffu, n, q4);
        const int32_t r1 = __shfl_sync(0xffffffffu, n, q4 + 1);
        const int32_t r2 = __shfl_sync(0xffffffffu, n, q4 + 2);
        const int32_t r3 = __shfl_sync(0xffffffffu, n, q4 + 3);
        if (lane < 8)
          tma_gather4(&S.raw[s][(uint32_t)(lane * 4) * row_bytes], tmap, (int32_t)c0, r0, r1, r2,
                      r3, &S.raw_full[s]);
      }
      continue;
    }

    if (warp == kTileW) {
      // ---------------- weight-tile stager ----------------
      // Each tile is first prefetched into L2 kPrefetch sub-chunks ahead of
      // its copy, so that the copy, which can only start once the stage's
      // previous MMAs are complete, waits for L2 rather than DRAM.
      const uint8_t* wt = pv.wtiles + (kb0 / kCK) * (int64_t)kWTileBytes;
      if (lane == 0)
        for (int j = 0; j < kPrefetch && j < n_sub; ++j)
          prefetch_l2(wt + (int64_t)(j + j0 < n_sub ? j + j0 : j + j0 - n_sub) * kWTileBytes,
                      kWTileBytes);
      for (int j = 0; j < n_sub; ++j) {
        const int seg = j / kSeg, jj = j - seg * kSeg;
        const uint32_t R = Ri + (uint32_t)(seg * rps + jj / kRound);
        const int s = (int)(R & 1u) * kRound + jj % kRound;
        const int pj = j + j0 < n_sub ? j + j0 : j + j0 - n_sub;
        if (lane == 0 && j + kPrefetch < n_sub) {
          const int jp = j + kPrefetch + j0;
          prefetch_l2(wt + (int64_t)(jp < n_sub ? jp : jp - n_sub) * kWTileBytes, kWTileBytes);
        }
        if (jj % kRound == 0 && R >= 2u &&
            !mbar_wait(&S.round_empty[R & 1u], ((R >> 1) - 1u) & 1u, err, lim)) {
          bail = true;
          break;
        }
        if (lane == 0) {
          mbar_arrive_expect_tx(&S.b_full[s], kWTileBytes);
          bulk_g2s(S.B[s], wt + (int64_t)pj * kWTileBytes, kWTileBytes, &S.b_full[s]);
          // a round cut short by its segment's end: complete the slot's
          // unused stages' phases too (plain arrivals)
          if (j == min((seg + 1) * kSeg, n_sub) - 1)
            for (int t = jj % kRound + 1; t < kRound; ++t)
              mbar_arrive(&S.b_full[(int)(R & 1u) * kRound + t]);
        }
        __syncwarp();
      }
      continue;
    }

    if (warp == kMmaW) {
      // ---------------- MMA issuer ----------------
      // Each round waits for its (up to kRound) sub-chunks of one segment,
      // issues all their MMAs behind one fence and releases its round slot
      // with one commit (one sub-chunk per round cost ~1,100 cycles however
      // few MMAs it held).
      if (n_sub == 0) continue;
      const uint32_t idS = idesc_f16(0u, kCM, kCN);  // FP16 A and B, FP32 accumulate
      const uint32_t rT = n_tm & 1u, rS = rT ^ 1u;
      for (int qs = 0; qs < n_seg && !bail; ++qs) {
        const int j = qs * kSeg, je = min(j + kSeg, n_sub);
        const uint32_t r = qs == 0 ? rT : rS;
        if (uses[r] > 0 && !mbar_wait(&S.regfree[r], (uses[r] - 1) & 1u, err, lim)) {
          bail = true;
          break;
        }
        ++uses[r];
        const uint32_t d = tmem + r * kDCols;
        tc_fence_after();
        for (int j1 = j; j1 < je && !bail; j1 += kRound) {
          const int nr = min(kRound, je - j1);
          const uint32_t R = Ri + (uint32_t)(qs * rps + (j1 - j) / kRound);
          const int s0 = (int)(R & 1u) * kRound;
          const uint32_t ph = (R >> 1) & 1u;
          for (int t = 0; t < nr && !bail; ++t)
            if (!mbar_wait(&S.a_full[s0 + t], ph, err, lim) ||
                !mbar_wait(&S.b_full[s0 + t], ph, err, lim))
              bail = true;
          if (bail) break;
          tc_fence_after();
          if (lane == 0) {
            for (int t = 0; t < nr; ++t) {
              const uint32_t a = tmem + kACol0 + (uint32_t)(s0 + t) * kAStageCols;
              const uint32_t bh = smem_u32(S.B[s0 + t]), bl = bh + kHalfTile;
#pragma unroll
              for (int kk = 0; kk < kCK / 16; ++kk) {
                const uint32_t o = kk * 32;             // bytes into a 64-byte tile row
                const uint32_t ac = 8u * (uint32_t)kk;  // columns into the value operand
                const uint32_t acc = (j1 + t > j || kk > 0) ? 1u : 0u;
                tc_mma_f16_ts(d, a + ac, smem_desc_k_sw64(bh + o), idS, acc);
                if (split) tc_mma_f16_ts(d, a + ac, smem_desc_k_sw64(bl + o), idS, 1u);
                if (vsplit) tc_mma_f16_ts(d, a + 16u + ac, smem_desc_k_sw64(bh + o), idS, 1u);
              }
            }
            tc_commit(&S.round_empty[R & 1u]);
            if (j1 + nr == je) tc_commit(&S.segdone[n_sg & 1u]);
          }
          __syncwarp();
        }
        ++n_sg;
      }
      ++n_tm;
      continue;
    }

    if (warp >= kDrainW0 && warp < kDrainW0 + 4) {
      // ---------------- drains and epilogue ----------------
      const int quarter = warp & 3;
      const int64_t c = c0 + 32 * quarter + lane;  // this thread's channel (TMEM lane)
      const bool cok = c < C;
      const int bbx = (int)(b % pv.nbx_b), bby = (int)(b / pv.nbx_b);
      const float qnan = __int_as_float(0x7fc00000);
      float* map = J.map;
      if (n_sub == 0) {
        for (int n = 0; n < kCN; ++n) {
          const int ix = bbx * HG_BX + (n % HG_BX), iy = bby * HG_BY + (n / HG_BX);
          if (ix < pv.nx && iy < pv.ny && cok)
            map[((int64_t)iy * pv.nx + ix) * J.ld_map + c] = qnan;
        }
        if (c0 == 0 && quarter == 0 && J.weight_out) {
          for (int n = lane; n < kCN; n += 32) {
            const int ix = bbx * HG_BX + (n % HG_BX), iy = bby * HG_BY + (n / HG_BX);
            if (ix < pv.nx && iy < pv.ny) J.weight_out[(int64_t)iy * pv.nx + ix] = 0.0f;
          }
        }
        continue;
      }
      const uint32_t lrow = (uint32_t)(quarter * 32) << 16;
      const uint32_t rT = n_tm & 1u, rS = rT ^ 1u;
      const uint32_t tseg = tmem + lrow + rS * kDCols, ttot = tmem + lrow + rT * kDCols;
      for (int qs = 0; qs < n_seg; ++qs) {
        if (!mbar_wait(&S.segdone[n_sg & 1u], (n_sg >> 1) & 1u, err, lim)) {
          bail = true;
          break;
        }
        ++n_sg;
        tc_fence_after();
        if (qs > 0) {
          uint32_t a[16], t[16];
#pragma unroll 1
          for (int cb = 0; cb < (int)kDCols / 16; ++cb) {
            tmem_ld_32x32b_x16(tseg + cb * 16, a);
            tmem_ld_32x32b_x16(ttot + cb * 16, t);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i)
              t[i] = __float_as_uint(__fadd_rn(__uint_as_float(t[i]), __uint_as_float(a[i])));
            tmem_st_32x32b_x16(ttot + cb * 16, t);
          }
          tmem_st_wait();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.regfree[rS]);
        }
      }
      if (bail) break;
      // epilogue: map[cell, c] = total / W[cell] * 2^-k_c (W x 2^15 as the
      // weight tiles carry it; the FP32 weights' sum for the split form, the
      // FP16-rounded weights' for the single form)
      const bool scaled = J.chmax != nullptr && J.dtype != HEGRID_F16;
      const float inv_c = scaled && cok ? pow2f_cm(-chan_scale_exp_cm(__ldg(J.chmax + c))) : 1.0f;
      uint32_t t[32];
#pragma unroll 1
      for (int cb = 0; cb < kCN / 32; ++cb) {
        tmem_ld_32x32b_x32(ttot + cb * 32, t);
        tmem_ld_wait();
        // lane l: cell cb * 32 + l (its W, reciprocal and map row)
        const int n = cb * 32 + lane;
        const int ix = bbx * HG_BX + (n % HG_BX), iy = bby * HG_BY + (n / HG_BX);
        const bool act = ix < pv.nx && iy < pv.ny;
        const int64_t m = (int64_t)iy * pv.nx + ix;
        const float Wm = act ? pv.wsum[(int64_t)(split ? 0 : 1) * pv.M + m] : 0.0f;
        const float W = Wm * kTcWeightScale;
        const float rW = W > 0.0f ? __frcp_rn(W) : 0.0f;
        if (c0 == 0 && quarter == 0 && J.weight_out && act) J.weight_out[m] = Wm;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float rWi = __shfl_sync(0xffffffffu, rW, i);
          const int acti = __shfl_sync(0xffffffffu, act ? 1 : 0, i);
          const int64_t mi = __shfl_sync(0xffffffffu, m, i);
          const float o =
              rWi > 0.0f ? __fmul_rn(__fmul_rn(__uint_as_float(t[i]), rWi), inv_c) : qnan;
          if (acti && cok) __stcs(map + mi * J.ld_map + c, o);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.regfree[rT]);
      ++n_tm;
      continue;
    }

    // ---------------- value warps (0-7) ----------------
    if (n_sub == 0) continue;
    {
      bool ok = true;
      if (split) {
        switch (J.dtype) {
          case HEGRID_F32: ok = values_item<HEGRID_F32, true>(S, J, n_sub, kSeg, c0, tmem, gr, Ri, err, lim, withhold); break;
          case HEGRID_BF16: ok = values_item<HEGRID_BF16, true>(S, J, n_sub, kSeg, c0, tmem, gr, Ri, err, lim, withhold); break;
          case HEGRID_F16: ok = values_item<HEGRID_F16, true>(S, J, n_sub, kSeg, c0, tmem, gr, Ri, err, lim, withhold); break;
          default: ok = values_item<HEGRID_BF16X2, true>(S, J, n_sub, kSeg, c0, tmem, gr, Ri, err, lim, withhold); break;
        }
      } else {
        switch (J.dtype) {
          case HEGRID_F32: ok = values_item<HEGRID_F32, false>(S, J, n_sub, kSeg, c0, tmem, gr, Ri, err, lim, withhold); break;
          case HEGRID_BF16: ok = values_item<HEGRID_BF16, false>(S, J, n_sub, kSeg, c0, tmem, gr, Ri, err, lim, withhold); break;
          case HEGRID_F16: ok = values_item<HEGRID_F16, false>(S, J, n_sub, kSeg, c0, tmem, gr, Ri, err, lim, withhold); break;
          default: ok = values_item<HEGRID_BF16X2, false>(S, J, n_sub, kSeg, c0, tmem, gr, Ri, err, lim, withhold); break;
        }
      }
      bail = !ok;
      ++n_tm;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaW) tmem_dealloc(tmem, kTmemColsCM);
}

// Dense weight tiles of a plan: for every used sub-chunk of every block, the
// hi and lo FP16 halves of its weights x 2^15 at the tile offsets the entries
// carry (zeros elsewhere), 16 KB per sub-chunk at (slot / 32) * 16 KB.  One
// CTA per (block, quarter of its sub-chunks); the tile is assembled in shared
// memory and written out with coalesced 16-byte stores.
constexpr int kBuildSplit = 4;
__global__ void __launch_bounds__(256) k_build_wtiles(PlanView pv, uint8_t* __restrict__ wt,
                                                      int64_t blk0) {
  __shared__ __align__(16) uint8_t tile[kWTileBytes];
  const int64_t b = blk0 + blockIdx.x / kBuildSplit;
  const int part = (int)(blockIdx.x % kBuildSplit);
  const int t = threadIdx.x;
  const int64_t s0 = pv.cand_off[b] / kCK;
  const int n_sub = pv.cand_cnt[b] / kCK;
  wtile_zero<256>(tile, t);
  __syncthreads();
  for (int j = part; j < n_sub; j += kBuildSplit) {
    const int64_t s = s0 + j;
    wtile_scatter<256>(tile, pv.ent_ck, pv.ent_w, pv.sub_off[s], pv.sub_off[s + 1], t);
    __syncthreads();
    wtile_flush<256>(tile, wt + s * (int64_t)kWTileBytes, t);
    __syncthreads();
  }
}

}  // namespace

int tcm_channel_tile() { return kCM; }
int tcm_default_seg() { return kDefaultSegCM; }
int64_t tcm_wtile_bytes(int64_t slots) { return (slots / kCK) * (int64_t)kWTileBytes; }

hegrid_status launch_build_wtiles(const PlanView& pv, uint8_t* wtiles, cudaStream_t s,
                                 int64_t blk0, int64_t n_blk) {
  if (n_blk < 0) n_blk = pv.n_blocks - blk0;
  if (n_blk <= 0) return HEGRID_OK;
  k_build_wtiles<<<(unsigned)(n_blk * kBuildSplit), 256, 0, s>>>(pv, wtiles, blk0);
  count_launch();
  HG_CUDA_TRY(launch_status());
  return HEGRID_OK;
}

hegrid_status launch_grid_tcm(const JobTable& jt, cudaStream_t s) {
  static int sms = 0;
  const size_t smem = sizeof(CmSmem) + 1024;
  if (!sms) {
    int dev;
    cudaGetDevice(&dev);
    HG_CUDA_TRY(cudaFuncSetAttribute(k_grid_tcm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  int64_t grid = std::min<int64_t>(jt.n_items, (int64_t)sms);
  if (grid < 1) return HEGRID_OK;
  if (fault_hit(kFaultWait)) {
    JobTable t = jt;
    t.inject = 1;
    t.wait_ns = kInjectWaitNs;
    k_grid_tcm<<<(unsigned)grid, kThreadsCM, smem, s>>>(t);
  } else {
    k_grid_tcm<<<(unsigned)grid, kThreadsCM, smem, s>>>(jt);
  }
  count_launch();
  HG_CUDA_TRY(launch_status());
  return HEGRID_OK;
}

}  // namespace hg
