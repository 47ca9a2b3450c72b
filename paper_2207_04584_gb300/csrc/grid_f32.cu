// Plain FP32 form of the cell update (Algorithm 1's accumulate and normalise
// steps, Eq. 1) on CUDA cores.
//
// A persistent CTA takes work items (field, 16x8 cell block, 128-channel tile)
// in a fixed stride, in the job's work order (the channel tiles of a block
// back to back, or channel tiles slowest with the blocks in bands of block
// columns).  For each K chunk of 32 candidate samples of the block:
//   * warp 0 stages the 32 sample rows (FP32, channel-contiguous; eight
//     four-row TMA tensor gathers of the 128-channel tile) and the chunk's
//     weight entries (two bulk copies of 16-byte aligned windows) into shared
//     memory, completing on an mbarrier,
//     double-buffered: chunk j + 1 is staged while chunk j is computed;
//     one CTA barrier per chunk (after the scatter; each warp clears its own
//     columns of the weight tile after computing);
//   * the threads scatter the staged entries into a dense 32 x 128 weight
//     tile and OR a per-patch occupancy mask;
//   * each warp owns a 4x4-cell patch and 128 channels; a thread accumulates
//     8 cells x 8 channels in registers, skipping samples that touch no cell
//     of its patch.
// Summation in two levels: the register sums cover kFlush chunks and are then
// added (FP32, round to nearest) into running totals that the thread keeps in
// tensor memory (TMEM, otherwise idle in this kernel: 64 columns of one lane
// per thread), so no FP32 sum runs over more than a few dozen of a cell's
// ~10^3 terms; this cuts the rounding error of a long sequential sum about
// threefold.
// The epilogue divides by W (NaN where W = 0) and writes the map row-major.
#include <cuda_runtime.h>

#include <algorithm>

#include "hegrid_internal.cuh"
#include "ptx.cuh"

namespace hg {
namespace {

constexpr int kThreads = 256;
constexpr int kKC = 32;   // candidates per K chunk
constexpr int kCT = 128;  // channels per tile
constexpr int kFlush = 4;   // chunks per register partial sum (then added to the TMEM total)
constexpr int kEB = 4;      // weight entries per thread loaded ahead of their stores
constexpr uint32_t kTmemCols = 128;  // 64 FP32 totals per thread: two warps per lane quarter
constexpr int kEntCap = 2048;           // weight entries staged per chunk (more: global)
constexpr int kEntStage = kEntCap - 8;  // entries copied (room for 16-byte alignment)

// Where a staged chunk's weight entries are: entry i < ns at byte ck_off + 2 i
// of eck[] and w_off + 4 i of ew[]; entries ns..n-1 are read from global.
struct EntWin {
  int64_t e_lo;
  int32_t n, ns;
  uint32_t ck_off, w_off;
};

struct __align__(128) SmemF32 {
  float V[2][kKC][kCT];         // staged sample rows
  float Wt[2][kKC][kCT];        // dense weight tile [k][cell column]
  uint8_t eck[2][kEntCap * 2];  // staged entry tile offsets (16-byte aligned window)
  uint8_t ew[2][kEntCap * 4];   // staged entry weights (16-byte aligned window)
  EntWin win[2];
  uint32_t pmask[2][kKC];  // per sample k: bit p set if any cell of patch p has it
  uint64_t bar[2];
  uint32_t tmem_base;
};

__device__ __forceinline__ int find_job(const JobTable& jt, int64_t item) {
  int j = 0;
  while (j + 1 < jt.n_jobs && jt.job[j + 1].item_base <= item) ++j;
  return j;
}

// Block-local cell (lx, ly) -> tile column (inverse of col_to_cell).
__device__ __forceinline__ int cell_to_col(int lx, int ly) {
  int p = (ly >> 2) * 4 + (lx >> 2);
  int py = ly & 3, px = lx & 3;
  int cs = py >> 1, i = (py & 1) * 4 + px;
  return p * 16 + cs * 8 + i;
}

// Tile column t (0..127) -> block-local cell (lx, ly): 8 patches of 4x4 cells,
// patches 4 across x 2 down; inside a patch, two 8-cell halves of 2 rows x 4.
__device__ __forceinline__ void col_to_cell(int t, int& lx, int& ly) {
  int p = t >> 4, q = t & 15;
  int cs = q >> 3, i = q & 7;
  int py = cs * 2 + (i >> 2), px = i & 3;
  ly = (p >> 2) * 4 + py;
  lx = (p & 3) * 4 + px;
}

__global__ void __launch_bounds__(kThreads, 2)
    k_grid_f32(const __grid_constant__ JobTable jt) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SmemF32& S = *reinterpret_cast<SmemF32*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&S.tmem_base, kTmemCols);
    tmem_relinquish();
  }
  {  // both weight tiles and patch masks start zero (and are left zero by every chunk)
    float4* wz = reinterpret_cast<float4*>(&S.Wt[0][0][0]);
    for (int i = tid; i < 2 * kKC * kCT / 4; i += kThreads) wz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid < 2 * kKC) (&S.pmask[0][0])[tid] = 0u;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // this thread's 64 running totals: one TMEM lane of its warp's lane quarter,
  // columns 0-63 (warps 0-3) or 64-127 (warps 4-7)
  const uint32_t taddr =
      S.tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * 64);
  uint32_t phase[2] = {0u, 0u};
  bool bail = false;

  for (int64_t item = blockIdx.x; item < jt.n_items && !bail; item += gridDim.x) {
    const GridJob& J = jt.job[find_job(jt, item)];
    const PlanView& pv = J.pv;
    const int64_t local = item - J.item_base;
    int64_t b, ct;
    if (J.band <= 0) {  // channel tiles of a block back to back
      b = local / J.n_ctiles;
      ct = local % J.n_ctiles;
    } else {  // channel tiles slowest, blocks in bands of J.band block columns
      const int64_t nb = J.pv.n_blocks;
      ct = local / nb;
      const int64_t bo = local - ct * nb;
      const int64_t per_band = (int64_t)J.band * J.pv.nby_b;
      const int64_t band = bo / per_band;
      const int64_t t = bo - band * per_band;
      const int64_t bw = min((int64_t)J.band, (int64_t)J.pv.nbx_b - band * J.band);
      b = (t / bw) * J.pv.nbx_b + band * J.band + (t % bw);
    }
    const int64_t c0 = ct * kCT;
    const int cw = (int)(J.C - c0 < kCT ? J.C - c0 : kCT);
    const int bbx = (int)(b % pv.nbx_b), bby = (int)(b / pv.nbx_b);
    const int64_t kb0 = pv.cand_off[b];
    const int n_chunks = pv.cand_cnt[b] / kKC;

    const int64_t* __restrict__ so = pv.sub_off + kb0 / kKC;  // the block's sub-chunks

    // Stage chunk j (warp 0): its 32 sample rows (one bulk copy per lane) and
    // its weight entries (two bulk copies of 16-byte aligned windows), all
    // completing on bar[j & 1].  Candidate indices come one chunk ahead in
    // registers, sub-chunk offsets 31 chunks at a time.
    int32_t n_cur = 0, n_next = 0;
    int64_t sob = 0;
    if (warp == 0 && n_chunks > 0) {
      n_cur = pv.cand_idx[kb0 + lane];
      if (n_chunks > 1) n_next = pv.cand_idx[kb0 + kKC + lane];
    }
    auto issue = [&](int j) {
      const int s = j & 1;
      const int jb = j % 31;
      if (jb == 0) sob = j + lane <= n_chunks ? __ldg(so + j + lane) : 0;
      const int64_t e_lo = __shfl_sync(0xffffffffu, sob, jb);
      const int64_t e_hi = __shfl_sync(0xffffffffu, sob, jb + 1);
      const int ne = (int)(e_hi - e_lo);
      const int ns = ne < kEntStage ? ne : kEntStage;
      const int64_t a0 = (e_lo * 2) & ~(int64_t)15, b0 = (e_lo * 4) & ~(int64_t)15;
      const uint32_t ab = ns > 0 ? (uint32_t)((((e_lo + ns) * 2 + 15) & ~(int64_t)15) - a0) : 0u;
      const uint32_t wb = ns > 0 ? (uint32_t)((((e_lo + ns) * 4 + 15) & ~(int64_t)15) - b0) : 0u;
      if (lane == 0) {
        EntWin w;
        w.e_lo = e_lo;
        w.n = ne;
        w.ns = ns;
        w.ck_off = (uint32_t)(e_lo * 2 - a0);
        w.w_off = (uint32_t)(e_lo * 4 - b0);
        S.win[s] = w;
        mbar_arrive_expect_tx(&S.bar[s], kKC * kCT * 4 + ab + wb);
      }
      __syncwarp();
      const int32_t n = n_cur;
      n_cur = n_next;
      if (j + 2 < n_chunks) n_next = pv.cand_idx[kb0 + (int64_t)(j + 2) * kKC + lane];
      // the 32 rows by eight four-row tensor gathers (channels past C arrive as zeros)
      {
        const int q4 = (lane & 7) * 4;
        const int32_t r0 = __shfl_sync(0xffffffffu, n, q4), r1 = __shfl_sync(0xffffffffu, n, q4 + 1);
        const int32_t r2 = __shfl_sync(0xffffffffu, n, q4 + 2), r3 = __shfl_sync(0xffffffffu, n, q4 + 3);
        if (lane < 8) tma_gather4(&S.V[s][q4][0], &J.rows, (int32_t)c0, r0, r1, r2, r3, &S.bar[s]);
      }
      if (lane == 0 && ab)
        bulk_g2s(S.eck[s], reinterpret_cast<const uint8_t*>(pv.ent_ck) + a0, ab, &S.bar[s]);
      if (lane == 1 && wb)
        bulk_g2s(S.ew[s], reinterpret_cast<const uint8_t*>(pv.ent_w) + b0, wb, &S.bar[s]);
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[i][e] = 0.0f;
    // add the register partial sums into the TMEM totals (the first flush of
    // an item stores them) and restart the partials (warp-uniform calls)
    auto flush = [&](bool first) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float t[8];
        if (first) {
#pragma unroll
          for (int e = 0; e < 8; ++e) t[e] = acc[i][e];
        } else {
          tmem_ld_32x32b_x8(taddr + i * 8, t);
          tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < 8; ++e) t[e] = __fadd_rn(t[e], acc[i][e]);
        }
        tmem_st_32x32b_x8(taddr + i * 8, t);
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[i][e] = 0.0f;
      }
      tmem_st_wait();
    };

    const int patch = warp, cs = lane >> 4, cg = lane & 15;
    if (warp == 0 && n_chunks > 0) issue(0);
    for (int j = 0; j < n_chunks; ++j) {
      const int s = j & 1;
      // weight tile for chunk j: wait for the staged rows and entries, then
      // scatter the entries into tile s (all zero: each warp cleared its own
      // columns after computing chunk j - 2, before the previous barrier)
      const bool staged = mbar_wait(&S.bar[s], phase[s], pv.err_word);
      if (staged) {
        const EntWin w = S.win[s];
        const uint32_t eck = smem_u32(S.eck[s]) + w.ck_off, ew = smem_u32(S.ew[s]) + w.w_off;
        // kEB entries per thread at a time, all loaded before any is stored, so
        // that entries beyond the staged ones (dense chunks) wait for global
        // memory once per batch rather than once per entry
        for (int i0 = tid; i0 < w.n; i0 += kEB * kThreads) {
          uint32_t ck[kEB];
          float wt[kEB];
#pragma unroll
          for (int b = 0; b < kEB; ++b) {
            const int i = i0 + b * kThreads;
            ck[b] = 0u;
            wt[b] = 0.0f;
            if (i < w.ns) {
              uint16_t h;
              asm volatile("ld.shared.u16 %0, [%1];" : "=h"(h) : "r"(eck + 2 * i));
              ck[b] = h;
              asm volatile("ld.shared.f32 %0, [%1];" : "=f"(wt[b]) : "r"(ew + 4 * i));
            } else if (i < w.n) {
              ck[b] = __ldg(pv.ent_ck + w.e_lo + i);
              wt[b] = __ldg(pv.ent_w + w.e_lo + i);
            }
          }
#pragma unroll
          for (int b = 0; b < kEB; ++b) {
            if (i0 + b * kThreads >= w.n) break;
            int col, k;
            tile_rk(ck[b], col, k);
            const int tc = cell_to_col(col % HG_BX, col / HG_BX);
            S.Wt[s][k][tc] = wt[b];
            atomicOr(&S.pmask[s][k], 1u << (tc >> 4));
          }
        }
      }
      if (__syncthreads_or(!staged)) {
        // give up (chunk j + 1 is not staged yet: no other copies in flight)
        bail = true;
        break;
      }
      phase[s] ^= 1u;
      // every warp is past chunk j - 1, so its staged rows and entry windows
      // (buffer s ^ 1) are free: stage chunk j + 1 while chunk j is computed
      if (warp == 0 && j + 1 < n_chunks) issue(j + 1);
      const uint32_t* pm = S.pmask[s];
      const float* wrow = &S.Wt[s][0][patch * 16 + cs * 8];
      const float* vrow = &S.V[s][0][cg * 8];
      for (int k = 0; k < kKC; ++k) {
        if (!((pm[k] >> patch) & 1u)) continue;
        float4 w0 = *reinterpret_cast<const float4*>(wrow + k * kCT);
        float4 w1 = *reinterpret_cast<const float4*>(wrow + k * kCT + 4);
        float4 v0 = *reinterpret_cast<const float4*>(vrow + k * kCT);
        float4 v1 = *reinterpret_cast<const float4*>(vrow + k * kCT + 4);
        float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[i][e] = __fmaf_rn(w[i], v[e], acc[i][e]);
      }
      // clear this warp's columns of tile s and its bit of the patch masks
      // (no other warp reads or writes them before the next barrier; the
      // warp's own lanes have all finished reading them)
      __syncwarp();
      {
        float4* wz = reinterpret_cast<float4*>(&S.Wt[s][0][patch * 16]);
#pragma unroll
        for (int i = lane; i < kKC * 4; i += 32)  // 32 rows x 4 float4 of 16 columns
          wz[(i >> 2) * (kCT / 4) + (i & 3)] = make_float4(0.f, 0.f, 0.f, 0.f);
        atomicAnd(&S.pmask[s][lane], ~(1u << patch));
      }
      if (j % kFlush == kFlush - 1 && j + 1 < n_chunks) {
        __syncwarp();
        flush(j == kFlush - 1);
      }
    }
    // every warp is done with this item's staged rows before the next item
    // stages its first chunk
    __syncthreads();

    if (bail) break;
    // the sums: TMEM total (if any partial was flushed) + the last partial
    if (n_chunks > kFlush) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float t[8];
        tmem_ld_32x32b_x8(taddr + i * 8, t);
        tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[i][e] = __fadd_rn(t[e], acc[i][e]);
      }
    }
    // epilogue: normalise and store
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int lx, ly;
      col_to_cell(patch * 16 + cs * 8 + i, lx, ly);
      int ix = bbx * HG_BX + lx, iy = bby * HG_BY + ly;
      if (ix >= pv.nx || iy >= pv.ny) continue;
      int64_t m = (int64_t)iy * pv.nx + ix;
      float W = pv.wsum[m];
      float* out = J.map + m * J.ld_map + c0 + cg * 8;
      int cbase = cg * 8;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        if (cbase + e < cw) out[e] = W > 0.0f ? __fdiv_rn(acc[i][e], W) : __int_as_float(0x7fc00000);
      }
      if (ct == 0 && cg == 0 && J.weight_out) J.weight_out[m] = W;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(S.tmem_base, kTmemCols);
}

}  // namespace

int f32_channel_tile() { return kCT; }

hegrid_status launch_grid_f32(const JobTable& jt, cudaStream_t s) {
  static int sms = 0;
  if (!sms) {
    int dev;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_grid_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(SmemF32));
  }
  int64_t grid = std::min<int64_t>(jt.n_items, (int64_t)sms * 2);
  if (grid < 1) return HEGRID_OK;
  k_grid_f32<<<(unsigned)grid, kThreads, sizeof(SmemF32), s>>>(jt);
  count_launch();
  HG_CUDA_TRY(launch_status());
  return HEGRID_OK;
}

}  // namespace hg
