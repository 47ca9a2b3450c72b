// Plain FP32 form of the cell update (Algorithm 1's accumulate and normalise
// steps, Eq. 1) on CUDA cores.
//
// A persistent CTA takes work items (field, 16x8 cell block, 128-channel tile)
// in a fixed stride, in the job's work order (the channel tiles of a block
// back to back, or channel tiles slowest with the blocks in bands of block
// columns).  For each K chunk of 32 candidate samples of the block:
//   * warp 0 stages the 32 sample rows (FP32, channel-contiguous) into shared
//     memory with bulk async copies (TMA engine, one row per lane) completing
//     on an mbarrier, double-buffered;
//   * each of 128 threads scatters its cell's pairs that fall in the chunk
//     into a dense 32 x 128 weight tile and ORs a per-patch occupancy mask;
//   * each warp owns a 4x4-cell patch and 128 channels; a thread accumulates
//     8 cells x 8 channels in registers, skipping samples that touch no cell
//     of its patch.
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
constexpr int kPre = 6;   // weight entries prefetched per thread and chunk

struct __align__(128) SmemF32 {
  float V[2][kKC][kCT];   // staged sample rows
  float Wt[2][kKC][kCT];  // dense weight tile [k][cell column]
  uint32_t pmask[2][kKC];  // per sample k: bit p set if any cell of patch p has it
  uint64_t bar[2];
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
  __syncthreads();
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
    const uint32_t row_bytes = (uint32_t)(((cw + 3) & ~3) * 4);
    const float* __restrict__ vals = static_cast<const float*>(J.values);
    const int bbx = (int)(b % pv.nbx_b), bby = (int)(b / pv.nbx_b);
    const int64_t kb0 = pv.cand_off[b];
    const int n_chunks = pv.cand_cnt[b] / kKC;

    const int64_t sub0 = kb0 / kKC;  // first 32-candidate sub-chunk of the block

    // Stage the 32 sample rows of chunk j: warp 0, one row per lane.
    auto issue = [&](int j) {
      const int s = j & 1;
      if (lane == 0) mbar_arrive_expect_tx(&S.bar[s], row_bytes * kKC);
      __syncwarp();
      const int32_t n = pv.cand_idx[kb0 + (int64_t)j * kKC + lane];
      bulk_g2s(&S.V[s][lane][0], vals + (int64_t)n * J.ld_values + c0, row_bytes, &S.bar[s]);
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[i][e] = 0.0f;

    const int patch = warp, cs = lane >> 4, cg = lane & 15;
    if (warp == 0 && n_chunks > 0) issue(0);
    int64_t e_lo = 0, e_hi = 0;
    if (n_chunks > 0) {
      e_lo = pv.sub_off[sub0];
      e_hi = pv.sub_off[sub0 + 1];
    }
    for (int j = 0; j < n_chunks; ++j) {
      const int s = j & 1;
      if (warp == 0 && j + 1 < n_chunks) issue(j + 1);
      // The chunk's weight entries, loaded before the tile is cleared so the
      // loads' latency overlaps the clearing and the barrier.
      uint32_t pck[kPre];
      float pw[kPre];
#pragma unroll
      for (int i = 0; i < kPre; ++i) {
        const int64_t e = e_lo + tid + (int64_t)i * kThreads;
        pck[i] = e < e_hi ? (uint32_t)__ldg(pv.ent_ck + e) : 0xffffffffu;
        pw[i] = e < e_hi ? __ldg(pv.ent_w + e) : 0.0f;
      }
      const int64_t e_next = j + 1 < n_chunks ? __ldg(pv.sub_off + sub0 + j + 2) : 0;
      // weight tile for chunk j: zero, then scatter the chunk's entries
      {
        float4* wz = reinterpret_cast<float4*>(&S.Wt[s][0][0]);
        for (int i = tid; i < kKC * kCT / 4; i += kThreads) wz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tid < kKC) S.pmask[s][tid] = 0u;
      }
      __syncthreads();
      {
        auto put = [&](uint32_t ck, float w) {
          int col, k;
          tile_rk(ck, col, k);
          const int tc = cell_to_col(col % HG_BX, col / HG_BX);
          S.Wt[s][k][tc] = w;
          atomicOr(&S.pmask[s][k], 1u << (tc >> 4));
        };
#pragma unroll
        for (int i = 0; i < kPre; ++i)
          if (pck[i] != 0xffffffffu) put(pck[i], pw[i]);
        for (int64_t e = e_lo + tid + (int64_t)kPre * kThreads; e < e_hi; e += kThreads)
          put(pv.ent_ck[e], pv.ent_w[e]);
        e_lo = e_hi;
        e_hi = e_next;
      }
      __syncthreads();
      const int timed_out = !mbar_wait(&S.bar[s], phase[s], pv.err_word);
      if (__syncthreads_or(timed_out)) {
        // give up: wait (bounded) for the other stage's copies, then leave
        if (tid == 0 && j + 1 < n_chunks) mbar_wait(&S.bar[s ^ 1], phase[s ^ 1], nullptr);
        bail = true;
        break;
      }
      phase[s] ^= 1u;
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
      __syncthreads();
    }

    if (bail) break;
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
  HG_CUDA_TRY(cudaGetLastError());
  return HEGRID_OK;
}

}  // namespace hg
