// Tensor-core form of the cell update (Eq. 1 accumulate + normalise) on
// tcgen05: per 16x8 cell block b and 256-channel tile, the sums
//     S[cell, c] = sum_k T[cell, k] V[k, c]
// run as dense MMAs over the block's candidate samples k (sorted spatially by
// the plan, 64 per chunk):  D[128 cells x 256 ch] (+)= A[128 x 16] * B[16 x 256]
// with A = the block's weight tile (built in shared memory from the plan's
// candidate-major entries) and B = the sample values of the chunk (K-major, so
// each channel row holds 64 samples).  FP32 accumulation lives in TMEM.
//
// Precision: values and weights are split into a high and a low 16-bit part
// (BF16, or FP16 for F16 input); HEGRID_MODE_TC_SPLIT issues hi*hi + hi*lo +
// lo*hi (the lo*lo term is below FP32 rounding), HEGRID_MODE_TC issues hi*hi.
// The main term and the two correction terms accumulate in separate TMEM
// regions (a small term added into a large FP32 accumulator loses its low
// bits), summed once in the epilogue.  W is the plan's compensated sum of
// exactly the quantised weights (hi, or hi + lo) that produced S.
//
// CTA: 8 producer warps (values -> B tiles, entries -> A tiles, 2-stage
// ring), warps 0-3 also run the epilogue (TMEM -> registers -> S / W ->
// global), and warp 8 allocates TMEM and issues the MMAs (one lane).
// Stages are handed over with mbarriers; MMA completion is signalled by
// tcgen05.commit.  Every wait is bounded (global timer) and reports a timeout
// through the plan's error word.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "hegrid_internal.cuh"
#include "ptx.cuh"

namespace hg {
namespace {

constexpr int kProducerWarps = 8;
constexpr int kProducers = kProducerWarps * 32;
constexpr int kThreads = kProducers + 32;  // + the MMA warp
constexpr int kK = 64;                     // candidates per chunk (one 128-byte row of BF16)
constexpr int kN = 256;                    // channels per tile
constexpr int kM = HG_BLOCK_CELLS;         // cells per block
constexpr uint32_t kTmemCols = 512;        // main sums in [0,256), corrections in [256,512)
constexpr uint32_t kCorrCol = 256;

struct __align__(1024) TcSmem {
  uint8_t A[2][2][kM * 128];   // [stage][hi, lo]: weight tiles, K-major, 128B swizzle
  uint8_t B[2][2][kN * 128];   // [stage][hi, lo]: value tiles, K-major, 128B swizzle
  uint64_t full[2], empty[2], done, tfree;
  uint32_t tmem_base;
};

// Byte offset of 16-byte chunk q of row r in a K-major, 128B-swizzled tile.
__device__ __forceinline__ uint32_t sw128(int r, int q) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((q ^ (r & 7)) << 4));
}

__device__ __forceinline__ int find_job(const JobTable& jt, int64_t item) {
  int j = 0;
  while (j + 1 < jt.n_jobs && jt.job[j + 1].item_base <= item) ++j;
  return j;
}

// Split x into hi + lo 16-bit floats (round to nearest for both parts).
__device__ __forceinline__ void split_bf16(float x, uint16_t& hi, uint16_t& lo) {
  __nv_bfloat16 h = __float2bfloat16_rn(x);
  __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = __bfloat16_as_ushort(h);
  lo = __bfloat16_as_ushort(l);
}

__device__ __forceinline__ void split_f16(float x, uint16_t& hi, uint16_t& lo) {
  __half h = __float2half_rn(x);
  __half l = __float2half_rn(x - __half2float(h));
  hi = __half_as_ushort(h);
  lo = __half_as_ushort(l);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

__device__ __forceinline__ void named_bar_producers() {
  asm volatile("bar.sync 1, %0;" ::"r"(kProducers) : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) k_grid_tc(const __grid_constant__ JobTable jt) {
  extern __shared__ unsigned char smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t* err = jt.job[0].pv.err_word;

  if (tid == 0) {
    mbar_init(&S.full[0], kProducerWarps);
    mbar_init(&S.full[1], kProducerWarps);
    mbar_init(&S.empty[0], 1);
    mbar_init(&S.empty[1], 1);
    mbar_init(&S.done, 1);
    mbar_init(&S.tfree, 4);
    fence_mbar_init();
  }
  if (warp == kProducerWarps) {
    tmem_alloc(&S.tmem_base, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  bool bail = false;
  uint32_t g = 0;        // chunks produced / consumed so far (stage = g & 1)
  uint32_t n_tm = 0;     // items that used TMEM so far

  for (int64_t item = blockIdx.x; item < jt.n_items && !bail; item += gridDim.x) {
    const GridJob& J = jt.job[find_job(jt, item)];
    const PlanView& pv = J.pv;
    const int64_t local = item - J.item_base;
    const int64_t b = local / J.n_ctiles;
    const int64_t c0 = (local % J.n_ctiles) * kN;
    const int64_t kb0 = pv.cand_off[b];
    const int n_chunks = (int)((pv.cand_off[b + 1] - kb0) / kK);
    const bool split = J.mode == HEGRID_MODE_TC_SPLIT;
    const bool f16 = J.dtype == HEGRID_F16;
    const bool vsplit = split && (J.dtype == HEGRID_F32 || J.dtype == HEGRID_BF16X2);

    if (warp == kProducerWarps) {
      // ---------------- MMA issuer ----------------
      if (n_chunks > 0) {
        if (n_tm > 0 && !mbar_wait(&S.tfree, (n_tm - 1) & 1u, err)) {
          bail = true;
        }
        tc_fence_after();
        const uint32_t fmt = f16 ? 0u : 1u;
        const uint32_t idS = idesc_f16(fmt, kM, kN);
        for (int j = 0; j < n_chunks && !bail; ++j, ++g) {
          const int s = g & 1;
          if (!mbar_wait(&S.full[s], (g >> 1) & 1u, err)) {
            bail = true;
            break;
          }
          tc_fence_after();
          if (lane == 0) {
            const uint32_t a_hi = smem_u32(S.A[s][0]), a_lo = smem_u32(S.A[s][1]);
            const uint32_t b_hi = smem_u32(S.B[s][0]), b_lo = smem_u32(S.B[s][1]);
#pragma unroll
            for (int kk = 0; kk < kK / 16; ++kk) {
              const uint32_t o = kk * 32;
              const uint32_t first = (j == 0 && kk == 0) ? 1u : 0u;
              // main term and the two correction terms in separate accumulators
              tc_mma_f16(tmem, smem_desc_k_sw128(a_hi + o), smem_desc_k_sw128(b_hi + o), idS,
                         1u - first);
              if (vsplit)
                tc_mma_f16(tmem + kCorrCol, smem_desc_k_sw128(a_hi + o),
                           smem_desc_k_sw128(b_lo + o), idS, 1u - first);
              if (split)
                tc_mma_f16(tmem + kCorrCol, smem_desc_k_sw128(a_lo + o),
                           smem_desc_k_sw128(b_hi + o), idS, vsplit ? 1u : 1u - first);
            }
            tc_commit(&S.empty[s]);
            if (j == n_chunks - 1) tc_commit(&S.done);
          }
          __syncwarp();
        }
        ++n_tm;
      }
      continue;
    }

    // ---------------- producers (warps 0-7) ----------------
    const int64_t C = J.C;
    const int64_t c = c0 + tid;  // this thread's channel = B row `tid`
    const bool cvalid = c < C;
    const int64_t sub0 = kb0 / 32;
    for (int j = 0; j < n_chunks && !bail; ++j, ++g) {
      const int s = g & 1;
      const uint32_t u = g >> 1;
      if (u >= 1 && !mbar_wait(&S.empty[s], (u - 1) & 1u, err)) {
        bail = true;
        break;
      }
      // B tiles: row tid holds 64 samples of channel c.  All 64 loads are
      // issued before any conversion (memory-level parallelism).
      {
        const int32_t* ci = pv.cand_idx + kb0 + (int64_t)j * kK;
        uint32_t raw[kK];
        if (J.dtype == HEGRID_F32 || J.dtype == HEGRID_BF16X2) {
          const uint32_t* vp = static_cast<const uint32_t*>(J.values);
#pragma unroll
          for (int k = 0; k < kK; ++k)
            raw[k] = cvalid ? __ldg(vp + (int64_t)__ldg(ci + k) * J.ld_values + c) : 0u;
        } else {
          const uint16_t* vp = static_cast<const uint16_t*>(J.values);
#pragma unroll
          for (int k = 0; k < kK; ++k)
            raw[k] = cvalid ? (uint32_t)__ldg(vp + (int64_t)__ldg(ci + k) * J.ld_values + c) : 0u;
        }
        const uint32_t bh = smem_u32(S.B[s][0]), bl = smem_u32(S.B[s][1]);
#pragma unroll
        for (int q = 0; q < kK / 8; ++q) {
          uint32_t h2[4], l2[4];
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            uint16_t h0, l0, h1, l1;
            const uint32_t x0 = raw[q * 8 + e], x1 = raw[q * 8 + e + 1];
            if (J.dtype == HEGRID_F32) {
              if (vsplit) {
                split_bf16(__uint_as_float(x0), h0, l0);
                split_bf16(__uint_as_float(x1), h1, l1);
              } else {
                h0 = __bfloat16_as_ushort(__float2bfloat16_rn(__uint_as_float(x0)));
                h1 = __bfloat16_as_ushort(__float2bfloat16_rn(__uint_as_float(x1)));
                l0 = l1 = 0;
              }
            } else if (J.dtype == HEGRID_BF16X2) {
              h0 = (uint16_t)(x0 & 0xffffu);
              l0 = (uint16_t)(x0 >> 16);
              h1 = (uint16_t)(x1 & 0xffffu);
              l1 = (uint16_t)(x1 >> 16);
            } else {
              h0 = (uint16_t)x0;
              h1 = (uint16_t)x1;
              l0 = l1 = 0;
            }
            h2[e / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
            l2[e / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
          }
          st_shared_v4(bh + sw128(tid, q), h2[0], h2[1], h2[2], h2[3]);
          if (vsplit) st_shared_v4(bl + sw128(tid, q), l2[0], l2[1], l2[2], l2[3]);
        }
      }
      // A tiles: zero, then scatter the chunk's weight entries
      {
        uint4* ah = reinterpret_cast<uint4*>(S.A[s][0]);
        uint4* al = reinterpret_cast<uint4*>(S.A[s][1]);
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        for (int i = tid; i < kM * 128 / 16; i += kProducers) {
          ah[i] = z;
          if (split) al[i] = z;
        }
      }
      named_bar_producers();
      {
        const int64_t e0 = pv.sub_off[sub0 + 2 * j], e1 = pv.sub_off[sub0 + 2 * j + 2];
        uint8_t* ah = S.A[s][0];
        uint8_t* al = S.A[s][1];
        for (int64_t e = e0 + tid; e < e1; e += kProducers) {
          const uint32_t ck = pv.ent_ck[e];
          const int r = (int)(ck >> 6), k = (int)(ck & 63u);
          const float w = pv.ent_w[e];
          uint16_t hi, lo;
          if (f16)
            split_f16(w, hi, lo);
          else
            split_bf16(w, hi, lo);
          const uint32_t off = sw128(r, k >> 3) + (k & 7) * 2;
          *reinterpret_cast<uint16_t*>(ah + off) = hi;
          if (split) *reinterpret_cast<uint16_t*>(al + off) = lo;
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.full[s]);
    }
    if (bail) break;

    // ---------------- epilogue (warps 0-3) ----------------
    if (warp < 4) {
      const int row = warp * 32 + lane;
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
      if (!mbar_wait(&S.done, (n_tm & 1u), err)) {
        bail = true;
        break;
      }
      ++n_tm;
      tc_fence_after();
      const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
      const int wvar = f16 ? (split ? 4 : 3) : (split ? 2 : 1);
      const float W = active ? pv.wsum[(int64_t)wvar * pv.M + m] : 0.0f;
      const bool ok = W > 0.0f;
      uint32_t r[32], rc[32];
#pragma unroll 1
      for (int cb = 0; cb < kN / 32; ++cb) {
        tmem_ld_32x32b_x32(tl + cb * 32, r);
        if (split) tmem_ld_32x32b_x32(tl + kCorrCol + cb * 32, rc);
        tmem_ld_wait();
        if (active) {
          const int64_t cbase = c0 + cb * 32;
          float v[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float sum = split ? __fadd_rn(__uint_as_float(r[i]), __uint_as_float(rc[i]))
                                    : __uint_as_float(r[i]);
            v[i] = ok ? __fdiv_rn(sum, W) : qnan;
          }
          if (cbase + 32 <= C && (((uintptr_t)(out + cbase) & 15u) == 0)) {
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              *reinterpret_cast<float4*>(out + cbase + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (cbase + i < C) out[cbase + i] = v[i];
          }
        }
      }
      if (active && c0 == 0 && J.weight_out) J.weight_out[m] = W;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.tfree);
    } else if (n_chunks > 0) {
      ++n_tm;
    }
  }

  // drain: make sure no MMA is still writing TMEM before it is freed
  if (warp == kProducerWarps && n_tm > 0 && !bail) mbar_wait(&S.done, (n_tm - 1) & 1u, nullptr);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kProducerWarps) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

int tc_channel_tile() { return kN; }

hegrid_status launch_grid_tc(const JobTable& jt, cudaStream_t s) {
  static int sms = 0;
  const size_t smem = sizeof(TcSmem) + 1024;
  if (!sms) {
    int dev;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    HG_CUDA_TRY(cudaFuncSetAttribute(k_grid_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  }
  int64_t grid = std::min<int64_t>(jt.n_items, (int64_t)sms);
  if (grid < 1) return HEGRID_OK;
  k_grid_tc<<<(unsigned)grid, kThreads, smem, s>>>(jt);
  count_launch();
  HG_CUDA_TRY(cudaGetLastError());
  return HEGRID_OK;
}

}  // namespace hg
