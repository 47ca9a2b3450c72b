// Tensor-core form of the cell update (Eq. 1 accumulate + normalise) on
// tcgen05: per 16x8 cell block b and 256-channel tile, the sums
//     S[cell, c] = sum_k T[cell, k] V[k, c]
// run as dense MMAs over the block's candidate samples k (sorted spatially by
// the plan, 64 per chunk):  D[128 cells x 256 ch] (+)= A[128 x 16] * B[16 x 256]
// with A = the block's weight tile (built in shared memory from the plan's
// candidate-major entries) and B = the sample values of the chunk (K-major, so
// each channel row holds 64 samples).  FP32 accumulation lives in TMEM.
//
// Precision: values and weights are split into a high and a low 16-bit part;
// HEGRID_MODE_TC_SPLIT issues hi*hi + hi*lo + lo*hi (the lo*lo term is below
// FP32 rounding), HEGRID_MODE_TC issues hi*hi.  The 16-bit format is chosen
// per 64-sample chunk: FP16 (11-bit halves, ~2^-22 residual) when every value
// of the chunk lies in [2^-7, 2^15] in magnitude (zeros allowed) -- or, for
// BF16 input, when FP16 holds every value exactly -- and BF16 (8-bit halves,
// ~2^-17 residual, full FP32 range) otherwise.  Chunks of one block may mix
// formats: each MMA carries its own instruction descriptor and all of them
// accumulate in FP32.  W is accumulated by the same MMAs against a tile of
// ones, so the map is normalised by the sum of exactly the quantised weights
// that produced S.
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
constexpr uint32_t kTmemCols = 512;        // S in [0,256), W in [256,272)
constexpr uint32_t kWCol = 256;

struct __align__(1024) TcSmem {
  uint8_t A[2][2][kM * 128];   // [stage][hi, lo]: weight tiles, K-major, 128B swizzle
  uint8_t B[2][2][kN * 128];   // [stage][hi, lo]: value tiles, K-major, 128B swizzle
  uint8_t ones[2][16 * 128];   // [bf16, f16] all-ones B operand for W
  uint32_t red[2][kProducerWarps][3];  // per stage and warp: max|v|, min|v|>0, non-finite
  uint32_t fmt16[2];                   // per stage: 1 = FP16 tiles, 0 = BF16 tiles
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

// The value a raw element encodes (dtype of the input).
__device__ __forceinline__ float value_of(uint32_t x, int32_t dtype) {
  switch (dtype) {
    case HEGRID_F32: return __uint_as_float(x);
    case HEGRID_BF16X2:
      return __bfloat162float(__ushort_as_bfloat16((uint16_t)(x & 0xffffu))) +
             __bfloat162float(__ushort_as_bfloat16((uint16_t)(x >> 16)));
    case HEGRID_BF16: return __bfloat162float(__ushort_as_bfloat16((uint16_t)x));
    default: return __half2float(__ushort_as_half((uint16_t)x));
  }
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
  // ones tiles (bf16 1.0 = 0x3f80, f16 1.0 = 0x3c00)
  for (int i = tid; i < 16 * 128 / 4; i += kThreads) {
    reinterpret_cast<uint32_t*>(S.ones[0])[i] = 0x3f803f80u;
    reinterpret_cast<uint32_t*>(S.ones[1])[i] = 0x3c003c00u;
  }
  fence_proxy_async_smem();
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
    const bool vsplit = split && (J.dtype == HEGRID_F32 || J.dtype == HEGRID_BF16X2);

    if (warp == kProducerWarps) {
      // ---------------- MMA issuer ----------------
      if (n_chunks > 0) {
        if (n_tm > 0 && !mbar_wait(&S.tfree, (n_tm - 1) & 1u, err)) {
          bail = true;
        }
        tc_fence_after();
        const uint32_t idS16 = idesc_f16(0u, kM, kN), idW16 = idesc_f16(0u, kM, 16);
        const uint32_t idSbf = idesc_f16(1u, kM, kN), idWbf = idesc_f16(1u, kM, 16);
        for (int j = 0; j < n_chunks && !bail; ++j, ++g) {
          const int s = g & 1;
          if (!mbar_wait(&S.full[s], (g >> 1) & 1u, err)) {
            bail = true;
            break;
          }
          tc_fence_after();
          if (lane == 0) {
            const bool h = S.fmt16[s] != 0u;
            const uint32_t idS = h ? idS16 : idSbf, idW = h ? idW16 : idWbf;
            const uint32_t a_hi = smem_u32(S.A[s][0]), a_lo = smem_u32(S.A[s][1]);
            const uint32_t b_hi = smem_u32(S.B[s][0]), b_lo = smem_u32(S.B[s][1]);
            const uint32_t on = smem_u32(S.ones[h ? 1 : 0]);
#pragma unroll
            for (int kk = 0; kk < kK / 16; ++kk) {
              const uint32_t o = kk * 32;
              const uint32_t acc = (j > 0 || kk > 0) ? 1u : 0u;
              tc_mma_f16(tmem, smem_desc_k_sw128(a_hi + o), smem_desc_k_sw128(b_hi + o), idS, acc);
              if (vsplit)
                tc_mma_f16(tmem, smem_desc_k_sw128(a_hi + o), smem_desc_k_sw128(b_lo + o), idS, 1u);
              if (split)
                tc_mma_f16(tmem, smem_desc_k_sw128(a_lo + o), smem_desc_k_sw128(b_hi + o), idS, 1u);
              tc_mma_f16(tmem + kWCol, smem_desc_k_sw128(a_hi + o), smem_desc_k_sw128(on + o), idW,
                         acc);
              if (split)
                tc_mma_f16(tmem + kWCol, smem_desc_k_sw128(a_lo + o), smem_desc_k_sw128(on + o),
                           idW, 1u);
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
      // Values of this thread's channel row: all 64 loads issued first.
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
      // Range of the chunk's values (decides the 16-bit format of the chunk).
      {
        float amax = 0.0f, amin = __int_as_float(0x7f800000);
        uint32_t bad = 0u;
#pragma unroll
        for (int k = 0; k < kK; ++k) {
          const float a = fabsf(value_of(raw[k], J.dtype));
          bad |= (a <= 3.0e38f) ? 0u : 1u;  // NaN or Inf
          amax = fmaxf(amax, a);
          if (a > 0.0f) amin = fminf(amin, a);
        }
        const uint32_t wmax = __reduce_max_sync(0xffffffffu, __float_as_uint(amax));
        const uint32_t wmin = __reduce_min_sync(0xffffffffu, __float_as_uint(amin));
        const uint32_t wbad = __reduce_or_sync(0xffffffffu, bad);
        if (lane == 0) {
          S.red[s][warp][0] = wmax;
          S.red[s][warp][1] = wmin;
          S.red[s][warp][2] = wbad;
        }
      }
      // A tiles: zero (the scatter follows the barrier)
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
      bool h16;
      {
        uint32_t mx = 0u, mn = 0x7f800000u, bd = 0u;
#pragma unroll
        for (int w = 0; w < kProducerWarps; ++w) {
          mx = max(mx, S.red[s][w][0]);
          mn = min(mn, S.red[s][w][1]);
          bd |= S.red[s][w][2];
        }
        const float fmx = __uint_as_float(mx), fmn = __uint_as_float(mn);
        if (J.dtype == HEGRID_F16) {
          h16 = true;
        } else if (bd) {
          h16 = false;
        } else if (J.dtype == HEGRID_BF16) {
          h16 = fmx <= 32768.0f && (mn == 0x7f800000u || fmn >= 6.103515625e-05f);
        } else {
          h16 = fmx <= 32768.0f && (fmx == 0.0f || fmx >= 0.0078125f);
        }
        if (tid == 0) S.fmt16[s] = h16 ? 1u : 0u;
      }
      // B tiles: row tid holds the 64 samples of channel c
      {
        const uint32_t bh = smem_u32(S.B[s][0]), bl = smem_u32(S.B[s][1]);
#pragma unroll
        for (int q = 0; q < kK / 8; ++q) {
          uint32_t h2[4], l2[4];
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            uint16_t h0, l0, h1, l1;
            const uint32_t x0 = raw[q * 8 + e], x1 = raw[q * 8 + e + 1];
            if (J.dtype == HEGRID_F16 || (J.dtype == HEGRID_BF16 && !h16)) {
              h0 = (uint16_t)x0;  // stored format already matches the chunk format
              h1 = (uint16_t)x1;
              l0 = l1 = 0;
            } else {
              const float v0 = value_of(x0, J.dtype), v1 = value_of(x1, J.dtype);
              if (h16) {
                split_f16(v0, h0, l0);
                split_f16(v1, h1, l1);
              } else {
                split_bf16(v0, h0, l0);
                split_bf16(v1, h1, l1);
              }
            }
            h2[e / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
            l2[e / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
          }
          st_shared_v4(bh + sw128(tid, q), h2[0], h2[1], h2[2], h2[3]);
          if (vsplit) st_shared_v4(bl + sw128(tid, q), l2[0], l2[1], l2[2], l2[3]);
        }
      }
      // A tiles: scatter the chunk's weight entries
      {
        const int64_t e0 = pv.sub_off[sub0 + 2 * j], e1 = pv.sub_off[sub0 + 2 * j + 2];
        uint8_t* ah = S.A[s][0];
        uint8_t* al = S.A[s][1];
        for (int64_t e = e0 + tid; e < e1; e += kProducers) {
          const uint32_t ck = pv.ent_ck[e];
          const int r = (int)(ck >> 6), k = (int)(ck & 63u);
          const float w = pv.ent_w[e];
          uint16_t hi, lo;
          if (h16)
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
      uint32_t r[32];
      tmem_ld_32x32b_x32(tl + kWCol, r);
      tmem_ld_wait();
      const float W = __uint_as_float(r[0]);
      const bool ok = W > 0.0f;
#pragma unroll 1
      for (int cb = 0; cb < kN / 32; ++cb) {
        tmem_ld_32x32b_x32(tl + cb * 32, r);
        tmem_ld_wait();
        if (active) {
          const int64_t cbase = c0 + cb * 32;
          float v[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = ok ? __fdiv_rn(__uint_as_float(r[i]), W) : qnan;
          if (cbase + 32 <= C && (((uintptr_t)(out + cbase) & 15u) == 0)) {
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              *reinterpret_cast<float4*>(out + cbase + i) =
                  make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
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
