// C ABI of the grid step: validation, work-item tables, batched launches,
// CUDA-graph batches and host-chunk streaming.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hegrid_internal.cuh"
#include "ptx.cuh"

namespace hg {
namespace {

// Rows of `row_units` words, dense in `src`, copied to rows `pitch_units`
// words apart in `dst` (the padding words are left as they are).  Host chunks
// whose rows are not a multiple of 16 bytes arrive by one dense copy and are
// spread to the grid kernels' 16-byte row pitch here, instead of by a 2-D
// copy, whose per-row transfers run the host link at a few GB/s for rows of
// a few hundred bytes.
template <typename U>
__global__ void __launch_bounds__(256) k_pad_rows(const U* __restrict__ src, U* __restrict__ dst,
                                                  int64_t n_units, int64_t row_units,
                                                  int64_t pitch_units) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_units; i += stride) {
    const int64_t r = i / row_units;
    dst[r * pitch_units + (i - r * row_units)] = src[i];
  }
}

cudaError_t pad_rows(const void* src, void* dst, int64_t n_rows, int64_t row_bytes,
                     int64_t pitch_bytes, int n_sm, cudaStream_t s) {
  const int blocks = std::max(1, n_sm) * 8;
  if (row_bytes % 8 == 0) {
    k_pad_rows<uint2><<<blocks, 256, 0, s>>>((const uint2*)src, (uint2*)dst, n_rows * (row_bytes / 8),
                                             row_bytes / 8, pitch_bytes / 8);
  } else if (row_bytes % 4 == 0) {
    k_pad_rows<uint32_t><<<blocks, 256, 0, s>>>((const uint32_t*)src, (uint32_t*)dst,
                                                n_rows * (row_bytes / 4), row_bytes / 4,
                                                pitch_bytes / 4);
  } else {
    k_pad_rows<uint16_t><<<blocks, 256, 0, s>>>((const uint16_t*)src, (uint16_t*)dst,
                                                n_rows * (row_bytes / 2), row_bytes / 2,
                                                pitch_bytes / 2);
  }
  count_launch();
  return launch_status();
}

// Per-channel masking, step 1: values with every non-finite entry replaced by
// 0 (same type and layout as the input) and the 0/1 finiteness mask (FP32 or
// BF16, rows ld_mask apart).  A BF16 hi/lo pair is finite if both halves are.
__device__ __forceinline__ bool bits_finite(uint32_t v, int dtype) {
  switch (dtype) {
    case HEGRID_F32: return (v & 0x7f800000u) != 0x7f800000u;
    case HEGRID_BF16: return (v & 0x7f80u) != 0x7f80u;
    case HEGRID_F16: return (v & 0x7c00u) != 0x7c00u;
    default: return (v & 0x7f80u) != 0x7f80u && (v & 0x7f800000u) != 0x7f800000u;  // BF16X2
  }
}

__global__ void __launch_bounds__(256) k_mask_split(const void* __restrict__ values, int dtype,
                                                    int64_t n_rows, int64_t C, int64_t ld,
                                                    void* __restrict__ clean,
                                                    void* __restrict__ mask, int mask_f32,
                                                    int64_t ld_mask) {
  const int64_t total = n_rows * C, stride = (int64_t)gridDim.x * blockDim.x;
  const bool wide = dtype == HEGRID_F32 || dtype == HEGRID_BF16X2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t n = i / C, c = i - n * C;
    const int64_t at = n * ld + c;
    bool ok;
    if (wide) {
      const uint32_t v = static_cast<const uint32_t*>(values)[at];
      ok = bits_finite(v, dtype);
      static_cast<uint32_t*>(clean)[at] = ok ? v : 0u;
    } else {
      const uint16_t v = static_cast<const uint16_t*>(values)[at];
      ok = bits_finite(v, dtype);
      static_cast<uint16_t*>(clean)[at] = ok ? v : (uint16_t)0;
    }
    if (mask_f32)
      static_cast<float*>(mask)[n * ld_mask + c] = ok ? 1.0f : 0.0f;
    else
      static_cast<uint16_t*>(mask)[n * ld_mask + c] = ok ? (uint16_t)0x3f80u : (uint16_t)0;
  }
}

// Step 3: map = (S_c / W) / (W_c / W) = S_c / W_c, NaN where W_c = 0; the
// per-channel weight sums W_c = (W_c / W) * W from the plan's W.
__global__ void __launch_bounds__(256) k_mask_divide(float* __restrict__ map, int64_t ld_map,
                                                     const float* __restrict__ q, int64_t M,
                                                     int64_t C, const float* __restrict__ W,
                                                     float* __restrict__ wc_out) {
  const int64_t total = M * C, stride = (int64_t)gridDim.x * blockDim.x;
  const float qnan = __int_as_float(0x7fc00000);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t m = i / C, c = i - m * C;
    const float r = q[i];
    const bool has = r > 0.0f;  // false for 0 and NaN (W = 0)
    float* o = map + m * ld_map + c;
    *o = has ? __fdiv_rn(*o, r) : qnan;
    if (wc_out) wc_out[m * ld_map + c] = has ? __fmul_rn(r, W[m]) : 0.0f;
  }
}

// Largest |v| of each channel, for the tensor-core forms' per-channel scale,
// for every entry of a batch in one launch: out[c] = max(out[c], |v[n, c]|
// over a CTA's rows) as the bits of a non-negative float (they order like the
// floats; NaN is dropped by fmaxf, Inf kept).  Each thread reads 16-byte
// vectors (kVec values) of one channel group, `cols` groups per CTA side by
// side and 256 / cols rows at a time; an entry's CTAs cover its channel groups
// (gy) times its row ranges (gx).  One atomicMax per channel and CTA, after a
// shared-memory reduction over the CTA's rows.
struct AbsmaxJob {
  const void* values;
  uint32_t* out;
  int64_t N, C, ld, rows_per_cta;
  int32_t dtype, nvec, cols, gy;
  int64_t block_base;  // first CTA of this entry
};
constexpr int kMaxAbsmaxJobs = kMaxJobs;
constexpr int kAbsmaxLeanThreads = 128;
struct AbsmaxTable {
  int32_t n;
  AbsmaxJob job[kMaxAbsmaxJobs];
};

template <int DT>
__device__ __forceinline__ void absmax_rows(const AbsmaxJob& J, int64_t cv, int64_t r0, int64_t r1,
                                            int rl, int rpt, float (&m)[8]) {
  constexpr bool kWide = DT == HEGRID_F32 || DT == HEGRID_BF16X2;
  const uint4* base =
      reinterpret_cast<const uint4*>(static_cast<const char*>(J.values) + (cv * 16));
  const int64_t pitch = J.ld * (kWide ? 4 : 2) / 16;  // row pitch in 16-byte vectors
#pragma unroll 4
  for (int64_t r = r0 + rl; r < r1; r += rpt) {
    const uint4 q = __ldcs(base + r * pitch);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (DT == HEGRID_F32) {
        m[i] = fmaxf(m[i], fabsf(__uint_as_float(w[i])));
      } else if (DT == HEGRID_BF16X2) {
        const float v = __uint_as_float(w[i] << 16) + __uint_as_float(w[i] & 0xffff0000u);
        m[i] = fmaxf(m[i], fabsf(v));
      } else if (DT == HEGRID_BF16) {
        m[2 * i] = fmaxf(m[2 * i], fabsf(__uint_as_float(w[i] << 16)));
        m[2 * i + 1] = fmaxf(m[2 * i + 1], fabsf(__uint_as_float(w[i] & 0xffff0000u)));
      } else {  // F16
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[i]));
        m[2 * i] = fmaxf(m[2 * i], fabsf(f.x));
        m[2 * i + 1] = fmaxf(m[2 * i + 1], fabsf(f.y));
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_chan_absmax(const __grid_constant__ AbsmaxTable tab) {
  __shared__ float red[256][8];
  int j = 0;
  while (j + 1 < tab.n && tab.job[j + 1].block_base <= (int64_t)blockIdx.x) ++j;
  const AbsmaxJob& J = tab.job[j];
  const int64_t local = (int64_t)blockIdx.x - J.block_base;
  const int64_t bx = local / J.gy, by = local - bx * J.gy;
  const int tid = threadIdx.x;
  const int cols = J.cols, rpt = 256 / cols;  // rows read side by side
  const int cslot = tid % cols, rl = tid / cols;
  const int64_t cv = by * cols + cslot;
  const int64_t r0 = bx * J.rows_per_cta;
  const int64_t r1 = r0 + J.rows_per_cta < J.N ? r0 + J.rows_per_cta : J.N;
  const bool wide = J.dtype == HEGRID_F32 || J.dtype == HEGRID_BF16X2;
  const int vec = wide ? 4 : 8;  // values per 16 bytes
  float m[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) m[e] = 0.0f;
  if (rl < rpt && cv < J.nvec) {
    switch (J.dtype) {
      case HEGRID_F32: absmax_rows<HEGRID_F32>(J, cv, r0, r1, rl, rpt, m); break;
      case HEGRID_BF16X2: absmax_rows<HEGRID_BF16X2>(J, cv, r0, r1, rl, rpt, m); break;
      case HEGRID_BF16: absmax_rows<HEGRID_BF16>(J, cv, r0, r1, rl, rpt, m); break;
      default: absmax_rows<HEGRID_F16>(J, cv, r0, r1, rl, rpt, m); break;
    }
  }
  if (rpt > 1) {
#pragma unroll
    for (int e = 0; e < 8; ++e) red[tid][e] = m[e];
    __syncthreads();
    if (tid < cols) {
      for (int k = 1; k < rpt; ++k)
#pragma unroll
        for (int e = 0; e < 8; ++e) m[e] = fmaxf(m[e], red[k * cols + tid][e]);
    }
  }
  if (rl == 0 && cv < J.nvec) {
    for (int e = 0; e < vec; ++e) {
      const int64_t c = cv * vec + e;
      if (c < J.C && m[e] > 0.0f) atomicMax(J.out + c, __float_as_uint(m[e]));
    }
  }
}

// The same maxima from one 128-thread CTA per SM, no shared memory and at
// most 32 registers a thread: each thread keeps its column group's maxima
// and adds them with atomicMax, so the pass leaves the SMs' shared memory and
// nearly all their registers and threads to kernels on other streams.
__global__ void __launch_bounds__(kAbsmaxLeanThreads, 16)
    k_chan_absmax_lean(const __grid_constant__ AbsmaxTable tab) {
  int j = 0;
  while (j + 1 < tab.n && tab.job[j + 1].block_base <= (int64_t)blockIdx.x) ++j;
  const AbsmaxJob& J = tab.job[j];
  const int64_t local = (int64_t)blockIdx.x - J.block_base;
  const int64_t bx = local / J.gy, by = local - bx * J.gy;
  const int tid = threadIdx.x;
  const int cols = J.cols, rpt = kAbsmaxLeanThreads / cols;
  const int cslot = tid % cols, rl = tid / cols;
  const int64_t cv = by * cols + cslot;
  const int64_t r0 = bx * J.rows_per_cta;
  const int64_t r1 = r0 + J.rows_per_cta < J.N ? r0 + J.rows_per_cta : J.N;
  const int vec = (J.dtype == HEGRID_F32 || J.dtype == HEGRID_BF16X2) ? 4 : 8;
  if (rl >= rpt || cv >= J.nvec) return;
  float m[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) m[e] = 0.0f;
  switch (J.dtype) {
    case HEGRID_F32: absmax_rows<HEGRID_F32>(J, cv, r0, r1, rl, rpt, m); break;
    case HEGRID_BF16X2: absmax_rows<HEGRID_BF16X2>(J, cv, r0, r1, rl, rpt, m); break;
    case HEGRID_BF16: absmax_rows<HEGRID_BF16>(J, cv, r0, r1, rl, rpt, m); break;
    default: absmax_rows<HEGRID_F16>(J, cv, r0, r1, rl, rpt, m); break;
  }
  for (int e = 0; e < vec; ++e) {
    const int64_t c = cv * vec + e;
    if (c < J.C && m[e] > 0.0f) atomicMax(J.out + c, __float_as_uint(m[e]));
  }
}

int elem_bytes(int dtype) {
  switch (dtype) {
    case HEGRID_F32: return 4;
    case HEGRID_BF16: return 2;
    case HEGRID_F16: return 2;
    case HEGRID_BF16X2: return 4;
    default: return 0;
  }
}

hegrid_status check_args(const hegrid_plan* plan, const hegrid_grid_args& a) {
  HG_ARG_CHECK(plan != nullptr, "plan is NULL");
  HG_ARG_CHECK(a.values != nullptr && a.map_out != nullptr, "values or map_out is NULL");
  HG_ARG_CHECK(a.n_channels >= 1, "n_channels must be >= 1");
  int eb = elem_bytes((int)a.dtype);
  HG_ARG_CHECK(eb > 0, "unknown dtype");
  HG_ARG_CHECK(a.ld_values >= a.n_channels, "ld_values < n_channels");
  HG_ARG_CHECK((a.ld_values * eb) % 16 == 0, "ld_values * element size must be a multiple of 16");
  HG_ARG_CHECK(((uintptr_t)a.values & 15u) == 0, "values must be 16-byte aligned");
  HG_ARG_CHECK(a.ld_map >= a.n_channels, "ld_map < n_channels");
  HG_ARG_CHECK(a.mode == HEGRID_MODE_FP32 || a.mode == HEGRID_MODE_TC ||
                   a.mode == HEGRID_MODE_TC_SPLIT,
               "unknown mode");
  if (a.mode == HEGRID_MODE_FP32 && a.dtype != HEGRID_F32) {
    set_error("HEGRID_MODE_FP32 needs HEGRID_F32 values");
    return HEGRID_ERR_UNSUPPORTED;
  }
  return HEGRID_OK;
}

GridJob make_job(const hegrid_plan* plan, const hegrid_grid_args& a, int64_t ctile) {
  GridJob j;
  std::memset(&j, 0, sizeof(j));
  j.pv = plan->view();
  j.values = a.values;
  j.dtype = (int32_t)a.dtype;
  j.mode = (int32_t)a.mode;
  j.C = a.n_channels;
  j.ld_values = a.ld_values;
  j.map = a.map_out;
  j.ld_map = a.ld_map;
  j.weight_out = a.weight_out;
  j.n_rows = plan->N;
  j.n_ctiles = (a.n_channels + ctile - 1) / ctile;
  if (a.mode == HEGRID_MODE_FP32) {
    j.band = plan->tune_f32_band;
    j.seg = 1;
  } else {
    j.band = plan->tune_tc_band != 0 ? plan->tune_tc_band : tc_default_band();
    j.seg = plan->tune_tc_seg > 0 ? plan->tune_tc_seg : tc_default_seg();
    j.group = plan->tune_tc_band != 0 ? plan->tune_tc_group : tc_default_group();
    // the block's height over its candidate window's (R on each side, plus up
    // to one bin of rounding), in map rows
    const double r_rows = plan->R_deg / plan->geom.dlat_deg;
    j.rot = (float)(HG_BY / (HG_BY + 2.0 * r_rows + plan->bin_cells));
  }
  return j;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// Encode j.rows for the tensor-core kernel (channel tile width `tile`).
hegrid_status encode_rows_map(GridJob& j, int tile) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return HEGRID_ERR_CUDA;
  }
  const bool wide = j.dtype == HEGRID_F32 || j.dtype == HEGRID_BF16X2;
  const int eb = wide ? 4 : 2;
  // The values as a 2-D array of raw 2- or 4-byte words: C channels (inner,
  // channels past C read as zero) x N sample rows, rows ld_values apart.
  cuuint64_t dims[2] = {(cuuint64_t)j.C, (cuuint64_t)j.n_rows};
  cuuint64_t strides[1] = {(cuuint64_t)j.ld_values * eb};
  cuuint32_t box[2] = {(cuuint32_t)tile, 1u}, estr[2] = {1u, 1u};
  CUresult r = enc(&j.rows, wide ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                   2, const_cast<void*>(j.values), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return HEGRID_ERR_CUDA;
  }
  return HEGRID_OK;
}

// Builds the plan's dense weight tiles (once; serialised by a host mutex)
// on stream s, after which `ready` is re-recorded on s so that every later
// user of the plan waits for them too.
hegrid_status ensure_wtiles(hegrid_plan* p, cudaStream_t s) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (p->wtiles) return HEGRID_OK;
  const int64_t bytes = tcm_wtile_bytes(p->slots);
  uint8_t* wt = nullptr;
  HG_CUDA_TRY(pool_alloc((void**)&wt, (size_t)std::max<int64_t>(bytes, 16), s));
  hegrid_plan tmp = *p;
  tmp.wtiles = wt;
  hegrid_status st = launch_build_wtiles(tmp.view(), wt, s);
  if (st != HEGRID_OK) {
    cudaFreeAsync(wt, s);
    return st;
  }
  HG_CUDA_TRY(cudaEventRecord(p->ready, s));
  p->wtiles = wt;
  p->bytes += bytes;
  return HEGRID_OK;
}

// The tensor-core kernel a job on plan p runs (1 cell-major, 2 channel-major,
// 3 cell-major with dense A tiles): the plan's choice (tune_tc_kernel, set
// by the caller or kept by the autotuner; 0, the default, is 1).  Kernels 2
// and 3 need the plan's dense weight tiles, built here if missing, except
// inside a stream capture, where the plain cell-major kernel runs until they
// exist.
hegrid_status tc_kernel_of(hegrid_plan* p, cudaStream_t s, int* kern) {
  *kern = 1;
  const int k = p->tune_tc_kernel;
  if (k != 2 && k != 3) return HEGRID_OK;
  if (!p->wtiles) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HG_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return HEGRID_OK;
    hegrid_status e = ensure_wtiles(p, s);
    if (e != HEGRID_OK) return e;
  }
  *kern = k;
  return HEGRID_OK;
}

// Launch all jobs of one kernel family (tile > 0: the cell-major
// tensor-core kernel of that channel tile; tile < 0: the channel-major one),
// kMaxJobs per launch.
hegrid_status launch_family(const std::vector<GridJob>& jobs, bool tc, cudaStream_t s,
                            int tile = 0, bool dense_a = false) {
  for (size_t base = 0; base < jobs.size(); base += kMaxJobs) {
    JobTable jt;
    std::memset(&jt, 0, sizeof(jt));
    jt.n_jobs = (int32_t)std::min<size_t>(kMaxJobs, jobs.size() - base);
    jt.inject = 0;
    jt.wait_ns = kWaitLimitNs;
    int64_t items = 0;
    for (int i = 0; i < jt.n_jobs; ++i) {
      jt.job[i] = jobs[base + i];
      jt.job[i].item_base = items;
      items += jt.job[i].pv.n_blocks * jt.job[i].n_ctiles;
    }
    jt.n_items = items;
    hegrid_status st = !tc ? launch_grid_f32(jt, s)
                       : tile < 0 ? launch_grid_tcm(jt, s)
                                  : launch_grid_tc(jt, s, tile, dense_a);
    if (st != HEGRID_OK) return st;
  }
  return HEGRID_OK;
}

// Channels of the entries whose tensor-core form scales each channel by a
// power of two (every dtype but FP16, which is exact as stored).
int64_t scaled_channels(int n, const hegrid_grid_args* args) {
  int64_t c = 0;
  for (int i = 0; i < n; ++i)
    if (args[i].mode != HEGRID_MODE_FP32 && args[i].dtype != HEGRID_F16) c += args[i].n_channels;
  return c;
}

// wait_ready: make `s` wait for each plan's creation (false inside a graph
// capture, where the caller has synchronised the plans on the host instead).
// chmax_buf: room for scaled_channels() channel maxima, or NULL to take it
// from the pool for this call; chmax_ready: chmax_buf already holds them
// (hegrid_chan_maxima), so the maximum pass is skipped.
hegrid_status grid_many(int n, hegrid_plan* const* plans, const hegrid_grid_args* args,
                        cudaStream_t s, bool wait_ready = true, uint32_t* chmax_buf = nullptr,
                        bool chmax_ready = false) {
  HG_ARG_CHECK(n >= 0, "n must be >= 0");
  HG_ARG_CHECK(n == 0 || (plans && args), "NULL plans or args");
  // tensor-core jobs grouped by kernel and channel tile (cell-major 64, 128,
  // 256, with A tiles built or from dense tiles; channel-major 128): one
  // launch each
  std::vector<GridJob> f32, tc[3], tcd[3], tcm;
  const int tiles[3] = {64, 128, 256};
  for (int i = 0; i < n; ++i) {
    hegrid_status st = check_args(plans[i], args[i]);
    if (st != HEGRID_OK) return st;
  }
  const int64_t n_scaled = scaled_channels(n, args);
  uint32_t* chmax = chmax_buf;
  if (n_scaled > 0 && chmax == nullptr)
    HG_CUDA_TRY(pool_alloc((void**)&chmax, sizeof(uint32_t) * (size_t)n_scaled, s));
  const bool own = chmax != chmax_buf;
  hegrid_status st = HEGRID_OK;
  std::vector<AbsmaxRequest> amax;
  auto run = [&]() -> hegrid_status {
    if (n_scaled > 0 && !chmax_ready)
      HG_CUDA_TRY(cudaMemsetAsync(chmax, 0, sizeof(uint32_t) * (size_t)n_scaled, s));
    int64_t at = 0;
    for (int i = 0; i < n; ++i) {
      if (wait_ready) HG_CUDA_TRY(cudaStreamWaitEvent(s, plans[i]->ready, 0));
      if (args[i].mode == HEGRID_MODE_FP32) {
        f32.push_back(make_job(plans[i], args[i], f32_channel_tile()));
        hegrid_status e = encode_rows_map(f32.back(), f32_channel_tile());
        if (e != HEGRID_OK) return e;
        continue;
      }
      int kern = 1;
      {
        hegrid_status e = tc_kernel_of(plans[i], s, &kern);
        if (e != HEGRID_OK) return e;
      }
      const bool cm = kern == 2;
      const int tile = cm ? tcm_channel_tile() : tc_channel_tile(args[i].n_channels);
      const int ti = tile == 64 ? 0 : tile == 128 ? 1 : 2;
      std::vector<GridJob>& fam = cm ? tcm : kern == 3 ? tcd[ti] : tc[ti];
      fam.push_back(make_job(plans[i], args[i], tile));
      {
        hegrid_status e = encode_rows_map(fam.back(), tile);
        if (e != HEGRID_OK) return e;
      }
      if (args[i].dtype != HEGRID_F16) {
        fam.back().chmax = chmax + at;
        AbsmaxRequest r;
        r.values = args[i].values;
        r.dtype = (int)args[i].dtype;
        r.n_rows = plans[i]->N;
        r.C = args[i].n_channels;
        r.ld = args[i].ld_values;
        r.out = chmax + at;
        amax.push_back(r);
        at += args[i].n_channels;
      }
    }
    // every entry's channel maxima in one launch, ahead of the grid kernels
    if (!chmax_ready) {
      hegrid_status e = launch_chan_absmax((int)amax.size(), amax.data(), s);
      if (e != HEGRID_OK) return e;
    }
    if (!f32.empty()) {
      hegrid_status e = launch_family(f32, false, s);
      if (e != HEGRID_OK) return e;
    }
    for (int t = 0; t < 3; ++t) {
      if (!tc[t].empty()) {
        hegrid_status e = launch_family(tc[t], true, s, tiles[t]);
        if (e != HEGRID_OK) return e;
      }
      if (!tcd[t].empty()) {
        hegrid_status e = launch_family(tcd[t], true, s, tiles[t], true);
        if (e != HEGRID_OK) return e;
      }
    }
    if (!tcm.empty()) {
      hegrid_status e = launch_family(tcm, true, s, -1);
      if (e != HEGRID_OK) return e;
    }
    return HEGRID_OK;
  };
  st = run();
  if (own) cudaFreeAsync(chmax, s);
  return st;
}

// Launches the maximum pass over n requests: the full kernel (256 threads,
// about ctas_per_sm CTAs per SM) or, lean, one k_chan_absmax_lean CTA per SM.
// Both kernels prefer the largest shared-memory carveout: an SM changes its
// L1 / shared-memory split only when it is idle, so a pass resident on every
// SM under a small carveout would keep kernels of other streams that need
// shared memory (plan creation's sort and pair kernels) off the GPU until it
// ends.
hegrid_status launch_absmax(int n, const AbsmaxRequest* req, cudaStream_t s, int ctas_per_sm,
                            bool lean) {
  if (n <= 0) return HEGRID_OK;
  int dev = 0, n_sm = 0;
  HG_CUDA_TRY(cudaGetDevice(&dev));
  static std::atomic<bool> carved[64];  // per device: the attribute is the current device's
  if (dev >= 0 && dev < 64 && !carved[dev].exchange(true)) {
    HG_CUDA_TRY(cudaFuncSetAttribute(k_chan_absmax, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
    HG_CUDA_TRY(cudaFuncSetAttribute(k_chan_absmax_lean,
                                     cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
  }
  const int threads = lean ? kAbsmaxLeanThreads : 256;
  if (lean) ctas_per_sm = 1;
  HG_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  for (int base = 0; base < n; base += kMaxAbsmaxJobs) {
    AbsmaxTable tab;
    std::memset(&tab, 0, sizeof(tab));
    tab.n = std::min(kMaxAbsmaxJobs, n - base);
    int64_t blocks = 0;
    for (int i = 0; i < tab.n; ++i) {
      const AbsmaxRequest& r = req[base + i];
      AbsmaxJob& J = tab.job[i];
      const int vec = (r.dtype == HEGRID_F32 || r.dtype == HEGRID_BF16X2) ? 4 : 8;
      // channel groups of 16 bytes (within ld: ld * element size is a multiple of 16)
      const int64_t nvec = (r.C + vec - 1) / vec;
      J.values = r.values;
      J.out = r.out;
      J.N = r.n_rows;
      J.C = r.C;
      J.ld = r.ld;
      J.dtype = r.dtype;
      J.nvec = (int32_t)nvec;
      J.cols = (int32_t)std::min<int64_t>(nvec, threads);
      const int rpt = threads / J.cols;
      J.gy = (int32_t)((nvec + J.cols - 1) / J.cols);
      // about ctas_per_sm CTAs per SM over all channel groups, each thread >= 32 rows
      int64_t gx = std::max<int64_t>(1, (ctas_per_sm * (int64_t)n_sm + J.gy - 1) / J.gy);
      gx = std::min<int64_t>(gx, std::max<int64_t>(1, r.n_rows / (32 * (int64_t)rpt)));
      J.rows_per_cta = (r.n_rows + gx - 1) / gx;
      J.block_base = blocks;
      blocks += gx * J.gy;
    }
    HG_ARG_CHECK(blocks < ((int64_t)1 << 31), "too many channel-maximum blocks");
    if (lean)
      k_chan_absmax_lean<<<(unsigned)blocks, kAbsmaxLeanThreads, 0, s>>>(tab);
    else
      k_chan_absmax<<<(unsigned)blocks, 256, 0, s>>>(tab);
    count_launch();
    HG_CUDA_TRY(launch_status());
  }
  return HEGRID_OK;
}

}  // namespace

hegrid_status launch_chan_absmax(int n, const AbsmaxRequest* req, cudaStream_t s,
                                 int ctas_per_sm) {
  return launch_absmax(n, req, s, ctas_per_sm, false);
}

}  // namespace hg

struct hegrid_batch {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  uint32_t* chmax;  // the channel maxima of the tensor-core entries (device, owned)
};

extern "C" {

hegrid_status hegrid_grid(hegrid_plan* plan, const void* values, hegrid_dtype dtype,
                          int64_t n_channels, int64_t ld_values, float* map_out, int64_t ld_map,
                          float* weight_out, uint32_t mode, void* stream) {
  hegrid_grid_args a;
  a.values = values;
  a.dtype = dtype;
  a.n_channels = n_channels;
  a.ld_values = ld_values;
  a.map_out = map_out;
  a.ld_map = ld_map;
  a.weight_out = weight_out;
  a.mode = mode;
  hegrid_plan* p[1] = {plan};
  return hg::grid_many(1, p, &a, (cudaStream_t)stream);
}

hegrid_status hegrid_chan_maxima(const void* values, hegrid_dtype dtype, int64_t n_samples,
                                 int64_t n_channels, int64_t ld_values, uint32_t* chmax_out,
                                 uint32_t flags, void* stream) {
  hg::set_error("");
  HG_ARG_CHECK(values != nullptr && chmax_out != nullptr, "values or chmax_out is NULL");
  HG_ARG_CHECK((flags & ~HEGRID_MAXIMA_BESIDE) == 0, "unknown hegrid_chan_maxima flag bits");
  HG_ARG_CHECK(n_samples >= 1, "n_samples must be >= 1");
  HG_ARG_CHECK(n_channels >= 1, "n_channels must be >= 1");
  const int eb = hg::elem_bytes((int)dtype);
  HG_ARG_CHECK(eb > 0, "unknown dtype");
  HG_ARG_CHECK(ld_values >= n_channels, "ld_values < n_channels");
  HG_ARG_CHECK((ld_values * eb) % 16 == 0, "ld_values * element size must be a multiple of 16");
  HG_ARG_CHECK(((uintptr_t)values & 15u) == 0, "values must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  HG_CUDA_TRY(cudaMemsetAsync(chmax_out, 0, sizeof(uint32_t) * (size_t)n_channels, s));
  hg::AbsmaxRequest r;
  r.values = values;
  r.dtype = (int)dtype;
  r.n_rows = n_samples;
  r.C = n_channels;
  r.ld = ld_values;
  r.out = chmax_out;
  return hg::launch_absmax(1, &r, s, 8, (flags & HEGRID_MAXIMA_BESIDE) != 0);
}

hegrid_status hegrid_grid_prescaled(hegrid_plan* plan, const void* values, hegrid_dtype dtype,
                                    int64_t n_channels, int64_t ld_values, const uint32_t* chmax,
                                    float* map_out, int64_t ld_map, float* weight_out,
                                    uint32_t mode, void* stream) {
  hg::set_error("");
  hegrid_grid_args a;
  a.values = values;
  a.dtype = dtype;
  a.n_channels = n_channels;
  a.ld_values = ld_values;
  a.map_out = map_out;
  a.ld_map = ld_map;
  a.weight_out = weight_out;
  a.mode = mode;
  hegrid_plan* p[1] = {plan};
  const bool need = mode != HEGRID_MODE_FP32 && dtype != HEGRID_F16;
  HG_ARG_CHECK(!need || chmax != nullptr, "chmax is NULL");
  return hg::grid_many(1, p, &a, (cudaStream_t)stream, true, const_cast<uint32_t*>(chmax),
                       need);
}

hegrid_status hegrid_grid_masked(hegrid_plan* plan, const void* values, hegrid_dtype dtype,
                                 int64_t n_channels, int64_t ld_values, float* map_out,
                                 int64_t ld_map, float* wc_out, uint32_t mode, void* stream) {
  hg::set_error("");
  hegrid_grid_args a;
  a.values = values;
  a.dtype = dtype;
  a.n_channels = n_channels;
  a.ld_values = ld_values;
  a.map_out = map_out;
  a.ld_map = ld_map;
  a.weight_out = nullptr;
  a.mode = mode;
  hegrid_status st = hg::check_args(plan, a);
  if (st != HEGRID_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = plan->N, M = plan->M, C = n_channels;
  const int eb = hg::elem_bytes((int)dtype);
  const bool mask_f32 = mode == HEGRID_MODE_FP32;  // the FP32 form takes FP32 values only
  const int64_t ldm = mask_f32 ? (C + 3) / 4 * 4 : (C + 7) / 8 * 8;
  int dev = 0, n_sm = 0;
  HG_CUDA_TRY(cudaGetDevice(&dev));
  HG_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  void *clean = nullptr, *mask = nullptr;
  float* q = nullptr;
  auto release = [&]() {
    if (clean) cudaFreeAsync(clean, s);
    if (mask) cudaFreeAsync(mask, s);
    if (q) cudaFreeAsync(q, s);
  };
  auto fail = [&](cudaError_t e, const char* what) {
    hg::set_error(std::string(what) + ": " + cudaGetErrorString(e));
    release();
    return e == cudaErrorMemoryAllocation ? HEGRID_ERR_OOM : HEGRID_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = hg::pool_alloc(&clean, (size_t)N * ld_values * eb, s)) != cudaSuccess)
    return fail(e, "scratch values");
  if ((e = hg::pool_alloc(&mask, (size_t)N * ldm * (mask_f32 ? 4 : 2), s)) != cudaSuccess)
    return fail(e, "scratch mask");
  if ((e = hg::pool_alloc((void**)&q, sizeof(float) * (size_t)M * C, s)) != cudaSuccess)
    return fail(e, "scratch weight fractions");
  const int blocks = std::max(1, n_sm) * 8;
  hg::k_mask_split<<<blocks, 256, 0, s>>>(values, (int)dtype, N, C, ld_values, clean, mask,
                                          mask_f32 ? 1 : 0, ldm);
  hg::count_launch();
  if ((e = hg::launch_status()) != cudaSuccess) return fail(e, "k_mask_split");
  // S_c / W and W_c / W: two passes of the same plan and form
  st = hegrid_grid(plan, clean, dtype, C, ld_values, map_out, ld_map, nullptr, mode, stream);
  if (st == HEGRID_OK)
    st = hegrid_grid(plan, mask, mask_f32 ? HEGRID_F32 : HEGRID_BF16, C, ldm, q, C, nullptr,
                     mode, stream);
  if (st != HEGRID_OK) {
    release();
    return st;
  }
  const float* W = plan->wsum + (mode == HEGRID_MODE_TC ? plan->M : 0);
  hg::k_mask_divide<<<blocks, 256, 0, s>>>(map_out, ld_map, q, M, C, W, wc_out);
  hg::count_launch();
  if ((e = hg::launch_status()) != cudaSuccess) return fail(e, "k_mask_divide");
  release();
  return HEGRID_OK;
}

hegrid_status hegrid_grid_batched(int n, hegrid_plan* const* plans, const hegrid_grid_args* args,
                                  void* stream) {
  return hg::grid_many(n, plans, args, (cudaStream_t)stream);
}

hegrid_status hegrid_batch_create(hegrid_batch** out, int n, hegrid_plan* const* plans,
                                  const hegrid_grid_args* args, void* stream) {
  HG_ARG_CHECK(out != nullptr, "out is NULL");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    hegrid_status st = hg::check_args(plans ? plans[i] : nullptr, args[i]);
    if (st != HEGRID_OK) return st;
  }
  // the plans must be complete before their launches are recorded; plans
  // tuned to a kernel that reads the dense weight tiles get them now (they
  // cannot be built inside the capture)
  for (int i = 0; i < n; ++i) HG_CUDA_TRY(cudaEventSynchronize(plans[i]->ready));
  for (int i = 0; i < n; ++i) {
    if (args[i].mode == HEGRID_MODE_FP32 || plans[i]->wtiles) continue;
    if (plans[i]->tune_tc_kernel != 2 && plans[i]->tune_tc_kernel != 3) continue;
    hegrid_status st = hg::ensure_wtiles(plans[i], (cudaStream_t)stream);
    if (st != HEGRID_OK) return st;
    HG_CUDA_TRY(cudaEventSynchronize(plans[i]->ready));
  }
  cudaStream_t cap;
  HG_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  hegrid_batch* b = new hegrid_batch();
  b->graph = nullptr;
  b->exec = nullptr;
  b->chmax = nullptr;
  const int64_t n_scaled = hg::scaled_channels(n, args);
  cudaError_t e = cudaSuccess;
  if (n_scaled > 0 &&
      (e = cudaMalloc((void**)&b->chmax, sizeof(uint32_t) * (size_t)n_scaled)) != cudaSuccess) {
    hg::set_error(std::string("channel maxima: ") + cudaGetErrorString(e));
    cudaStreamDestroy(cap);
    delete b;
    return e == cudaErrorMemoryAllocation ? HEGRID_ERR_OOM : HEGRID_ERR_CUDA;
  }
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  hegrid_status st = HEGRID_OK;
  if (e == cudaSuccess) {
    st = hg::grid_many(n, plans, args, cap, false, b->chmax);
    cudaError_t e2 = cudaStreamEndCapture(cap, &b->graph);
    if (st == HEGRID_OK && e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess && st == HEGRID_OK) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  cudaStreamDestroy(cap);
  if (st != HEGRID_OK || e != cudaSuccess) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->chmax) cudaFree(b->chmax);
    delete b;
    if (st == HEGRID_OK) {
      hg::set_error(std::string("graph capture failed: ") + cudaGetErrorString(e));
      st = HEGRID_ERR_CUDA;
    }
    return st;
  }
  *out = b;
  return HEGRID_OK;
}

hegrid_status hegrid_batch_launch(hegrid_batch* batch, void* stream) {
  HG_ARG_CHECK(batch != nullptr, "batch is NULL");
  HG_CUDA_TRY(cudaGraphLaunch(batch->exec, (cudaStream_t)stream));
  return HEGRID_OK;
}

hegrid_status hegrid_batch_destroy(hegrid_batch* batch) {
  if (!batch) return HEGRID_OK;
  cudaGraphExecDestroy(batch->exec);
  cudaGraphDestroy(batch->graph);
  if (batch->chmax) cudaFree(batch->chmax);
  delete batch;
  return HEGRID_OK;
}

// Streaming: a ring of (up to) two device chunk buffers and two map buffers.
// Chunk k's H2D copy runs on the copy-in stream, its kernel on the compute
// stream, its D2H copy on the copy-out stream; events order reuse of ring
// slots.  Host rows that are not a multiple of 16 bytes are copied densely
// into a staging slot and spread to the padded pitch by k_pad_rows on the
// compute stream, ahead of the grid kernel.
hegrid_status hegrid_grid_stream(hegrid_plan* plan, const void* const* host_chunks, int n_chunks,
                                 int64_t chunk_channels, hegrid_dtype dtype, uint32_t mode,
                                 float* host_map, int64_t ld_host_map, float* host_weight) {
  HG_ARG_CHECK(plan != nullptr, "plan is NULL");
  HG_ARG_CHECK(n_chunks >= 1 && host_chunks != nullptr, "need at least one chunk");
  HG_ARG_CHECK(chunk_channels >= 1, "chunk_channels must be >= 1");
  HG_ARG_CHECK(host_map != nullptr, "host_map is NULL");
  HG_ARG_CHECK(ld_host_map >= (int64_t)n_chunks * chunk_channels, "ld_host_map too small");
  int eb = 0;
  switch (dtype) {
    case HEGRID_F32: eb = 4; break;
    case HEGRID_BF16: eb = 2; break;
    case HEGRID_F16: eb = 2; break;
    case HEGRID_BF16X2: eb = 4; break;
    default: HG_ARG_CHECK(false, "unknown dtype");
  }
  for (int k = 0; k < n_chunks; ++k) HG_ARG_CHECK(host_chunks[k] != nullptr, "NULL chunk");
  const int64_t N = plan->N, M = plan->M;
  // device rows padded to 16 bytes
  const int64_t ldv = ((chunk_channels * eb + 15) / 16 * 16) / eb;
  const bool padded = ldv != chunk_channels;
  const int n_slots = n_chunks < 2 ? 1 : 2;
  const size_t hbytes = (size_t)N * chunk_channels * eb;  // one host chunk
  const size_t vbytes = (size_t)N * ldv * eb;
  const size_t mbytes = (size_t)M * chunk_channels * sizeof(float);
  int n_sm = 0;
  {
    int dev = 0;
    HG_CUDA_TRY(cudaGetDevice(&dev));
    HG_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  }
  void* dv[2] = {nullptr, nullptr};
  void* dstage[2] = {nullptr, nullptr};
  float* dm[2] = {nullptr, nullptr};
  float* dw = nullptr;
  cudaStream_t sin = nullptr, scomp = nullptr, sout = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_k[2] = {nullptr, nullptr},
              ev_out[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  hegrid_status st = HEGRID_OK;
  auto cleanup = [&]() {
    if (sin) cudaStreamSynchronize(sin);
    if (scomp) cudaStreamSynchronize(scomp);
    if (sout) cudaStreamSynchronize(sout);
    for (int i = 0; i < 2; ++i) {
      if (dv[i]) cudaFreeAsync(dv[i], scomp);
      if (dstage[i]) cudaFreeAsync(dstage[i], scomp);
      if (dm[i]) cudaFreeAsync(dm[i], scomp);
      if (ev_in[i]) cudaEventDestroy(ev_in[i]);
      if (ev_k[i]) cudaEventDestroy(ev_k[i]);
      if (ev_out[i]) cudaEventDestroy(ev_out[i]);
      if (ev_free[i]) cudaEventDestroy(ev_free[i]);
    }
    if (dw) cudaFreeAsync(dw, scomp);
    if (scomp) cudaStreamSynchronize(scomp);
    if (sin) cudaStreamDestroy(sin);
    if (scomp) cudaStreamDestroy(scomp);
    if (sout) cudaStreamDestroy(sout);
  };
#define HG_STREAM_TRY(expr)                                                    \
  do {                                                                         \
    cudaError_t _e = (expr);                                                   \
    if (_e != cudaSuccess) {                                                   \
      hg::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));       \
      st = _e == cudaErrorMemoryAllocation ? HEGRID_ERR_OOM : HEGRID_ERR_CUDA; \
      cleanup();                                                               \
      return st;                                                               \
    }                                                                          \
  } while (0)
  HG_STREAM_TRY(cudaStreamCreateWithFlags(&scomp, cudaStreamNonBlocking));
  for (int i = 0; i < n_slots; ++i) {
    HG_STREAM_TRY(hg::pool_alloc(&dv[i], vbytes, scomp));
    if (padded) HG_STREAM_TRY(hg::pool_alloc(&dstage[i], hbytes, scomp));
    HG_STREAM_TRY(hg::pool_alloc((void**)&dm[i], mbytes, scomp));
    HG_STREAM_TRY(cudaEventCreateWithFlags(&ev_in[i], cudaEventDisableTiming));
    HG_STREAM_TRY(cudaEventCreateWithFlags(&ev_k[i], cudaEventDisableTiming));
    HG_STREAM_TRY(cudaEventCreateWithFlags(&ev_out[i], cudaEventDisableTiming));
    HG_STREAM_TRY(cudaEventCreateWithFlags(&ev_free[i], cudaEventDisableTiming));
  }
  HG_STREAM_TRY(hg::pool_alloc((void**)&dw, sizeof(float) * M, scomp));
  // the buffers are allocated on the compute stream; the copy-in stream starts after that
  cudaEvent_t ev_alloc = nullptr;
  HG_STREAM_TRY(cudaEventCreateWithFlags(&ev_alloc, cudaEventDisableTiming));
  HG_STREAM_TRY(cudaEventRecord(ev_alloc, scomp));
  HG_STREAM_TRY(cudaStreamCreateWithFlags(&sin, cudaStreamNonBlocking));
  HG_STREAM_TRY(cudaStreamWaitEvent(sin, ev_alloc, 0));
  cudaEventDestroy(ev_alloc);
  HG_STREAM_TRY(cudaStreamCreateWithFlags(&sout, cudaStreamNonBlocking));
  for (int k = 0; k < n_chunks; ++k) {
    const int r = k % n_slots;
    // slot r's buffers are free once chunk k-n_slots's kernel finished
    if (k >= n_slots) HG_STREAM_TRY(cudaStreamWaitEvent(sin, ev_k[r], 0));
    HG_STREAM_TRY(cudaMemcpyAsync(padded ? dstage[r] : dv[r], host_chunks[k], hbytes,
                                  cudaMemcpyHostToDevice, sin));
    HG_STREAM_TRY(cudaEventRecord(ev_in[r], sin));
    HG_STREAM_TRY(cudaStreamWaitEvent(scomp, ev_in[r], 0));
    if (padded)
      HG_STREAM_TRY(hg::pad_rows(dstage[r], dv[r], N, chunk_channels * eb, ldv * eb, n_sm, scomp));
    // slot r's map buffer is free once chunk k-n_slots's D2H finished
    if (k >= n_slots) HG_STREAM_TRY(cudaStreamWaitEvent(scomp, ev_out[r], 0));
    st = hegrid_grid(plan, dv[r], dtype, chunk_channels, ldv, dm[r], chunk_channels,
                     k == 0 ? dw : nullptr, mode, scomp);
    if (st != HEGRID_OK) {
      cleanup();
      return st;
    }
    HG_STREAM_TRY(cudaEventRecord(ev_k[r], scomp));
    HG_STREAM_TRY(cudaStreamWaitEvent(sout, ev_k[r], 0));
    if (ld_host_map == chunk_channels)  // the chunk's map rows are contiguous on the host
      HG_STREAM_TRY(cudaMemcpyAsync(host_map + (int64_t)k * chunk_channels, dm[r], mbytes,
                                    cudaMemcpyDeviceToHost, sout));
    else
      HG_STREAM_TRY(cudaMemcpy2DAsync(host_map + (int64_t)k * chunk_channels,
                                      ld_host_map * sizeof(float), dm[r],
                                      chunk_channels * sizeof(float),
                                      chunk_channels * sizeof(float), M, cudaMemcpyDeviceToHost,
                                      sout));
    if (k == 0 && host_weight)
      HG_STREAM_TRY(
          cudaMemcpyAsync(host_weight, dw, sizeof(float) * M, cudaMemcpyDeviceToHost, sout));
    HG_STREAM_TRY(cudaEventRecord(ev_out[r], sout));
  }
  HG_STREAM_TRY(cudaStreamSynchronize(sout));
  HG_STREAM_TRY(cudaStreamSynchronize(scomp));
#undef HG_STREAM_TRY
  cleanup();
  return HEGRID_OK;
}

// ---------------------------------------------------------------------------
// Autotuning
// ---------------------------------------------------------------------------
hegrid_status hegrid_autotune(hegrid_plan* plan, const void* values, hegrid_dtype dtype,
                              int64_t n_channels, int64_t ld_values, uint32_t mode, void* stream,
                              hegrid_tune_report* report) {
  hg::set_error("");
  HG_ARG_CHECK(plan != nullptr, "plan is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const bool tc = mode != HEGRID_MODE_FP32;
  // candidate shapes
  std::vector<hegrid_tune_point> pts;
  auto add = [&](int band, int seg, int group, int kernel) {
    band = band < 0 ? -std::min(-band, plan->nbx_b) : std::min(band, plan->nbx_b);
    for (const auto& q : pts)
      if (q.band == band && q.seg == seg && q.group == group && q.kernel == kernel) return;
    hegrid_tune_point q;
    q.band = band;
    q.seg = seg;
    q.group = group;
    q.kernel = kernel;
    q.ms = -1.0f;
    pts.push_back(q);
  };
  const int bands[] = {2, 4, 8, 16, 1 << 30};
  if (tc) {
    // both work orders (channel tiles slowest / fastest) at segments of 16,
    // and the shorter segment at one band of each
    // both kernels (channel-major only where its 128-channel tiles fill),
    // both orders of the channel tiles (slowest / side by side: all of a
    // block's, or in pairs) at segments of 16, and the shorter segment at one
    // band of each
    const bool cm = n_channels > 64;
    for (int kern = cm ? 2 : 1; kern >= 1; --kern) {
      for (int b : bands) {
        add(b, 16, 0, kern);
        add(-b, 16, 0, kern);
      }
      add(4, 8, 0, kern);
      add(-4, 8, 0, kern);
      add(-2, 16, 2, kern);
      add(-4, 16, 2, kern);
      add(-8, 16, 2, kern);
    }
    // the cell-major kernel with dense A tiles, at the shapes that suit the
    // cell-major kernel
    add(-2, 16, 0, 3);
    add(-4, 16, 2, 3);
    add(-8, 16, 0, 3);
    add(4, 16, 0, 3);
  } else {
    add(0, 1, 0, 0);
    for (int b : bands) add(b, 1, 0, 0);
  }
  // scratch map (discarded)
  float* scratch = nullptr;
  const size_t map_bytes = sizeof(float) * (size_t)plan->M * (size_t)std::max<int64_t>(n_channels, 1);
  HG_CUDA_TRY(hg::pool_alloc((void**)&scratch, map_bytes, s));
  hegrid_grid_args a;
  a.values = values;
  a.dtype = dtype;
  a.n_channels = n_channels;
  a.ld_values = ld_values;
  a.map_out = scratch;
  a.ld_map = n_channels;
  a.weight_out = nullptr;
  a.mode = mode;
  const int32_t keep[5] = {plan->tune_f32_band, plan->tune_tc_band, plan->tune_tc_seg,
                           plan->tune_tc_group, plan->tune_tc_kernel};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hegrid_status st = HEGRID_OK;
  auto fail = [&](hegrid_status code) {
    plan->tune_f32_band = keep[0];
    plan->tune_tc_band = keep[1];
    plan->tune_tc_seg = keep[2];
    plan->tune_tc_group = keep[3];
    plan->tune_tc_kernel = keep[4];
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(scratch, s);
    return code;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    hg::set_error("cudaEventCreate failed");
    return fail(HEGRID_ERR_CUDA);
  }
  hegrid_plan* pl[1] = {plan};
  // Kernels 2 and 3 read the plan's dense weight tiles.  If the plan has not
  // built them yet, they are built here (timed) and that time is added to
  // those shapes' per-call times: the choice then holds for a plan gridded
  // once; a plan that already holds its tiles is tuned on per-call times.
  // The build is timed as a rebuild into the tiles just allocated: the cost a
  // plan pays when the library's pool already holds the memory (the first
  // allocation of a process maps it, a one-time cost).
  float build_ms = 0.0f;
  if (tc && !plan->wtiles) {
    if ((st = hg::ensure_wtiles(plan, s)) != HEGRID_OK) return fail(st);
    if (cudaEventRecord(e0, s) != cudaSuccess) return fail(HEGRID_ERR_CUDA);
    if ((st = hg::launch_build_wtiles(plan->view(), plan->wtiles, s)) != HEGRID_OK)
      return fail(st);
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&build_ms, e0, e1) != cudaSuccess) {
      hg::set_error("timing the weight-tile build failed");
      return fail(HEGRID_ERR_CUDA);
    }
  }
  int best = -1;
  for (size_t i = 0; i < pts.size(); ++i) {
    if (tc) {
      plan->tune_tc_band = pts[i].band;
      plan->tune_tc_seg = pts[i].seg;
      plan->tune_tc_group = pts[i].group;
      plan->tune_tc_kernel = pts[i].kernel;
    } else {
      plan->tune_f32_band = pts[i].band > 0 ? pts[i].band : -1;
    }
    constexpr int kReps = 2;
    if ((st = hg::grid_many(1, pl, &a, s)) != HEGRID_OK) return fail(st);
    if (cudaEventRecord(e0, s) != cudaSuccess) return fail(HEGRID_ERR_CUDA);
    for (int r = 0; r < kReps; ++r)
      if ((st = hg::grid_many(1, pl, &a, s)) != HEGRID_OK) return fail(st);
    float ms = 0.0f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      hg::set_error("timing the autotune candidates failed");
      return fail(HEGRID_ERR_CUDA);
    }
    pts[i].ms = ms / kReps + (pts[i].kernel >= 2 ? build_ms : 0.0f);
    if (best < 0 || pts[i].ms < pts[best].ms) best = (int)i;
  }
  if (tc) {
    plan->tune_tc_band = pts[best].band;
    plan->tune_tc_seg = pts[best].seg;
    plan->tune_tc_group = pts[best].group;
    plan->tune_tc_kernel = pts[best].kernel;
  } else {
    plan->tune_f32_band = pts[best].band > 0 ? pts[best].band : -1;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(scratch, s);
  if (report) {
    report->n = (int32_t)std::min<size_t>(pts.size(), HEGRID_TUNE_MAX);
    report->best = best;
    for (int i = 0; i < report->n; ++i) report->pt[i] = pts[i];
  }
  return HEGRID_OK;
}

hegrid_status hegrid_plan_set_tuning(hegrid_plan* plan, uint32_t mode, int32_t band, int32_t seg,
                                     int32_t group, int32_t kernel) {
  hg::set_error("");
  HG_ARG_CHECK(plan != nullptr, "plan is NULL");
  if (mode == HEGRID_MODE_FP32) {
    HG_ARG_CHECK(band >= -1, "band must be >= -1 for HEGRID_MODE_FP32");
    plan->tune_f32_band = band;
  } else {
    HG_ARG_CHECK(mode == HEGRID_MODE_TC || mode == HEGRID_MODE_TC_SPLIT, "unknown mode");
    HG_ARG_CHECK(band != INT32_MIN, "band out of range");
    HG_ARG_CHECK(seg >= 0 && seg <= 16, "seg must be in [0, 16]");
    HG_ARG_CHECK(group >= 0, "group must be >= 0");
    HG_ARG_CHECK(kernel >= 0 && kernel <= 3, "kernel must be 0, 1, 2 or 3");
    plan->tune_tc_band = band;
    plan->tune_tc_seg = seg;
    plan->tune_tc_group = group;
    plan->tune_tc_kernel = kernel;
  }
  return HEGRID_OK;
}

hegrid_status hegrid_autotune_bins(int64_t n_samples, const double* lon_deg, const double* lat_deg,
                                   int coords_on_device, const hegrid_map_geom* geom,
                                   const hegrid_kernel* kern, void* stream,
                                   int32_t* best_bin_cells, float* ms) {
  hg::set_error("");
  HG_ARG_CHECK(best_bin_cells != nullptr, "best_bin_cells is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  HG_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    hg::set_error("cudaEventCreate failed");
    return HEGRID_ERR_CUDA;
  }
  float best_ms = 0.0f;
  int best = 0;
  hegrid_status st = HEGRID_OK;
  for (int B = 1; B <= 4 && st == HEGRID_OK; ++B) {
    float tmin = -1.0f;
    for (int rep = 0; rep < 3 && st == HEGRID_OK; ++rep) {  // first: warm-up
      hegrid_plan* p = nullptr;
      cudaEventRecord(e0, s);
      st = hegrid_plan_create(&p, n_samples, lon_deg, lat_deg, coords_on_device, geom, kern,
                              (uint32_t)B, stream);
      cudaEventRecord(e1, s);
      if (st != HEGRID_OK) break;
      float t = 0.0f;
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&t, e0, e1);
      hegrid_plan_destroy(p);
      if (rep > 0 && (tmin < 0.0f || t < tmin)) tmin = t;
    }
    if (st != HEGRID_OK) break;
    if (ms) ms[B - 1] = tmin;
    if (best == 0 || tmin < best_ms) {
      best = B;
      best_ms = tmin;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != HEGRID_OK) return st;
  *best_bin_cells = best;
  return HEGRID_OK;
}

}  // extern "C"
