// Internal definitions shared by the translation units of libhegrid.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "hegrid.h"

// Cell blocks: 16 cells along RA x 8 cells along Dec = 128 cells, the M
// dimension of the tensor-core tiles and the CTA of the plan kernels.
#define HG_BX 16
#define HG_BY 8
#define HG_BLOCK_CELLS 128
// Candidate lists of a block are padded to a multiple of this many samples
// (the K chunk of the grid kernels).
#define HG_KPAD 64

namespace hg {

// W per cell is kept for each weight representation the grid kernels
// multiply by: 0 the FP32 weights (FP32 form, tensor-core split form), 1 the
// weights rounded to FP16 (tensor-core single form) (wsum[v * M + m]).
constexpr int kWsumVariants = 2;

// The tensor-core forms multiply weights scaled by this power of two (exact),
// so that the low FP16 half of a weight split stays a normal number down to
// weights of about 2^-17; W is scaled to match.
constexpr float kTcWeightScale = 32768.0f;

// Weight entries address a K-major, 64-byte-swizzled 128 x 32 tile of 16-bit
// values (one block's cells x one 32-candidate sub-chunk): byte offset of
// (cell r, candidate k), and back.  The tensor-core kernel stores weights at
// this offset directly; the FP32 kernel decodes (r, k).
__host__ __device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)(r * 64 + ((((k >> 3) ^ ((r >> 1) & 3)) << 4) | ((k & 7) << 1)));
}
__host__ __device__ __forceinline__ void tile_rk(uint32_t off, int& r, int& k) {
  r = (int)(off >> 6);
  k = (int)(((((off >> 4) & 3u) ^ ((uint32_t)(r >> 1) & 3u)) << 3) | ((off >> 1) & 7u));
}

// Thread-local error message for hegrid_last_error().
void set_error(const std::string& msg);

// Process-wide count of kernel launches made by the library.
void count_launch(int n = 1);
// The launch error to report after a launch: cudaGetLastError(), or an
// injected launch failure (HEGRID_FAULT=launch:N).
cudaError_t launch_status();
// Fault injection (HEGRID_FAULT): true exactly once, at the N-th event of
// `kind` since the variable was last changed.
enum { kFaultNone = 0, kFaultAlloc = 1, kFaultLaunch = 2, kFaultWait = 3 };
bool fault_hit(int kind);

// Stream-ordered allocation from the library's per-device pool (freed blocks
// are kept for reuse); release with cudaFreeAsync.
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st);

#define HG_CUDA_TRY(expr)                                                           \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) {                                                        \
      ::hg::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));          \
      return _e == cudaErrorMemoryAllocation ? HEGRID_ERR_OOM : HEGRID_ERR_CUDA;    \
    }                                                                               \
  } while (0)

#define HG_ARG_CHECK(cond, msg)                                                     \
  do {                                                                              \
    if (!(cond)) {                                                                  \
      ::hg::set_error(std::string("invalid argument: ") + (msg));                   \
      return HEGRID_ERR_INVALID_ARG;                                                \
    }                                                                               \
  } while (0)

// What the grid kernels need from a plan, by value (kernel parameter / device
// work-queue entry).
struct PlanView {
  int32_t nx, ny;           // map
  int32_t nbx_b, nby_b;     // cell blocks along RA / Dec
  int64_t M;                // cells
  int64_t n_blocks;
  const float* wsum;        // [kWsumVariants * M] W per cell and weight representation
  const int64_t* cand_off;  // [n_blocks+1] first candidate slot of each block (multiple of 64)
  const int32_t* cand_cnt;  // [n_blocks] candidates of each block, padded to a multiple of 64
  const int32_t* cand_idx;  // [n_cand] original sample index per slot
  const int64_t* sub_off;   // [slots/32+1] first entry of each 32-candidate sub-chunk
                            // (a block's last sub-chunk is followed by its end sentinel)
  const uint16_t* ent_ck;   // [P] entry: tile_off(block-local cell, candidate & 31)
  const float* ent_w;       // [P] FP32 weight of the entry
  // [slots/32] dense weight tiles of the channel-major tensor-core kernel
  // (16 KB per sub-chunk: FP16 hi then lo halves of the weights x 2^15, 128
  // cells x 32 candidates, K-major, 64-byte swizzle); NULL until built
  const uint8_t* wtiles;
  int32_t* err_word;        // device error word (bounded waits)
};

}  // namespace hg

struct hegrid_plan {
  hegrid_map_geom geom;
  hegrid_kernel kern;
  int device;
  int64_t N, M, n_bins, n_blocks;
  int64_t P_ub, slots;  // entries and candidate slots reserved (upper bounds)
  int64_t P, n_cand;    // pairs and used candidate slots (-1 until read back)
  int32_t bin_cells, padx, pady, nbx, nby, nbx_b, nby_b;
  double sigma_rad, R_rad, R_deg;
  // device arrays (owned)
  int32_t* perm;
  int32_t* bin_off;
  int64_t* cand_off;
  int64_t* blk_pair_off;
  int32_t* cand_cnt;
  unsigned long long* totals;  // device: pairs, used candidate slots
  int32_t* cand_idx;
  int64_t* sub_off;
  uint16_t* ent_ck;
  float* ent_w;
  float* wsum;
  int32_t* err_word;
  int64_t bytes;
  // Launch shapes chosen by hegrid_autotune (0: defaults): FP32 band, tensor
  // core band, segment length and channel-tile group.
  int32_t tune_f32_band, tune_tc_band, tune_tc_seg, tune_tc_group;
  // Tensor-core kernel: 0 (default) and 1: cell-major; 2: channel-major;
  // 3: cell-major with its A tiles from the dense weight tiles (2 and 3 where
  // the tiles exist or can be built).
  int32_t tune_tc_kernel;
  // Dense weight tiles of the channel-major kernel (owned; built by the first
  // grid call that runs it, on that call's stream, which then re-records
  // `ready`).
  uint8_t* wtiles;
  // Recorded on the creation stream after the last plan kernel.  The plan's
  // memory comes from a stream-ordered pool, so every other stream must wait
  // on this event before touching it.
  cudaEvent_t ready;
  hg::PlanView view() const {
    hg::PlanView v;
    v.nx = geom.nx;
    v.ny = geom.ny;
    v.nbx_b = nbx_b;
    v.nby_b = nby_b;
    v.M = M;
    v.n_blocks = n_blocks;
    v.wsum = wsum;
    v.cand_off = cand_off;
    v.cand_cnt = cand_cnt;
    v.cand_idx = cand_idx;
    v.sub_off = sub_off;
    v.ent_ck = ent_ck;
    v.ent_w = ent_w;
    v.wtiles = wtiles;
    v.err_word = err_word;
    return v;
  }
};

// Grid launchers (one per kernel family).  Work items are (field, cell block,
// channel tile); persistent CTAs take items blockIdx.x, blockIdx.x + gridDim.x,
// ... so no device queue state is shared between launches.
namespace hg {

struct GridJob {
  // Tensor map of the values (rows = samples, boxes of one channel tile, one
  // row high) for the grid kernels' row gathers.
  CUtensorMap rows;
  PlanView pv;
  const void* values;
  int32_t dtype;
  int32_t mode;
  int64_t C, ld_values;
  float* map;
  int64_t ld_map;
  float* weight_out;
  // Tensor-core modes: the largest |v| of each channel (float bits, [C]),
  // which sets the channel's power-of-two scale; NULL: unscaled.
  const uint32_t* chmax;
  int64_t n_rows;     // samples (rows of the values)
  // Launch shape (see hegrid_autotune): blocks per band of the work order
  // (0: channel tiles fastest, FP32 kernel only) and chunks per accumulation
  // segment (tensor-core kernel).
  int32_t band, seg;
  // Tensor-core kernel: channel tiles run side by side in groups of `group`
  // (band < 0; 0: all of a block's tiles), and the sweep over a block's
  // candidates starts at the fraction frac(-row * rot) of it (0: no rotation).
  int32_t group;
  float rot;
  int64_t n_ctiles;   // channel tiles
  int64_t item_base;  // first work item of this job in the queue
};

// Up to kMaxJobs fields per launch, passed by value as a kernel parameter.
constexpr int kMaxJobs = 64;
struct JobTable {
  int32_t n_jobs;
  int32_t inject;    // tensor-core kernel: 1 = withhold one producer arrive (tests)
  int64_t n_items;
  uint64_t wait_ns;  // limit of the kernels' bounded waits
  GridJob job[kMaxJobs];
};

hegrid_status launch_grid_f32(const JobTable& jt, cudaStream_t s);
// For each request: out[c] (zeroed by the caller) = max(out[c], largest |v|
// of channel c) as float bits, for the C channels of `values` (NaN ignored,
// Inf kept); all requests in one launch (kMaxJobs per launch).
struct AbsmaxRequest {
  const void* values;
  int dtype;
  int64_t n_rows, C, ld;
  uint32_t* out;
};
hegrid_status launch_chan_absmax(int n, const AbsmaxRequest* req, cudaStream_t s,
                                 int ctas_per_sm = 8);
// `tile`: the channel tile of every job in the table (tc_channel_tile(C));
// dense_a: the A tiles come from the plans' dense weight tiles (every job's
// plan must have them).
hegrid_status launch_grid_tc(const JobTable& jt, cudaStream_t s, int tile, bool dense_a);
int f32_channel_tile();
// Tensor-core channel tile for C channels: the narrowest of 64, 128, 256
// that holds C, else 256.
int tc_channel_tile(int64_t C);
int tc_default_band();
int tc_default_seg();
int tc_default_group();
// Channel-major tensor-core kernel (grid_tcm.cu): its channel tile (128), the
// bytes of a plan's dense weight tiles for `slots` candidate slots, their
// build, and the grid launch (every job's plan must have its tiles).
int tcm_channel_tile();
int64_t tcm_wtile_bytes(int64_t slots);
hegrid_status launch_build_wtiles(const PlanView& pv, uint8_t* wtiles, cudaStream_t s,
                                 int64_t blk0 = 0, int64_t n_blk = -1);
hegrid_status launch_grid_tcm(const JobTable& jt, cudaStream_t s);

}  // namespace hg
