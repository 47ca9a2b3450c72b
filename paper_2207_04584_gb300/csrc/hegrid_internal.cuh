// Internal definitions shared by the translation units of libhegrid.so.
#pragma once

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

// W per cell is kept for each weight representation: 0 FP32, 1 BF16 hi,
// 2 BF16 hi+lo, 3 FP16 hi, 4 FP16 hi+lo (wsum[v * M + m]).
constexpr int kWsumVariants = 5;

// Thread-local error message for hegrid_last_error().
void set_error(const std::string& msg);

// Process-wide count of kernel launches made by the library.
void count_launch(int n = 1);

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
  const int64_t* cand_off;  // [n_blocks+1] candidate slots per block (padded to 64)
  const int32_t* cand_idx;  // [n_cand] original sample index per slot
  const int64_t* sub_off;   // [n_cand/32+1] first entry of each 32-candidate sub-chunk
  const uint16_t* ent_ck;   // [P] entry: (block-local cell << 6) | (candidate & 63)
  const float* ent_w;       // [P] FP32 weight of the entry
  int32_t* err_word;        // device error word (bounded waits)
};

}  // namespace hg

struct hegrid_plan {
  hegrid_map_geom geom;
  hegrid_kernel kern;
  int device;
  int64_t N, M, P, n_bins, n_blocks, n_cand;
  int32_t bin_cells, padx, pady, nbx, nby, nbx_b, nby_b;
  double sigma_rad, R_rad, R_deg;
  // device arrays (owned)
  int32_t* perm;
  int32_t* bin_off;
  int64_t* cand_off;
  int64_t* blk_pair_off;
  int32_t* cand_idx;
  int64_t* sub_off;
  uint16_t* ent_ck;
  float* ent_w;
  float* wsum;
  int32_t* err_word;
  int64_t bytes;
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
    v.cand_idx = cand_idx;
    v.sub_off = sub_off;
    v.ent_ck = ent_ck;
    v.ent_w = ent_w;
    v.err_word = err_word;
    return v;
  }
};

// Grid launchers (one per kernel family).  Work items are (field, cell block,
// channel tile); persistent CTAs take items blockIdx.x, blockIdx.x + gridDim.x,
// ... so no device queue state is shared between launches.
namespace hg {

struct GridJob {
  PlanView pv;
  const void* values;
  int32_t dtype;
  int32_t mode;
  int64_t C, ld_values;
  float* map;
  int64_t ld_map;
  float* weight_out;
  int64_t n_ctiles;   // channel tiles
  int64_t item_base;  // first work item of this job in the queue
};

// Up to kMaxJobs fields per launch, passed by value as a kernel parameter.
constexpr int kMaxJobs = 64;
struct JobTable {
  int32_t n_jobs;
  int64_t n_items;
  GridJob job[kMaxJobs];
};

hegrid_status launch_grid_f32(const JobTable& jt, cudaStream_t s);
hegrid_status launch_grid_tc(const JobTable& jt, cudaStream_t s);
int f32_channel_tile();
int tc_channel_tile();

}  // namespace hg
