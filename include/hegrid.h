/*
 * hegrid.h -- C ABI of libhegrid.so: GB300-native convolution gridding of
 * non-uniform, multi-channel single-dish samples onto a regular map.
 *
 * The operation is Eq. 1 of HEGrid (Sec. 2.2): for every target cell g,
 *     map[g, c] = sum_n w(g; s_n) v[s_n, c] / W[g],   W[g] = sum_n w(g; s_n),
 * with a Gaussian kernel w = exp(-d^2 / (2 sigma^2)) of the great-circle
 * separation d, truncated at d <= R (Algorithm 1, Sec. 4.1.2, inclusive),
 * sigma = FWHM / sqrt(8 ln 2), R = support_sigmas * sigma.  The weights are
 * computed once per (sample, cell) pair by hegrid_plan_create and shared by
 * every channel (the "shared component" of Sec. 4.3.1).
 *
 * Conventions for every call:
 *   - Pointers marked "device" are CUDA device (or managed) addresses on the
 *     current device; "host" pointers are CPU memory (pinned where stated).
 *   - The caller owns every input and output buffer.  A plan owns all of its
 *     internal device memory and frees it in hegrid_plan_destroy.
 *   - Calls return a status and never throw.  Argument errors are returned
 *     before any launch.  hegrid_last_error() returns a thread-local message
 *     describing the last failure.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Layouts are row-major: values[n * ld_values + c], map[m * ld_map + c]
 *     with cell index m = iy * nx + ix (ix along RA, iy along Dec).
 */
#ifndef HEGRID_H
#define HEGRID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hegrid_plan hegrid_plan;   /* opaque; owns its device memory */
typedef struct hegrid_batch hegrid_batch; /* opaque; a captured batched launch */

typedef enum {
  HEGRID_OK = 0,
  HEGRID_ERR_INVALID_ARG = -1,
  HEGRID_ERR_OOM = -2,
  HEGRID_ERR_CUDA = -3,
  HEGRID_ERR_TIMEOUT = -4, /* a bounded device-side wait gave up */
  HEGRID_ERR_UNSUPPORTED = -5
} hegrid_status;

/* Storage type of the sample values. */
typedef enum {
  HEGRID_F32 = 0,
  HEGRID_BF16 = 1,
  HEGRID_F16 = 2,
  HEGRID_BF16X2 = 3 /* two bf16 per value, hi then lo: v = hi + lo */
} hegrid_dtype;

/* Target map: the regular nx x ny grid of Sec. 2.2.  Cell (ix, iy) has its
 * centre at lon0 + (ix - (nx-1)/2) dlon, lat0 + (iy - (ny-1)/2) dlat (degrees);
 * no projection. */
typedef struct {
  int32_t nx, ny;
  double lon0_deg, lat0_deg;
  double dlon_deg, dlat_deg;
} hegrid_map_geom;

/* Gaussian kernel by its FWHM; support_sigmas is R / sigma (e.g. 3.0). */
typedef struct {
  double fwhm_deg;
  double support_sigmas;
} hegrid_kernel;

/* hegrid_grid modes */
#define HEGRID_MODE_FP32 0u     /* CUDA-core FP32 gather/accumulate */
#define HEGRID_MODE_TC 1u       /* tcgen05 tensor cores, one FP16 pass */
#define HEGRID_MODE_TC_SPLIT 2u /* tcgen05 with FP16 hi/lo splits of values and weights */

/* plan_create flags: bits 0-7 give the bin edge in map cells (0 = default 2).
 * Bits 8-12, HEGRID_PLAN_HEALPIX(k) with 1 <= k <= 13, select the paper's own
 * pixelisation instead (Sec. 4.1.1): samples are keyed by their HEALPix
 * RING-scheme pixel at nside = 2^k (Gorski et al. 2005) and found through a
 * table of rings x pixel ranges over the padded map; the bin edge is then
 * unused.  The pairs, weights and maps are the same as with map bins (only the
 * candidate search differs); bin_off of hegrid_plan_export then indexes the
 * table's pixels, ring by ring from the north. */
#define HEGRID_PLAN_BIN_CELLS(b) ((uint32_t)(b) & 0xffu)
#define HEGRID_PLAN_HEALPIX(k) (((uint32_t)(k) & 0x1fu) << 8)
/* Bit 13: the map is a Sanson-Flamsteed (sinusoidal, about lon0) grid instead
 * of the plain lon/lat grid: cell (ix, iy) has lat = lat0 + (iy - (ny-1)/2)
 * dlat and lon = lon0 + x / cos(lat), x = (ix - (nx-1)/2) dlon, so dlon is a
 * length along the parallel and cells are equal in area.  Map bins only (not
 * with HEGRID_PLAN_HEALPIX). */
#define HEGRID_PLAN_SFL (1u << 13)
/* Bit 14: plan creation also writes the plan's dense weight tiles (16 KB per
 * 32-candidate sub-chunk: the FP16 high and low halves of the weights x 2^15,
 * 128 cells x 32 candidates), which tensor-core kernels 2 and 3 of
 * hegrid_plan_set_tuning read; without it those kernels build the tiles on
 * their first call.  Plan creation then runs its pair kernel in two halves on
 * two streams (the second created and released by the call) and builds each
 * half's tiles after its pairs, so that the memory-bound build overlaps the
 * other half's pair kernel.  The tiles are the same bytes either way; they
 * take 16 KB per 32 candidate slots (counted in hegrid_plan_info's bytes). */
#define HEGRID_PLAN_DENSE_TILES (1u << 14)

/*
 * hegrid_plan_create -- bin the samples and build the shared weights.
 * (Sec. 4.1.1 pre-processing and Algorithm 1's contribution search, on the GPU.)
 *
 * n_samples        number of samples N (>= 1, < 2^31).
 * lon_deg, lat_deg N coordinates in degrees (FP64); host memory if
 *                  coords_on_device == 0, device memory otherwise.  Not kept.
 * geom, kern       map geometry and kernel (host structs, copied).
 * flags            HEGRID_PLAN_BIN_CELLS(b) or HEGRID_PLAN_HEALPIX(k), optionally
 *                  | HEGRID_PLAN_SFL (not with HEALPix) | HEGRID_PLAN_DENSE_TILES,
 *                  or 0; other bits, k > 13, or HEALPix with SFL: INVALID_ARG.
 * stream           stream for every launch; the call synchronises it once to
 *                  learn the sizes of the pair ranges it reserves (upper
 *                  bounds from the binned samples); the rest is asynchronous.
 *
 * Errors: INVALID_ARG (N < 1, nx/ny < 1, cell size <= 0, FWHM <= 0, support
 * <= 0); UNSUPPORTED (a cell row within R of a pole, a padded map wider than
 * 360 deg, R > 11 deg, more than 2^31 candidate slots over all cell blocks); OOM; CUDA.
 * On error *out is set to NULL.
 */
hegrid_status hegrid_plan_create(hegrid_plan **out, int64_t n_samples, const double *lon_deg,
                                 const double *lat_deg, int coords_on_device,
                                 const hegrid_map_geom *geom, const hegrid_kernel *kern,
                                 uint32_t flags, void *stream);

/*
 * hegrid_grid -- Eq. 1 for every cell and channel (the cell-update step of
 * Algorithm 1, normalisation included).  Fully asynchronous on `stream`.
 *
 * values      device [n_samples x ld_values] of `dtype`, in the caller's own
 *             sample order (the plan keeps the permutation); 16-byte aligned,
 *             ld_values * element size a multiple of 16 bytes, ld_values >= C.
 *             For HEGRID_BF16X2, ld_values counts values (pairs).
 * n_channels  C >= 1.
 * map_out     device FP32 [M x ld_map], ld_map >= C, M = nx * ny.  Cells with
 *             W = 0 get NaN.
 * weight_out  device FP32 [M] or NULL: W[m] as used for the normalisation.
 * mode        HEGRID_MODE_FP32 (dtype F32 only), HEGRID_MODE_TC or
 *             HEGRID_MODE_TC_SPLIT (any dtype).  The tensor-core modes work in
 *             channel tiles of 64, 128 or 256 channels (the narrowest that
 *             holds C, 256 above it); the FP32 mode in tiles of 128.
 *             In the tensor-core modes each channel is multiplied by an exact
 *             power of two that puts its largest |v| in [2^14, 2^15) before the
 *             FP16 conversion (and divided out in the normalisation), so a
 *             channel keeps its accuracy relative to its own values whatever
 *             the other channels of its tile hold; for F32, BF16X2 and BF16
 *             values this takes one extra read of the values (a per-channel
 *             maximum) and C * 4 bytes of stream-ordered scratch from the
 *             library's pool.  FP16 values are used as stored.
 * Non-finite values are outside this call's contract (see hegrid_grid_masked).
 *
 * Errors: INVALID_ARG (NULL plan/values/map, bad C/ld/alignment/dtype/mode);
 * UNSUPPORTED (mode not available for dtype); CUDA (launch failure).
 */
hegrid_status hegrid_grid(hegrid_plan *plan, const void *values, hegrid_dtype dtype,
                          int64_t n_channels, int64_t ld_values, float *map_out, int64_t ld_map,
                          float *weight_out, uint32_t mode, void *stream);

/*
 * hegrid_chan_maxima -- the largest |v| of each channel of `values` (as FP32
 * bits; NaN ignored), the statistic that sets each channel's power-of-two
 * scale in the tensor-core modes (see hegrid_grid; the scale is part of the
 * FP16 conversion that Eq. 1's products go through on the tensor cores, the
 * paper has no counterpart).  It depends on the values only, not on a plan,
 * so a caller can run it on another stream while the plan is being created
 * and pass the result to hegrid_grid_prescaled.  Asynchronous on `stream`.
 *
 * values     device [n_samples x ld_values] of `dtype`, as for hegrid_grid.
 * chmax_out  device uint32 [n_channels], written (caller-owned).
 * flags      0: the pass takes the whole GPU (every SM's threads; HBM-bound).
 *            HEGRID_MAXIMA_BESIDE: one 128-thread CTA per SM without shared
 *            memory, so that kernels on other streams (plan creation) keep
 *            their SM slots while it runs; alone it takes about three times
 *            as long.  Other bits: INVALID_ARG.
 *
 * Errors: INVALID_ARG (NULL pointers, n_samples < 1, n_channels < 1, bad
 * ld/alignment/dtype/flags); CUDA (launch failure).
 */
#define HEGRID_MAXIMA_BESIDE (1u << 0)
hegrid_status hegrid_chan_maxima(const void *values, hegrid_dtype dtype, int64_t n_samples,
                                 int64_t n_channels, int64_t ld_values, uint32_t *chmax_out,
                                 uint32_t flags, void *stream);

/*
 * hegrid_grid_prescaled -- hegrid_grid with the channel maxima already
 * computed by hegrid_chan_maxima on the same values (device [n_channels],
 * complete in stream order before this call's work, e.g. through an event):
 * the tensor-core modes skip their own pass over the values and the scratch
 * for the maxima.  Maxima of other values give wrong maps (values above a
 * channel's stated maximum overflow its FP16 scale).  chmax may be NULL for
 * HEGRID_MODE_FP32 and for HEGRID_F16 values, which are not scaled.  The map
 * is identical to hegrid_grid's on the same inputs.
 *
 * Errors: as for hegrid_grid; INVALID_ARG also for chmax NULL where it is
 * needed.
 */
hegrid_status hegrid_grid_prescaled(hegrid_plan *plan, const void *values, hegrid_dtype dtype,
                                    int64_t n_channels, int64_t ld_values, const uint32_t *chmax,
                                    float *map_out, int64_t ld_map, float *weight_out,
                                    uint32_t mode, void *stream);

/* Free the plan and all of its device memory (synchronises the device).
 * NULL is a no-op.  Returns OK.  (Library service; no step of the paper.) */
hegrid_status hegrid_plan_destroy(hegrid_plan *plan);

/* One entry of a batched launch (the arguments of hegrid_grid). */
typedef struct {
  const void *values;
  hegrid_dtype dtype;
  int64_t n_channels, ld_values;
  float *map_out;
  int64_t ld_map;
  float *weight_out;
  uint32_t mode;
} hegrid_grid_args;

/*
 * hegrid_grid_batched -- grid n independent fields in one persistent launch
 * per kernel kind (the multi-pipeline FIFO of Sec. 4.2, as one device work
 * queue).  plans[i] and args[i] describe field i (host arrays, read during
 * the call; the device buffers they name stay the caller's).  Asynchronous.
 * Errors: INVALID_ARG (n < 0; plans or args NULL with n > 0; any entry that
 * hegrid_grid would reject -- every entry is checked before the first
 * launch); UNSUPPORTED and CUDA as for hegrid_grid.  n = 0 does nothing.
 */
hegrid_status hegrid_grid_batched(int n, hegrid_plan *const *plans, const hegrid_grid_args *args,
                                  void *stream);

/*
 * hegrid_batch_create / _launch / _destroy -- the same batch (Sec. 4.2's
 * pipelines) with its work queue uploaded once and its launches captured in a
 * CUDA graph; launch
 * replays the graph on `stream`.  The plans and buffers named in args must
 * outlive the batch.  create waits (on the host) for the plans to be built,
 * first builds, on `stream`, the dense weight tiles of plans tuned to a kernel
 * that reads them (hegrid_plan_set_tuning kernel 2 or 3), and sets *out (NULL
 * on error).
 * Errors: create: INVALID_ARG (out NULL, and as for hegrid_grid_batched),
 * OOM (the dense tiles), CUDA (capture or instantiation failed); launch: INVALID_ARG (batch NULL),
 * CUDA; destroy: NULL is a no-op, returns OK.
 */
hegrid_status hegrid_batch_create(hegrid_batch **out, int n, hegrid_plan *const *plans,
                                  const hegrid_grid_args *args, void *stream);
hegrid_status hegrid_batch_launch(hegrid_batch *batch, void *stream);
hegrid_status hegrid_batch_destroy(hegrid_batch *batch);

/*
 * hegrid_grid_stream -- grid n_chunks channel chunks that live in host memory
 * (Sec. 4.3.2: pinned host buffers, asynchronous copies overlapped with the
 * kernel).  Chunk k holds channels [k*chunk_channels, (k+1)*chunk_channels) as
 * host [n_samples x chunk_channels] of `dtype` (pinned memory recommended).
 * host_map is host FP32 [M x ld_host_map] with ld_host_map >= n_chunks *
 * chunk_channels; host_weight is host FP32 [M] or NULL.  Uses internal
 * streams and a device ring of two chunk buffers (one for a single chunk);
 * blocks until done.  Each chunk crosses the host link as one dense copy;
 * rows that are not a multiple of 16 bytes are then spread on the device to
 * the 16-byte row pitch the grid kernels read, through a staging buffer of
 * one chunk per ring slot.
 * Errors: INVALID_ARG (NULL plan, host_map or chunk pointer; n_chunks < 1;
 * chunk_channels < 1; ld_host_map < n_chunks * chunk_channels; unknown dtype;
 * and the checks of hegrid_grid); OOM (the device ring); CUDA.
 */
hegrid_status hegrid_grid_stream(hegrid_plan *plan, const void *const *host_chunks, int n_chunks,
                                 int64_t chunk_channels, hegrid_dtype dtype, uint32_t mode,
                                 float *host_map, int64_t ld_host_map, float *host_weight);

/*
 * hegrid_grid_masked -- Eq. 1 with per-channel masking: in channel c a sample
 * whose value is not finite (NaN, +-Inf) contributes to neither sum, so the
 * channel has its own weight sum W_c[m] = sum of w(m; s_n) over the samples
 * with a finite value there, and map[m, c] = sum_n w v / W_c[m] (NaN where
 * W_c[m] = 0).  The paper leaves invalid data implicit; this is the reading
 * that keeps the shared weights: two grid passes of the same plan and form,
 * one over the values with non-finite entries replaced by 0 and one over
 * their 0/1 finiteness mask, each normalised by the plan's W, so that their
 * ratio is S_c / W_c.  Arguments as for hegrid_grid; wc_out is device FP32
 * [M x ld_map] receiving W_c, or NULL.  Scratch from the library's pool
 * (freed before return, stream-ordered): the cleaned values (the input's
 * size), the mask (N x C FP32 for HEGRID_MODE_FP32, BF16 otherwise) and an
 * M x C FP32 map.  Asynchronous on `stream`.  Errors as for hegrid_grid.
 */
hegrid_status hegrid_grid_masked(hegrid_plan *plan, const void *values, hegrid_dtype dtype,
                                 int64_t n_channels, int64_t ld_values, float *map_out,
                                 int64_t ld_map, float *wc_out, uint32_t mode, void *stream);

/* Plan sizes of the neighbour search of Algorithm 1 (any output may be
 * NULL): pairs P, bins, cell blocks, candidate
 * slots in use (padded to 64 per block), device bytes held.  Waits until the
 * plan has been built.  Errors: INVALID_ARG (plan NULL); CUDA. */
hegrid_status hegrid_plan_info(const hegrid_plan *plan, int64_t *n_pairs, int64_t *n_bins,
                               int64_t *n_blocks, int64_t *n_cand, int64_t *bytes);

/*
 * hegrid_plan_export -- copy plan structures to host buffers (any may be NULL):
 * the binning (Sec. 4.1.1's index, here map bins or HEALPix rings), the
 * neighbour lists of Algorithm 1 and the kernel weights of Eq. 1:
 *   perm[N]          sample indices sorted by (bin key, index); discarded last
 *   bin_off[n_bins+1] start of each bin in perm (bin_off[n_bins] = kept count)
 *   nb_off[M+1]      CSR row offsets of the (cell -> sample) pairs
 *   nb_idx[P]        sample index of each pair, ascending per cell (canonical)
 *   nb_w[P]          FP32 weight of each pair, in the same order as nb_idx
 *   weight[M]        W[m] = sum of the FP32 weights of cell m
 * Synchronises the plan's device work.  Errors: INVALID_ARG (plan NULL); CUDA
 * (a failed copy, or an entry count that disagrees with the pair total).
 */
hegrid_status hegrid_plan_export(const hegrid_plan *plan, int32_t *perm, int32_t *bin_off,
                                 int64_t *nb_off, int32_t *nb_idx, float *nb_w, float *weight);

/*
 * Autotuning of launch shapes on the caller's own data (the paper tunes its
 * block size and stream count by sweeps, Sec. 5.3; here the library times the
 * candidates and keeps the fastest).
 *
 * hegrid_autotune -- time the grid step of `plan` for `mode` over a fixed set
 * of launch shapes and store the fastest in the plan; later hegrid_grid,
 * hegrid_grid_batched, hegrid_batch_create and hegrid_grid_stream calls on
 * this plan use it.  Shapes: the work order's band width in cell-block
 * columns (which blocks run concurrently and so share sample rows in L2),
 * for the tensor-core modes also the kernel (cell-major, cell-major with
 * dense A tiles, and channel-major when n_channels > 64; the two that read
 * the plan's dense weight tiles are charged the tiles' build, timed here as a
 * rebuild into memory the pool already holds, unless the plan held its tiles
 * before the call), the order of channel tiles (negative band:
 * the tiles of a block side by side) and the accumulation segment length (8 or 16
 * sub-chunks of 32 candidates; both keep the split form well inside its error
 * bound: the tensor core's FP32 accumulate loses about 2^-22 of the running
 * sum per MMA, so the error grows with the segment).  values,
 * dtype, n_channels, ld_values as for hegrid_grid; the maps computed while
 * timing go to a scratch buffer (stream-ordered pool) and are discarded.
 * Synchronises `stream`.  report (may be NULL) receives every shape timed
 * (milliseconds per grid call, mean of 2 after 1 warm-up) and the index of
 * the one kept.  Errors: INVALID_ARG (plan NULL, and the checks of
 * hegrid_grid); UNSUPPORTED, OOM (the scratch map) and CUDA as for hegrid_grid.
 */
#define HEGRID_TUNE_MAX 40
typedef struct {
  int32_t band;   /* blocks per band (0: the channel tiles of a block back to back) */
  int32_t seg;    /* 32-candidate sub-chunks per accumulation segment (tensor-core modes) */
  int32_t group;  /* channel tiles side by side when band < 0 (tensor-core modes; 0: all) */
  int32_t kernel; /* tensor-core kernel: 1 cell-major, 2 channel-major, 3 cell-major with
                     dense A tiles (0: default) */
  float ms;       /* time per grid call */
} hegrid_tune_point;
typedef struct {
  int32_t n, best;
  hegrid_tune_point pt[HEGRID_TUNE_MAX];
} hegrid_tune_report;
hegrid_status hegrid_autotune(hegrid_plan *plan, const void *values, hegrid_dtype dtype,
                              int64_t n_channels, int64_t ld_values, uint32_t mode, void *stream,
                              hegrid_tune_report *report);

/*
 * hegrid_plan_set_tuning -- set the launch shape hegrid_autotune would keep
 * (for instance one found in an earlier run; the tuning of Sec. 5.3).  band: blocks per band
 * (0: default).  FP32 mode: >= 1, or -1: the channel tiles of a block back to back.
 * Tensor-core modes: > 0 runs the channel tiles one after another over all
 * blocks, < 0 runs the channel tiles of each block side by side (bands of
 * -band block columns), so that they share the block's weight entries in L2:
 * `group` tiles at a time (0: all of them; the groups follow one another over
 * all blocks, so that fewer blocks run at once and more of them share sample
 * rows in L2); group is ignored for band > 0 and for FP32 mode.
 * kernel (tensor-core modes): 1 runs the cell-major kernel (cells x channels
 * per MMA, weight tiles built in shared memory from the plan's entries, one
 * per channel tile); 2 the channel-major kernel (channels x cells per MMA,
 * the values gathered into shared memory and stored into tensor memory as
 * the MMA's A operand, the weights from dense tiles built once per plan,
 * 128-channel tiles: the first grid call that
 * runs it builds them, 16 KB per 32 candidate slots, on its stream, outside
 * a stream capture, where the cell-major kernel runs until they exist);
 * 3 the cell-major kernel with its A tiles copied whole from those dense
 * tiles (the same maps as 1, bit for bit; all 16 producer warps convert B);
 * 0: the default, the cell-major kernel.  FP32 mode ignores it.
 * seg: 32-candidate sub-chunks per accumulation segment for the tensor-core
 * modes, 1..16 (0: default 16; longer segments would leave the split form
 * too little margin inside its error bound).  The 64-channel tile moves two sub-chunks per step and rounds
 * seg down to an even count (at least 2).
 * INVALID_ARG otherwise (also group < 0, kernel outside 0..3).
 */
hegrid_status hegrid_plan_set_tuning(hegrid_plan *plan, uint32_t mode, int32_t band, int32_t seg,
                                     int32_t group, int32_t kernel);

/*
 * hegrid_autotune_bins -- time hegrid_plan_create (plus destroy) for bin edges
 * of 1..4 map cells (the plan_create flags; the index-resolution study of
 * Sec. 5.3) on the given samples and return
 * the fastest in *best_bin_cells; ms[4] (may be NULL) receives the times.
 * Arguments as for hegrid_plan_create.  Synchronises the device.
 * Errors: INVALID_ARG (best_bin_cells NULL, and as for hegrid_plan_create);
 * UNSUPPORTED, OOM and CUDA as for hegrid_plan_create.
 */
hegrid_status hegrid_autotune_bins(int64_t n_samples, const double *lon_deg, const double *lat_deg,
                                   int coords_on_device, const hegrid_map_geom *geom,
                                   const hegrid_kernel *kern, void *stream,
                                   int32_t *best_bin_cells, float *ms);

/*
 * hegrid_fp32_peak -- measure the GPU's FP32 FMA throughput (TFLOP/s, 2 flop
 * per FMA): every SM runs independent FMA chains for a few milliseconds.  The
 * roofline of HEGRID_MODE_FP32, whose bound is the CUDA-core ALU.
 * Synchronises `stream`.  Errors: INVALID_ARG (tflops NULL); OOM; CUDA.
 * (Measurement service; no step of the paper.)
 */
hegrid_status hegrid_fp32_peak(double *tflops, void *stream);

/* Device-side error word of the plan: OK, or TIMEOUT if a bounded wait of a
 * kernel that used the plan gave up (the kernel then returned early and its
 * outputs are incomplete).  Waits for the plan's creation.  Errors:
 * INVALID_ARG (plan NULL); CUDA.  (Library service; no step of the paper.) */
hegrid_status hegrid_status_poll(const hegrid_plan *plan);

/* Number of CUDA kernels this library has launched in this process (for
 * profiling and launch accounting; counts launches recorded into graphs once,
 * at capture). */
int64_t hegrid_launch_count(void);

/* Bytes of the current device's library pool (the stream-ordered pool every
 * plan, batch scratch and per-call scratch comes from) that are allocated now
 * (*used_bytes) and held from the device (*reserved_bytes, freed blocks kept for
 * reuse included); either pointer may be NULL.  Stream-ordered frees count once
 * the stream has reached them.  For leak checks, e.g. after a failed call.
 * Errors: INVALID_ARG (both NULL); CUDA.  (Library service; no step of the
 * paper.)
 *
 * Failure-path testing: the environment variable HEGRID_FAULT, read at each
 * allocation and launch, injects one failure -- "alloc:N" makes the N-th pool
 * allocation fail (the call returns OOM), "launch:N" makes the N-th kernel
 * launch report a launch failure (the call returns CUDA), and "wait:N" runs the
 * N-th tensor-core grid kernel with one producer arrive withheld and a 20 ms
 * wait limit, so that the kernel's bounded waits run out and hegrid_status_poll
 * returns TIMEOUT.  Counts start when the variable's text changes; unset or any
 * other text injects nothing. */
hegrid_status hegrid_pool_usage(int64_t *used_bytes, int64_t *reserved_bytes);

/* Thread-local message describing the most recent failure ("" if none). */
const char *hegrid_last_error(void);

/*
 * hegrid_bin_sort_noalloc -- the plan's bin key, stable radix sort and bin
 * offsets (perm and bin_off, exactly as hegrid_plan_export returns them) for
 * callers that cannot allocate device memory: code running where
 * cudaMalloc/cudaMallocAsync is not permitted or not wanted, such as an
 * allocator-controlled host framework that forbids foreign allocations, a
 * real-time loop that must not block on the allocator, or a region where the
 * caller has promised a fixed memory budget.  It calls no cudaMalloc,
 * cudaFree or allocating library routine.  (The paper has no counterpart: its
 * sort ran on the CPU.)
 *
 * Scratch lives in one fixed device array of about 8.5 MB compiled into the
 * library; every GPU that loads the library holds it until the process
 * exits.  Hence n_samples <= 524288 (HEGRID_NOALLOC_MAX_SAMPLES); larger
 * inputs return INVALID_ARG before any launch.  All calls share the array:
 * calls that overlap on the GPU (different streams, or the same stream from
 * several threads without ordering) race and corrupt each other's result.
 * Every scratch word a call reads was written by that same call, so nothing
 * has to be cleared between calls.  The first call on each device looks up
 * the array's device address (with that device current) and keeps it for the
 * life of the process; make that first call before any stream capture.  A
 * device or primary-context reset (cudaDeviceReset) after that first call is
 * not supported: the kept address would no longer be the array's.
 *
 * lon_deg, lat_deg  device FP64 [n_samples] (caller-owned).
 * geom, kern, flags as for hegrid_plan_create, plain-grid map bins only:
 * HEGRID_PLAN_HEALPIX, HEGRID_PLAN_SFL and HEGRID_PLAN_DENSE_TILES are
 * INVALID_ARG here.
 * perm_out          device int32 [n_samples].
 * bin_off_out       device int32 [bin_off_capacity], capacity >= n_bins + 1.
 * n_bins_out        host; set to the number of bins even when the capacity is
 *                   too small (INVALID_ARG), so the caller can size the buffer.
 * Asynchronous on `stream`.
 */
#define HEGRID_NOALLOC_MAX_SAMPLES 524288
hegrid_status hegrid_bin_sort_noalloc(int64_t n_samples, const double *lon_deg,
                                      const double *lat_deg, const hegrid_map_geom *geom,
                                      const hegrid_kernel *kern, uint32_t flags, int32_t *perm_out,
                                      int32_t *bin_off_out, int64_t bin_off_capacity,
                                      int64_t *n_bins_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HEGRID_H */
