// Plan construction: the shared component of HEGrid (Sec. 4.1.1 and 4.3.1)
// rebuilt for the GPU.
//
//   a1  coordinate prep: unit vectors of the samples in FP64
//   a2  bin key of the padded map (replaces the HEALPix pixel index)
//   a3  stable LSD radix sort of (key, index) and bin-range offsets (the LUT)
//   a4  per-cell neighbour lists (Algorithm 1's ring/pixel search and its
//       d <= R test), one pass into ranges reserved by upper bounds
//   a5  FP32 weights of every in-radius pair, computed once and shared by all
//       channels, plus W[m] = sum of the weights
//
// Work on cells is organised in 16 x 8 cell blocks: a CTA owns one block, stages
// the samples of the bins around it in shared memory and tests them against
// its 128 cells.  The membership test runs in FP32 in a block-local frame with
// a proven error band; pairs inside the band are decided in FP64.  Weights are
// computed in float-float arithmetic from the same frame.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hegrid_internal.cuh"

namespace hg {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
const char* last_error() { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// Host-side fault injection for the failure-path tests.  HEGRID_FAULT =
// "alloc:N" makes the N-th pool allocation fail with out-of-memory, "launch:N"
// makes the N-th kernel launch report a launch failure at its next error
// check, "wait:N" runs the N-th tensor-core grid launch with one producer
// arrive withheld and a short wait limit, so that its bounded waits run out
// (the counts start when the variable's text last changed).  Unset: no effect
// beyond one getenv per event.
// ---------------------------------------------------------------------------
namespace {
struct FaultState {
  std::mutex mu;
  std::string text;  // the variable as last parsed
  int kind = kFaultNone;
  int64_t n = 0, seen = 0;
};
FaultState& fault_state() {
  static FaultState st;
  return st;
}
thread_local bool t_launch_fault = false;
}  // namespace

bool fault_hit(int kind) {
  const char* env = std::getenv("HEGRID_FAULT");
  FaultState& f = fault_state();
  std::lock_guard<std::mutex> lock(f.mu);
  const std::string text = env ? env : "";
  if (text != f.text) {
    f.text = text;
    f.kind = kFaultNone;
    f.n = 0;
    f.seen = 0;
    const size_t c = text.find(':');
    if (c != std::string::npos) {
      const std::string what = text.substr(0, c);
      const long long n = std::atoll(text.c_str() + c + 1);
      if (n >= 1) {
        f.n = n;
        f.kind = what == "alloc" ? kFaultAlloc : what == "launch" ? kFaultLaunch
                                              : what == "wait" ? kFaultWait : kFaultNone;
      }
    }
  }
  if (f.kind != kind) return false;
  return ++f.seen == f.n;
}

static std::atomic<int64_t> g_launches{0};
void count_launch(int n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  for (int i = 0; i < n; ++i)
    if (fault_hit(kFaultLaunch)) t_launch_fault = true;
}
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

cudaError_t launch_status() {
  if (t_launch_fault) {
    t_launch_fault = false;
    return cudaErrorLaunchFailure;
  }
  return cudaGetLastError();
}

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kDeg = kPi / 180.0;

// ---------------------------------------------------------------------------
// a1 + a2: per-sample unit vector and bin key.
// ---------------------------------------------------------------------------
struct KeyParams {
  double lon0, lat0, dlon, dlat, cx, cy, wx, wy;
  double rdlon, rdlat;  // RN(1 / dlon), RN(1 / dlat)
  int32_t bin_cells, nbx;
  uint32_t n_bins;
  int32_t sfl;  // 1: Sanson-Flamsteed map, bins of projected x = (lon - lon0) cos(lat)
};

// Sanson-Flamsteed map (the sinusoidal projection about lon0): cells lie on
// the regular grid of x = (lon - lon0) cos(lat), y = lat - lat0, so the cell
// (ix, iy) has lon = lon0 + x / cos(lat).  The x-range that holds every point
// within R of a cell at RA offset a_c and latitude lat_c: such points have
// |lon - lon_c| <= H = asin(sin R / cos lat_c) and latitudes within R, where
// cos(lat) lies between the cosines of the ends (1 if the range holds the
// equator); x is extreme at those bounds.  (Same arithmetic on host and
// device; the host's sizes the padding identically to the oracle.)
__host__ __device__ __forceinline__ void sfl_xrange(double a_c, double lat_c, double R_deg,
                                                    double sinR, double& x_lo, double& x_hi) {
  const double H = asin(sinR / cos(lat_c * kDeg)) / kDeg;
  const double c1 = cos((lat_c - R_deg) * kDeg), c2 = cos((lat_c + R_deg) * kDeg);
  const double cmin = fmin(c1, c2);
  const double cmax = (lat_c - R_deg <= 0.0 && lat_c + R_deg >= 0.0) ? 1.0 : fmax(c1, c2);
  const double a = a_c - H, b = a_c + H;
  x_lo = a >= 0.0 ? a * cmin : a * cmax;
  x_hi = b >= 0.0 ? b * cmax : b * cmin;
}

// ---------------------------------------------------------------------------
// HEALPix variant of a2: the paper's own pixelisation (Sec. 4.1.1), RING
// scheme (Gorski et al. 2005).  N = nside: 4N - 1 rings from the north pole;
// ring i holds 4i pixels in the north cap (i < N), 4N in the belt (N <= i <=
// 3N), 4(4N - i) in the south cap; pixel j's centre is at RA (j + s/2) 360 /
// n_i with s = 1 in the caps and (i - N + 1) mod 2 in the belt.  The key of a
// sample is its pixel's position in a table of the rings that reach the
// padded map and, in each, the pixels whose centres lie within two pixels of
// the map's RA range widened by the kernel (the ring -> pixel-range LUT of
// Sec. 4.1.1).
// ---------------------------------------------------------------------------
struct HpxRing {
  int32_t n;     // pixels in the ring
  int32_t J0;    // first pixel of the ring's range (unwrapped; 0 for a whole ring)
  int32_t cnt;   // pixels in the range
  int32_t half;  // 1: pixel centres offset by half a pixel
  int64_t base;  // first bin of the ring
};

struct HpxParams {
  int32_t nside, ring0, n_rings;
  uint32_t n_bins;
  const HpxRing* rings;
};

// Ring (1 .. 4N-1) and pixel in ring of the point z = sin(lat), t = RA / 90
// deg in [0, 4).  In the belt the pixel edges are the lines t -+ 3z/4 =
// const spaced 1/N: the two edge indices give the ring (difference) and the
// pixel (sum).  In a cap, within each 90-degree face, the edge indices along
// tp = t mod 1 and 1 - tp scaled by N sqrt(3 (1 - |z|)) give the ring from the
// pole, and cap pixels are exact 360 / n_i slices of their ring.  Single IEEE
// operations (no contraction): the bin key is reproducible bit for bit.
__device__ __forceinline__ void hpx_ang2pix(int32_t N, double z, double t, int32_t& ring,
                                            int32_t& pix) {
  const double Nd = (double)N;
  const double az = fabs(z);
  if (az <= 2.0 / 3.0) {
    const double t1 = __dmul_rn(Nd, __dadd_rn(0.5, t));
    const double t2 = __dmul_rn(__dmul_rn(Nd, 0.75), z);
    const int64_t jp = (int64_t)floor(__dsub_rn(t1, t2));
    const int64_t jm = (int64_t)floor(__dadd_rn(t1, t2));
    const int64_t ir = N + 1 + jp - jm;  // 1 .. 2N+1 from the ring at z = 2/3
    const int64_t kshift = 1 - (ir & 1);
    int64_t ip = (jp + jm - N + kshift + 1) / 2;
    ip = ((ip % (4 * (int64_t)N)) + 4 * (int64_t)N) % (4 * (int64_t)N);
    ring = (int32_t)(N - 1 + ir);
    pix = (int32_t)ip;
    return;
  }
  const double tp = __dsub_rn(t, floor(t));
  const double tmp = __dmul_rn(Nd, __dsqrt_rn(__dmul_rn(3.0, __dsub_rn(1.0, az))));
  const int64_t jp = (int64_t)floor(__dmul_rn(tp, tmp));
  const int64_t jm = (int64_t)floor(__dmul_rn(__dsub_rn(1.0, tp), tmp));
  int64_t ir = jp + jm + 1;  // ring from the nearest pole, 1 .. N
  if (ir > N) ir = N;
  int64_t ip = (int64_t)floor(__dmul_rn(t, (double)ir));
  if (ip >= 4 * ir) ip = 4 * ir - 1;
  ring = (int32_t)(z > 0.0 ? ir : 4 * (int64_t)N - ir);
  pix = (int32_t)ip;
}

// Continuous ring coordinate of z (ring centres at integers).  A pixel of
// ring i lies between the centres of rings i - 1 and i + 1.
__host__ __device__ __forceinline__ float hpx_rho_f(int32_t N, float z) {
  const float Nf = (float)N;
  if (z > 2.0f / 3.0f) return Nf * sqrtf(fmaxf(3.0f * (1.0f - z), 0.0f));
  if (z < -2.0f / 3.0f) return 4.0f * Nf - Nf * sqrtf(fmaxf(3.0f * (1.0f + z), 0.0f));
  return Nf * (2.0f - 1.5f * z);
}

// Bins [x, y] of ring e whose pixels can hold a point with RA in [pa, pb]
// (degrees, unwrapped): pixels whose centres lie within two pixels of the
// range (a pixel's RA extent is its centre +- half a pixel); x > y if none.
__device__ __forceinline__ int2 hpx_span(const HpxRing& e, float pa, float pb) {
  const float s = (float)e.n * (1.0f / 360.0f);
  const float h = e.half ? 0.5f : 0.0f;
  const int ja = (int)ceilf(pa * s - h - 2.0f), jb = (int)floorf(pb * s - h + 2.0f);
  if (e.cnt == e.n) {  // the whole ring is in the table (J0 = 0)
    if (jb - ja + 1 >= e.n) return make_int2(0, e.n - 1);
    const int a = ((ja % e.n) + e.n) % e.n, b = a + (jb - ja);
    return b >= e.n ? make_int2(0, e.n - 1) : make_int2(a, b);
  }
  return make_int2(max(ja - e.J0, 0), min(jb - e.J0, e.cnt - 1));
}

// floor(RN(RN(x / d) + c)), the key's FP64 expression, exactly, without the
// division where that is safe: y0 = x * rcp + c (rcp = RN(1 / d)) lies within
// a few units of 2^-53 (|x / d| + |c|) of RN(RN(x / d) + c), so when no integer
// lies within 1e-12 (|x / d| + |c| + 1) of y0 both have the same floor;
// otherwise (and for non-finite or huge values) the correctly rounded
// expression decides.
__device__ __forceinline__ double floor_div_add(double x, double d, double rcp, double c) {
  const double q0 = x * rcp;
  const double y0 = q0 + c;
  const double f = floor(y0);
  const double eps = 1e-12 * (fabs(q0) + fabs(c) + 1.0);
  if (y0 - f > eps && (f + 1.0) - y0 > eps) return f;
  return floor(__dadd_rn(__ddiv_rn(x, d), c));
}

// a - 360 floor(RN(RN(a + 180) / 360)) exactly: for RN(a + 180) in [0, 360)
// the quotient rounds into [0, 1) (the largest double below 360, over 360,
// rounds to 1 - 2^-53), so the floor is 0 without dividing.
__device__ __forceinline__ double wrap_ra(double a) {
  const double x = __dadd_rn(a, 180.0);
  if (x >= 0.0 && x < 360.0) return a;
  return __dsub_rn(a, __dmul_rn(360.0, floor(__ddiv_rn(x, 360.0))));
}

template <bool kHpx>
__global__ void k_prep(int32_t N, const double* __restrict__ lon, const double* __restrict__ lat,
                       KeyParams kp, HpxParams hp, uint32_t* __restrict__ key,
                       int32_t* __restrict__ idx) {
  int32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double lo = lon[n], la = lat[n];
  // sin and cos of the latitude only where the key needs them (the HEALPix
  // ring index, the projected x); the unit vectors follow the sort
  double sd = 0.0, cd = 1.0;
  if (kHpx || kp.sfl) sincos(la * kDeg, &sd, &cd);
  uint32_t k;
  if constexpr (kHpx) {
    // RA wrapped into [0, 360), then the ring-scheme pixel of (sin(lat), RA)
    const double a = __dsub_rn(lo, __dmul_rn(360.0, floor(__ddiv_rn(lo, 360.0))));
    int32_t ring, pix;
    hpx_ang2pix(hp.nside, sd, __ddiv_rn(a, 90.0), ring, pix);
    k = hp.n_bins;
    const int32_t r = ring - hp.ring0;
    if (r >= 0 && r < hp.n_rings) {
      const HpxRing e = hp.rings[r];
      const int32_t jr = ((pix - e.J0) % e.n + e.n) % e.n;
      if (jr < e.cnt) k = (uint32_t)(e.base + jr);
    }
  } else {
    // Bin key: the floor of an expression of single IEEE operations (no
    // contraction), so the key is reproducible bit for bit by any IEEE-754
    // implementation; the floors are taken exactly (floor_div_add, wrap_ra).
    double a = wrap_ra(__dsub_rn(lo, kp.lon0));
    if (kp.sfl) a = __dmul_rn(a, cd);  // projected x
    double fx = floor_div_add(a, kp.dlon, kp.rdlon, kp.cx);
    double fy = floor_div_add(__dsub_rn(la, kp.lat0), kp.dlat, kp.rdlat, kp.cy);
    k = kp.n_bins;
    if (isfinite(fx) && isfinite(fy) && fx >= 0.0 && fy >= 0.0 && fx < kp.wx && fy < kp.wy) {
      int64_t bx = (int64_t)fx / kp.bin_cells, by = (int64_t)fy / kp.bin_cells;
      k = (uint32_t)(by * kp.nbx + bx);
    }
  }
  key[n] = k;
  idx[n] = n;
}

// ---------------------------------------------------------------------------
// a3: stable LSD radix sort (8-bit digits) of (key, index).
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;  // rounds of 256 consecutive elements per tile
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads)
    k_radix_hist(const uint32_t* __restrict__ keys, int32_t N, int shift, int32_t n_tiles,
                 int32_t* __restrict__ hist) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < N) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];  // digit-major
}

__global__ void __launch_bounds__(kSortThreads)
    k_radix_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                    uint32_t* __restrict__ kout, int32_t* __restrict__ vout, int32_t N, int shift,
                    int32_t n_tiles, const int32_t* __restrict__ offs) {
  constexpr int W = kSortThreads / 32;
  __shared__ int32_t wcnt[W][257];
  __shared__ int32_t woff[W][257];
  __shared__ int32_t run[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = offs[(int64_t)tid * n_tiles + blockIdx.x];
  for (int w = 0; w < W; ++w) wcnt[w][tid] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + r * kSortThreads + tid;
    bool valid = i < N;
    uint32_t k = valid ? kin[i] : 0u;
    int32_t v = valid ? vin[i] : 0;
    int d = valid ? (int)((k >> shift) & 255u) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      int dd = tid;  // one digit per thread
      int32_t acc = run[dd];
      for (int w = 0; w < W; ++w) {
        woff[w][dd] = acc;
        acc += wcnt[w][dd];
        wcnt[w][dd] = 0;
      }
      run[dd] = acc;
    }
    __syncthreads();
    if (valid) {
      int32_t dst = woff[warp][d] + rank;
      kout[dst] = k;
      vout[dst] = v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Exclusive scans (three-phase, 4096 items per CTA).
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads)
    k_scan_tiles(const TI* in, int64_t n, TO* out, TO* tile_sums) {
  __shared__ TO warp_sums[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)tid * kScanItems;
  TO v[kScanItems];
  TO local = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = (base + j < n) ? (TO)in[base + j] : (TO)0;
    local += v[j];
  }
  TO x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    TO y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    TO s = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      TO y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;
  }
  __syncthreads();
  TO excl = x - local + (warp > 0 ? warp_sums[warp - 1] : (TO)0);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < n) out[base + j] = excl;
    excl += v[j];
  }
  if (tid == kScanThreads - 1 && tile_sums) tile_sums[blockIdx.x] = warp_sums[31];
}

template <typename TO>
__global__ void k_scan_add(TO* __restrict__ out, int64_t n, const TO* __restrict__ tile_offs) {
  int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  TO add = tile_offs[blockIdx.x];
  for (int j = 0; j < kScanItems; ++j, i += kScanThreads)
    if (i < n) out[i] += add;
}

template <typename T>
__global__ void k_set_total(T* out, int64_t n, const T* excl_last, const T* in_last) {
  out[n] = *excl_last + *in_last;
}

// out[0..n] = exclusive scan of in[0..n) with out[n] = total.  `tmp` needs
// scan_tmp_elems(n) elements.
constexpr int64_t scan_tmp_elems(int64_t n) {
  int64_t t = 0;
  while (n > kScanTile) {
    n = (n + kScanTile - 1) / kScanTile;
    t += n + 1;
  }
  return t + 1;
}

template <typename TI, typename TO>
void scan_exclusive(const TI* in, int64_t n, TO* out, TO* tmp, cudaStream_t s);

template <typename TO>
void scan_in_place(TO* data, int64_t n, TO* tmp, cudaStream_t s) {
  // data holds n inputs; replaced by their exclusive scan (no total).
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles <= 1) {
    k_scan_tiles<TO, TO><<<1, kScanThreads, 0, s>>>(data, n, data, (TO*)nullptr);
    count_launch();
    return;
  }
  TO* sums = tmp;
  k_scan_tiles<TO, TO><<<(unsigned)tiles, kScanThreads, 0, s>>>(data, n, data, sums);
  count_launch();
  scan_in_place<TO>(sums, tiles, tmp + tiles + 1, s);
  k_scan_add<TO><<<(unsigned)tiles, kScanThreads, 0, s>>>(data, n, sums);
  count_launch();
}

template <typename TI, typename TO>
void scan_exclusive(const TI* in, int64_t n, TO* out, TO* tmp, cudaStream_t s) {
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles <= 1) {
    k_scan_tiles<TI, TO><<<1, kScanThreads, 0, s>>>(in, n, out, (TO*)nullptr);
    count_launch();
  } else {
    TO* sums = tmp;
    k_scan_tiles<TI, TO><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, out, sums);
    count_launch();
    scan_in_place<TO>(sums, tiles, tmp + tiles + 1, s);
    k_scan_add<TO><<<(unsigned)tiles, kScanThreads, 0, s>>>(out, n, sums);
    count_launch();
  }
}

// bin_off[k] = first sorted position with key >= k, for k in [0, n_bins].
__global__ void k_bin_offsets(const uint32_t* __restrict__ skey, int32_t N, uint32_t n_bins,
                              int32_t* __restrict__ bin_off) {
  int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  int64_t prev = s > 0 ? (int64_t)skey[s - 1] : -1;
  int64_t cur = skey[s];
  for (int64_t k = prev + 1; k <= cur && k <= (int64_t)n_bins; ++k) bin_off[k] = s;
  if (s == N - 1)
    for (int64_t k = cur + 1; k <= (int64_t)n_bins; ++k) bin_off[k] = N;
}

// Unit vectors (FP64) of the samples in sorted order: the FP64 sines and
// cosines bound this kernel, so the gathered coordinate reads cost little.
__global__ void k_unit_sorted(const int32_t* __restrict__ perm, int32_t N,
                              const double* __restrict__ lon, const double* __restrict__ lat,
                              double* __restrict__ sx, double* __restrict__ sy,
                              double* __restrict__ sz) {
  int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int32_t n = perm[s];
  double sa, ca, sd, cd;
  sincos(lon[n] * kDeg, &sa, &ca);
  sincos(lat[n] * kDeg, &sd, &cd);
  sx[s] = cd * ca;
  sy[s] = cd * sa;
  sz[s] = sd;
}

// ---------------------------------------------------------------------------
// a4 + a5: block-local neighbour search and weights.
// ---------------------------------------------------------------------------
// Candidate windows of a cell block and of each warp's 8 x 4 tile of it.
// Padded-map bins: rows by0..by1, columns bx0..bx1 (int4 x, y, z, w).
// HEALPix: rings r0..r1 and, in each, the bins of the pixels that can hold a
// point with RA in [pa, pb] (hpx_span).
struct HWin {
  int32_t r0, r1;
  float pa, pb;
};

struct WinArgs {
  const int4* win;    // [n_blocks] padded-map bins
  const int4* wwin;   // [4 n_blocks]
  const HWin* hwin;   // [n_blocks] HEALPix
  const HWin* hwwin;  // [4 n_blocks]
  HpxParams hp;
};

// Sample range [lo, hi) of window row `row` (a bin row, or a ring).
template <bool kHpx>
__device__ __forceinline__ void window_row(const WinArgs& wa, const int32_t* __restrict__ bin_off,
                                           int32_t nbx, int row, int4 w, HWin h, int32_t& lo,
                                           int32_t& hi) {
  if constexpr (kHpx) {
    lo = hi = 0;
    if (row < h.r0 || row > h.r1) return;
    const HpxRing e = wa.hp.rings[row - wa.hp.ring0];
    const int2 sp = hpx_span(e, h.pa, h.pb);
    if (sp.x > sp.y) return;
    lo = bin_off[e.base + sp.x];
    hi = bin_off[e.base + sp.y + 1];
  } else {
    lo = hi = 0;
    if (row < w.x || row > w.y) return;
    lo = bin_off[(int64_t)row * nbx + w.z];
    hi = bin_off[(int64_t)row * nbx + w.w + 1];
  }
}

struct PairParams {
  int32_t nx, ny, nbx_b, nbx;  // map, cell blocks along RA, bins along RA
  int32_t sfl;                 // 1: Sanson-Flamsteed cell centres
  int64_t M;
  double lon0, lat0, dlon, dlat;
  double cR2;       // chord^2 at R: 4 sin^2(R/2), FP64
  float lo_thr;     // FP32 c^2 below this: inside for sure
  float hi_thr;     // FP32 c^2 above this: outside for sure
  float k_hi, k_lo; // 1 / (2 sigma^2) in rad^-2 as float-float
};

constexpr int kChunk = 128;  // candidates staged per round (= threads per CTA)

__device__ __forceinline__ void unit_vec(double lon_deg, double lat_deg, double& x, double& y,
                                         double& z) {
  double sa, ca, sd, cd;
  sincos(lon_deg * kDeg, &sa, &ca);
  sincos(lat_deg * kDeg, &sd, &cd);
  x = cd * ca;
  y = cd * sa;
  z = sd;
}

// Exact difference a - b = s + e of two floats (Knuth's TwoSum on a, -b).
__device__ __forceinline__ void two_diff(float a, float b, float& s, float& e) {
  s = __fsub_rn(a, b);
  float v = __fsub_rn(s, a);
  e = __fsub_rn(__fsub_rn(a, __fsub_rn(s, v)), __fadd_rn(b, v));
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

// Gaussian weight of a pair from block-local float-float coordinates.
//   chord c = |u_m - u_n| (float-float), d^2 = c^2 g(c^2/4) with
//   g(h) = asin^2(sqrt h)/h = 1 + h/3 + 8h^2/45 + 4h^3/35 + 128h^4/1575 + ...
//   (the power series of arcsin^2), w = exp(-d^2 / (2 sigma^2)).
// Relative error ~3 ulp of FP32 for h <= 0.01.
__device__ __forceinline__ float pair_weight(const float (&mh)[3], const float (&ml)[3],
                                             const float (&nh)[3], const float (&nl)[3],
                                             float k_hi, float k_lo) {
  float h[3], l[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float s, e;
    two_diff(mh[i], nh[i], s, e);
    h[i] = s;
    l[i] = __fadd_rn(e, __fsub_rn(ml[i], nl[i]));
  }
  float p[3], pe[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    p[i] = __fmul_rn(h[i], h[i]);
    pe[i] = __fmaf_rn(h[i], h[i], -p[i]) + 2.0f * h[i] * l[i];
  }
  float s01, t01, S, t2;
  two_sum(p[0], p[1], s01, t01);
  two_sum(s01, p[2], S, t2);
  float Slo = t01 + t2 + pe[0] + pe[1] + pe[2];
  float ch = __fadd_rn(S, Slo);
  float cl = __fsub_rn(Slo, __fsub_rn(ch, S));
  float hh = 0.25f * ch;
  float corr =
      hh * (1.0f / 3.0f + hh * (8.0f / 45.0f + hh * (4.0f / 35.0f + hh * (128.0f / 1575.0f))));
  float xl = cl + ch * corr;
  float xh = __fadd_rn(ch, xl);
  xl = __fsub_rn(xl, __fsub_rn(xh, ch));
  float th = __fmul_rn(xh, k_hi);
  float tl = __fmaf_rn(xh, k_hi, -th) + xh * k_lo + xl * k_hi;
  return expf(-th) * (1.0f - tl);
}

// One CTA per 16x8 cell block; thread t owns block-local cell thread_cell(t)
// (each warp an 8 x 4 tile).  The samples of the bins around the block are
// staged kChunk at a time, one bin row at a time; each warp tests those in
// its own tile's bin window against its cells.  The block writes, inside the
// slot and entry ranges its upper bounds reserved: the candidate list
// (original sample indices, union order, padded to HG_KPAD), its padded
// length, the weight entries in 32-candidate sub-chunks (entry =
// tile_off(cell, candidate & 31), FP32 weight; inside each sub-chunk the
// entries of a cell are contiguous, cells in thread order), the offsets of
// every sub-chunk plus an end sentinel, and W[m].
// Neumaier-compensated running sum.
struct CSum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ float value() const { return s + c; }
};

// 32 x 32 bit-matrix transpose across a warp: bit j of lane i's word becomes
// bit i of lane j's word (five rounds of swapping off-diagonal sub-blocks).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
  uint32_t lo = 0x0000ffffu;  // bits j with (j & s) == 0
#pragma unroll
  for (int s = 16; s > 0; s >>= 1, lo ^= lo << s) {
    const uint32_t p = __shfl_xor_sync(0xffffffffu, x, s);
    x = (lane & s) ? ((x & ~lo) | ((p & ~lo) >> s)) : ((x & lo) | ((p & lo) << s));
  }
  return x;
}

// Position of the (j+1)-th set bit of x (j < popc(x)).
__device__ __forceinline__ int select_bit(uint32_t x, int j) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) {
    const int c = __popc(x & ((1u << w) - 1u));
    if (j >= c) {
      j -= c;
      pos += w;
      x >>= w;
    }
  }
  return pos;
}

// Block-local cell of thread t: each warp owns an 8 x 4 tile of the 16 x 8
// block (warp w: columns 8 (w & 1) .. +7, rows 4 (w >> 1) .. +3), so that a
// warp's bin window is narrower than the block's in both directions.
__host__ __device__ __forceinline__ int thread_cell(int t) {
  const int w = t >> 5, lane = t & 31;
  return ((w >> 1) * 4 + (lane >> 3)) * HG_BX + (w & 1) * 8 + (lane & 7);
}

template <bool kHpx>
__global__ void __launch_bounds__(kChunk)
    k_block_pairs(PairParams pp, WinArgs wa, const int32_t* __restrict__ bin_off,
                  const int32_t* __restrict__ perm, const double* __restrict__ sx,
                  const double* __restrict__ sy, const double* __restrict__ sz,
                  const int64_t* __restrict__ cand_off, const int64_t* __restrict__ blk_pair_off,
                  int32_t* __restrict__ cand_cnt, int32_t* __restrict__ cand_idx,
                  int64_t* __restrict__ sub_off, uint16_t* __restrict__ ent_ck,
                  float* __restrict__ ent_w, float* __restrict__ wsum,
                  unsigned long long* __restrict__ totals, int32_t blk0) {
  constexpr int kQ = kChunk / 32;
  // staged candidates' block-local coordinates as float-float (x, y, z, -)
  __shared__ float4 s_eh[kChunk];
  __shared__ float4 s_el[kChunk];
  __shared__ double s_u[3][kChunk];
  __shared__ int32_t s_n[kChunk];
  __shared__ uint32_t s_umask[kQ];
  __shared__ int32_t s_red[kQ];
  // Cell coordinates (by block-local cell), candidate-major masks (bit i
  // of s_cm[k][w]: the cell of thread 32 w + i has staged candidate k),
  // entries before each staged candidate, candidate index within its
  // 32-candidate sub-chunk.
  __shared__ float4 s_mh[kChunk];
  __shared__ float4 s_ml[kChunk];
  __shared__ uint32_t s_cm[kChunk][kQ];
  __shared__ int32_t s_loc[kChunk];
  __shared__ int32_t s_gred[kQ][kQ];       // per group, per warp: summed (cA | cB << 16)
  __shared__ int32_t s_ginc[kQ][kChunk];   // per group, per thread: inclusive warp prefix
  __shared__ uint16_t s_ent[32 * kChunk];  // (cell << 5 | candidate) of a group
  __shared__ float s_w[32 * kChunk];       // weights of a span of groups, by cell
  __shared__ uint32_t s_pab[kQ][kChunk];   // per group, per cell: entry -> s_w slot shifts
  __shared__ double s_sc[HG_BX + HG_BY][2];  // (sin, cos) of the column RAs, then row latitudes
  __shared__ double s_b0[3];                 // unit vector of the block centre

  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int b = blk0 + (int)blockIdx.x;  // a launch covers blocks blk0 ..
  const int bbx = b % pp.nbx_b, bby = b / pp.nbx_b;
  const int cell = thread_cell(t);
  const int ix = bbx * HG_BX + (cell % HG_BX), iy = bby * HG_BY + (cell / HG_BX);
  const bool active = ix < pp.nx && iy < pp.ny;
  const int64_t m = (int64_t)iy * pp.nx + ix;
  // this block's and this warp's candidate windows
  int4 wb = make_int4(1, 0, 0, 0), ww = make_int4(1, 0, 0, 0);
  HWin hb = {1, 0, 0.0f, 0.0f}, hw = {1, 0, 0.0f, 0.0f};
  if constexpr (kHpx) {
    hb = wa.hwin[b];
    hw = wa.hwwin[4 * (int64_t)b + wid];
  } else {
    wb = wa.win[b];
    ww = wa.wwin[4 * (int64_t)b + wid];
  }
  const int row0 = kHpx ? hb.r0 : wb.x, row1 = kHpx ? hb.r1 : wb.y;

  // Block-local frame: origin at the unit vector of the block's centre.
  double bx0, by0, bz0;
  // (x, lat) -> lon of a cell centre: x itself on the plain grid, x / cos(lat)
  // on the Sanson-Flamsteed map
  auto lon_of = [&](double x, double lat) {
    return pp.sfl ? pp.lon0 + x / cos(lat * kDeg) : pp.lon0 + x;
  };
  // FP64 sines and cosines once per block (the FP64 pipe is slow): the
  // block centre's unit vector, and on the plain grid (RA by column, latitude
  // by row) those of the block's 16 column RAs and 8 row latitudes, which a
  // cell's unit vector combines; the Sanson-Flamsteed map takes its own per cell.
  if (t == HG_BX + HG_BY) {
    const double xb = ((double)bbx * HG_BX + 0.5 * (HG_BX - 1) - 0.5 * (pp.nx - 1)) * pp.dlon;
    const double lb = pp.lat0 + ((double)bby * HG_BY + 0.5 * (HG_BY - 1) - 0.5 * (pp.ny - 1)) * pp.dlat;
    unit_vec(lon_of(xb, lb), lb, s_b0[0], s_b0[1], s_b0[2]);
  } else if (!pp.sfl && t < HG_BX) {
    sincos((pp.lon0 + ((double)(bbx * HG_BX + t) - 0.5 * (pp.nx - 1)) * pp.dlon) * kDeg,
           &s_sc[t][0], &s_sc[t][1]);
  } else if (!pp.sfl && t < HG_BX + HG_BY) {
    const int r = t - HG_BX;
    sincos((pp.lat0 + ((double)(bby * HG_BY + r) - 0.5 * (pp.ny - 1)) * pp.dlat) * kDeg,
           &s_sc[t][0], &s_sc[t][1]);
  }
  __syncthreads();
  bx0 = s_b0[0];
  by0 = s_b0[1];
  bz0 = s_b0[2];
  double um[3];
  if (!pp.sfl) {
    const double sa = s_sc[cell % HG_BX][0], ca = s_sc[cell % HG_BX][1];
    const double sd = s_sc[HG_BX + cell / HG_BX][0], cd = s_sc[HG_BX + cell / HG_BX][1];
    um[0] = cd * ca;
    um[1] = cd * sa;
    um[2] = sd;
  } else {
    const double lc = pp.lat0 + ((double)iy - 0.5 * (pp.ny - 1)) * pp.dlat;
    unit_vec(lon_of(((double)ix - 0.5 * (pp.nx - 1)) * pp.dlon, lc), lc, um[0], um[1], um[2]);
  }
  float mh[3], ml[3];
  {
    double e[3] = {um[0] - bx0, um[1] - by0, um[2] - bz0};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      mh[i] = __double2float_rn(e[i]);
      ml[i] = __double2float_rn(e[i] - (double)mh[i]);
    }
  }

  s_mh[cell] = make_float4(mh[0], mh[1], mh[2], 0.0f);
  s_ml[cell] = make_float4(ml[0], ml[1], ml[2], 0.0f);
  int64_t kcount = 0;  // union size so far (local index of the next candidate)
  int64_t erun = 0;    // entries of the block so far
  // W of the cell for each weight representation the grid kernels use
  // (FP32; FP16-rounded as the tensor-core single form rounds them), so
  // that every form normalises by the sum of exactly the weights it
  // multiplied.
  CSum wsv;         // FP32 weights, compensated
  float w16 = 0.0f;  // FP16-rounded weights x kTcWeightScale (plain sum: single form only)
  const int64_t cbase = cand_off[b], ebase = blk_pair_off[b], sbase = cbase / 32;
  for (int row = row0; row <= row1; ++row) {
    // the row's samples (staged), and the part this warp tests: the bins of
    // its own window, a contiguous sub-range
    int32_t s_beg, s_end, w_lo, w_hi;
    window_row<kHpx>(wa, bin_off, pp.nbx, row, wb, hb, s_beg, s_end);
    window_row<kHpx>(wa, bin_off, pp.nbx, row, ww, hw, w_lo, w_hi);
    for (int32_t base = s_beg; base < s_end; base += kChunk) {
      const int32_t s = base + t;
      const int nk = min(kChunk, s_end - base);
      if (s < s_end) {
        double u[3] = {sx[s], sy[s], sz[s]};
        double e[3] = {u[0] - bx0, u[1] - by0, u[2] - bz0};
        float hv[3], lv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          hv[i] = __double2float_rn(e[i]);
          lv[i] = __double2float_rn(e[i] - (double)hv[i]);
          s_u[i][t] = u[i];
        }
        s_eh[t] = make_float4(hv[0], hv[1], hv[2], 0.0f);
        s_el[t] = make_float4(lv[0], lv[1], lv[2], 0.0f);
        s_n[t] = perm[s];
      }
      if (t < kQ) s_umask[t] = 0u;
      // The staged candidates this warp tests (those of its own window).
      const int k0 = max(w_lo - base, 0), k1 = min(w_hi - base, nk);
      __syncthreads();

      // Phase 1: membership of each staged candidate for this thread's cell.
      // FP32 test first (bit set in `in32` when surely inside, in `maybe`
      // when not surely outside); pairs inside the FP32 error band are
      // decided in FP64 afterwards.
      uint32_t mask[kQ];
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        const int r0 = max(k0 - 32 * q, 0), r1 = min(k1 - 32 * q, 32);
        uint32_t in32 = 0u, maybe = 0u;
#pragma unroll 4
        for (int r = r0; r < r1; ++r) {
          const float4 n4 = s_eh[32 * q + r];
          const float dx = mh[0] - n4.x, dy = mh[1] - n4.y, dz = mh[2] - n4.z;
          const float c2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
          const uint32_t bit = 1u << r;
          if (c2 <= pp.lo_thr) in32 |= bit;
          if (c2 <= pp.hi_thr) maybe |= bit;
        }
        uint32_t band = active ? maybe & ~in32 : 0u;
        while (band) {
          const int r = __ffs(band) - 1;
          band &= band - 1u;
          const int k = 32 * q + r;
          const double ex = um[0] - s_u[0][k], ey = um[1] - s_u[1][k], ez = um[2] - s_u[2][k];
          if (ex * ex + ey * ey + ez * ez <= pp.cR2) in32 |= 1u << r;
        }
        mask[q] = active ? in32 : 0u;
      }
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        uint32_t wmask = __reduce_or_sync(0xffffffffu, mask[q]);
        if (lane == 0 && wmask) atomicOr(&s_umask[q], wmask);
        s_cm[32 * q + lane][wid] = transpose32(mask[q], lane);
      }
      __syncthreads();
      uint32_t um4[kQ];
      int ucount = 0;
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        um4[q] = s_umask[q];
        ucount += __popc(um4[q]);
      }
      {
        // entries of staged candidate t and their exclusive prefix over the
        // staged candidates
        int cc = 0;
#pragma unroll
        for (int w = 0; w < kQ; ++w) cc += __popc(s_cm[t][w]);
        int incl = cc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        if (lane == 31) s_red[wid] = incl;
        // Per group of 32 staged candidates: this cell's entry counts on each
        // side of the sub-chunk boundary that may fall inside the group
        // (candidate r_split starts a new sub-chunk), packed in 16-bit halves,
        // and their inclusive prefix over the warp; published with s_red by
        // the one barrier below.
        {
          int ub = 0;
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            const uint32_t uq = um4[q];
            const int jb = (int)((32 - ((kcount + ub) & 31)) & 31);
            ub += __popc(uq);
            const int r_split = jb < __popc(uq) ? select_bit(uq, jb) : 32;
            const uint32_t amask = r_split >= 32 ? 0xffffffffu : ((1u << r_split) - 1u);
            const int v = __popc(mask[q] & amask) | (__popc(mask[q] & ~amask) << 16);
            int inc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int y = __shfl_up_sync(0xffffffffu, inc, o);
              if (lane >= o) inc += y;
            }
            s_ginc[q][t] = inc;
            if (lane == 31) s_gred[q][wid] = inc;
          }
        }
        __syncthreads();
        int wpre = 0, total = 0;
#pragma unroll
        for (int w = 0; w < kQ; ++w) {
          if (w < wid) wpre += s_red[w];
          total += s_red[w];
        }
        const int pre_t = wpre + incl - cc;
        // candidate list and sub-chunk offsets (by the candidate's own thread)
        if (cc > 0) {
          int before = 0;
#pragma unroll
          for (int q = 0; q < kQ; ++q)
            before += __popc(q < wid ? um4[q] : q == wid ? um4[q] & ((1u << lane) - 1u) : 0u);
          const int64_t loc = kcount + before;
          cand_idx[cbase + loc] = s_n[t];
          if ((loc & 31) == 0) sub_off[sbase + loc / 32] = ebase + erun + pre_t;
          s_loc[t] = (int)(loc & 31);
        }
        // The staged candidates in groups of 32 (at most 32 x 128 entries):
        // list the group's (cell, candidate) pairs in entry order, compute
        // the weights one entry per thread (coalesced writes), and add them
        // into W of each cell in candidate order.  Within a group, entries
        // are grouped by cell (in thread order) on each side of the
        // 32-candidate sub-chunk boundary that may fall inside it (candidate
        // r_split starts a new sub-chunk), so every sub-chunk's entries stay
        // contiguous.  The groups form spans: the whole staged chunk when all
        // its weights fit s_w, else each group alone (a span of part of the
        // chunk saves less than its by-cell writes cost in bank conflicts).
        // s_w holds a span's weights by cell (each cell's weights of the span
        // contiguous, in the order they are added: group by group, each
        // group's two sides in turn, candidates in order), so that W takes
        // one pass per span whose length is the cell's own entry count over
        // the span (a pass per group would cost every warp its busiest cell's
        // count in each group).
        uint32_t span_start;  // bit q: group q starts a span
        {
          int acc = 0;
          uint32_t nonempty = 0u;
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            acc += s_red[q];
            if (s_red[q] > 0) nonempty |= 1u << q;
          }
          span_start = acc <= 32 * kChunk ? (nonempty & (0u - nonempty)) : nonempty;
        }
        // this cell's slot in s_w for each group (span start + the cell's
        // entries in the span's earlier groups): the span start is the
        // cell's exclusive prefix over the cells of its entries in the span
        int slot[kQ];
        {
          int exT[kQ];
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            int wp = 0;
#pragma unroll
            for (int w = 0; w < kQ; ++w)
              if (w < wid) wp += s_gred[q][w];
            const int in2 = wp + s_ginc[q][t];
            exT[q] = (in2 & 0xffff) + (in2 >> 16) - __popc(mask[q]);
          }
          int sum = 0;
#pragma unroll
          for (int q = kQ - 1; q >= 0; --q) {
            if (s_red[q] > 0) sum += exT[q];
            slot[q] = sum;  // at a span's first group: the span's start
            if ((span_start >> q) & 1u) sum = 0;
          }
          int base = 0;
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            if (s_red[q] == 0) continue;
            if ((span_start >> q) & 1u) base = slot[q];
            slot[q] = base;
            base += __popc(mask[q]);
          }
        }
        int sp0 = 0, sp1 = 0;  // this cell's s_w slots of the pending span
        auto add_span = [&]() {
          for (int e = sp0; e < sp1; ++e) {
            const float wgt = s_w[e];
            wsv.add(wgt);
            w16 += __half2float(__float2half_rn(wgt * kTcWeightScale));
          }
        };
        int ubefore = 0;  // union candidates of the staged chunk before group q
        int g0 = 0;       // entries of the staged chunk before group q
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          const int gT = s_red[q];  // the group's candidates are warp q's staged ones
          const uint32_t uq = um4[q];
          const int jb = (int)((32 - ((kcount + ubefore) & 31)) & 31);
          ubefore += __popc(uq);
          g0 += q > 0 ? s_red[q - 1] : 0;
          if (gT == 0) continue;
          if ((span_start >> q) & 1u) {
            // the previous span's weights (published by the barrier after
            // its last weight pass; s_w is next written after this group's
            // listing barrier)
            add_span();
            sp0 = sp1 = slot[q];
          }
          const int r_split = jb < __popc(uq) ? select_bit(uq, jb) : 32;
          const uint32_t amask = r_split >= 32 ? 0xffffffffu : ((1u << r_split) - 1u);
          const int cA = __popc(mask[q] & amask), cB = __popc(mask[q] & ~amask);
          // exclusive prefix of (cA, cB) over the cells, packed in 16-bit halves
          const int v = cA | (cB << 16);
          int wp = 0, tot = 0;
#pragma unroll
          for (int w = 0; w < kQ; ++w) {
            if (w < wid) wp += s_gred[q][w];
            tot += s_gred[q][w];
          }
          const int ex = wp + s_ginc[q][t] - v;
          const int a0 = ex & 0xffff, b0 = (tot & 0xffff) + (ex >> 16);
          const int totA = tot & 0xffff;
          // entry e of this cell sits at s_w slot e + shift (A side: entries
          // a0.. go to slot[q]..; B side: entries b0.. follow them)
          s_pab[q][cell] = (uint32_t)(slot[q] - a0) & 0xffffu |
                           (uint32_t)(slot[q] + cA - b0) << 16;
          sp1 += cA + cB;
          {
            int pa = a0, pb = b0;
            uint32_t mm = mask[q];
            while (mm) {
              const int r = __ffs(mm) - 1;
              mm &= mm - 1u;
              s_ent[r < r_split ? pa++ : pb++] = (uint16_t)((cell << 5) | r);
            }
          }
          __syncthreads();
          for (int e = t; e < gT; e += kChunk) {
            const int ent = s_ent[e];
            const int ec = ent >> 5, k = 32 * q + (ent & 31);
            const float4 ch4 = s_mh[ec], cl4 = s_ml[ec], nh4 = s_eh[k], nl4 = s_el[k];
            const float ch[3] = {ch4.x, ch4.y, ch4.z}, cl[3] = {cl4.x, cl4.y, cl4.z};
            const float nh[3] = {nh4.x, nh4.y, nh4.z}, nl[3] = {nl4.x, nl4.y, nl4.z};
            const float wgt = pair_weight(ch, cl, nh, nl, pp.k_hi, pp.k_lo);
            const int64_t pos = ebase + erun + g0 + e;
            ent_ck[pos] = (uint16_t)tile_off(ec, s_loc[k]);
            ent_w[pos] = wgt;
            const uint32_t pab = s_pab[q][ec];
            s_w[e + (int)(int16_t)(e < totA ? pab & 0xffffu : pab >> 16)] = wgt;
          }
          __syncthreads();
        }
        add_span();
        erun += total;
      }
      kcount += ucount;
      __syncthreads();
    }
  }
  if (active) {
    wsum[m] = wsv.value();
    wsum[pp.M + m] = w16 * (1.0f / kTcWeightScale);
  }
  // Pad the candidate list to a multiple of HG_KPAD with a valid sample index
  // (its weight is zero in every cell); empty sub-chunks and the end
  // sentinel point at the block's end.
  const int64_t padded = (kcount + HG_KPAD - 1) / HG_KPAD * HG_KPAD;
  const int32_t filler = kcount > 0 ? cand_idx[cbase] : 0;
  for (int64_t i = kcount + t; i < padded; i += kChunk) cand_idx[cbase + i] = filler;
  for (int64_t j = (kcount + 31) / 32 + t; j <= padded / 32; j += kChunk)
    sub_off[sbase + j] = ebase + erun;
  if (t == 0) {
    cand_cnt[b] = (int32_t)padded;
    atomicAdd(&totals[0], (unsigned long long)erun);
    atomicAdd(&totals[1], (unsigned long long)padded);
  }
}

// Upper bounds per block, for the slot and entry ranges the pair kernel fills:
// candidates <= the samples of the block's bin window (+ HG_KPAD padding + one
// sub-chunk for the end sentinel); pairs <= sum over the block's cells of the
// samples in each cell's own bin window (the bins that can hold a sample
// within R of the cell, the same construction as the block window).
struct BoundParams {
  int32_t nx, ny, nbx_b, nbx, nby, bin_cells, padx, pady;
  int32_t sfl;  // 1: Sanson-Flamsteed map (x-ranges of sfl_xrange)
  double lon0, lat0, dlat, dlon, R_deg, sinR, eps_px;
};

template <bool kHpx>
__global__ void __launch_bounds__(kChunk)
    k_block_bounds(BoundParams bp, WinArgs wa, const int32_t* __restrict__ bin_off,
                   int64_t* __restrict__ slots_ub, int64_t* __restrict__ pairs_ub) {
  __shared__ long long s_sum[kChunk / 32];
  __shared__ double s_H[HG_BY];  // RA half-width H of the block's rows (FP64, once per row)
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int b = blockIdx.x;
  const int bbx = b % bp.nbx_b, bby = b / bp.nbx_b;
  const int ix = bbx * HG_BX + (t % HG_BX), iy = bby * HG_BY + (t / HG_BX);
  if (t < HG_BY) {
    const double lat = bp.lat0 + ((double)(bby * HG_BY + t) - 0.5 * (bp.ny - 1)) * bp.dlat;
    s_H[t] = asin(bp.sinR / cos(fabs(lat) * kDeg)) / kDeg;
  }
  __syncthreads();
  long long cnt = 0;
  if (ix < bp.nx && iy < bp.ny) {
    const double lat = bp.lat0 + ((double)iy - 0.5 * (bp.ny - 1)) * bp.dlat;
    const double H = s_H[t / HG_BX];
    if constexpr (kHpx) {
      // the cell's own window: rings that can hold a point within R of the
      // cell, RA within H of it (FP32; the two-pixel and two-ring margins of
      // the window cover its rounding)
      const HpxParams& hp = wa.hp;
      const double lon = bp.lon0 + ((double)ix - 0.5 * (bp.nx - 1)) * bp.dlon;
      const float z_lo = sinf((float)((lat - bp.R_deg) * kDeg));
      const float z_hi = sinf((float)((lat + bp.R_deg) * kDeg));
      const int r0 = max(hp.ring0, (int)floorf(hpx_rho_f(hp.nside, z_hi)) - 2);
      const int r1 = min(hp.ring0 + hp.n_rings - 1, (int)ceilf(hpx_rho_f(hp.nside, z_lo)) + 2);
      const HWin h = {r0, r1, (float)(lon - H) - 1e-4f, (float)(lon + H) + 1e-4f};
      for (int r = r0; r <= r1; ++r) {
        int32_t lo, hi;
        window_row<true>(wa, bin_off, bp.nbx, r, make_int4(0, 0, 0, 0), h, lo, hi);
        cnt += hi - lo;
      }
    } else {
      const double qy_lo = iy + bp.pady + 0.5 - bp.R_deg / bp.dlat - bp.eps_px;
      const double qy_hi = iy + bp.pady + 0.5 + bp.R_deg / bp.dlat + bp.eps_px;
      double qx_lo = ix + bp.padx + 0.5 - H / bp.dlon - bp.eps_px;
      double qx_hi = ix + bp.padx + 0.5 + H / bp.dlon + bp.eps_px;
      if (bp.sfl) {
        const double xc = ((double)ix - 0.5 * (bp.nx - 1)) * bp.dlon;
        double xl, xh;
        sfl_xrange(xc / cos(lat * kDeg), lat, bp.R_deg, bp.sinR, xl, xh);
        qx_lo = xl / bp.dlon + 0.5 * bp.nx + bp.padx - bp.eps_px;
        qx_hi = xh / bp.dlon + 0.5 * bp.nx + bp.padx + bp.eps_px;
      }
      const int B = bp.bin_cells;
      const int by0 = max(0, (int)floor(qy_lo) / B), by1 = min(bp.nby - 1, (int)floor(qy_hi) / B);
      const int bx0 = max(0, (int)floor(qx_lo) / B), bx1 = min(bp.nbx - 1, (int)floor(qx_hi) / B);
      for (int by = by0; by <= by1; ++by)
        cnt += bin_off[(int64_t)by * bp.nbx + bx1 + 1] - bin_off[(int64_t)by * bp.nbx + bx0];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) s_sum[wid] = cnt;
  __syncthreads();
  if (t == 0) {
    long long tot = 0;
    for (int w = 0; w < kChunk / 32; ++w) tot += s_sum[w];
    pairs_ub[b] = tot;
    long long ws = 0;
    int4 wb = make_int4(1, 0, 0, 0);
    HWin hb = {1, 0, 0.0f, 0.0f};
    if constexpr (kHpx)
      hb = wa.hwin[b];
    else
      wb = wa.win[b];
    for (int row = kHpx ? hb.r0 : wb.x; row <= (kHpx ? hb.r1 : wb.y); ++row) {
      int32_t lo, hi;
      window_row<kHpx>(wa, bin_off, bp.nbx, row, wb, hb, lo, hi);
      ws += hi - lo;
    }
    slots_ub[b] = (ws + HG_KPAD - 1) / HG_KPAD * HG_KPAD + HG_KPAD;
  }
}

// Device memory of plans comes from a library-owned, stream-ordered pool per
// device whose release threshold keeps freed blocks for reuse, so repeated plan
// creation does not pay for cudaMalloc/cudaFree.
cudaMemPool_t plan_pool() {
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
  }
  return pools[dev];
}

}  // namespace

cudaError_t pool_alloc(void** p, size_t sz, cudaStream_t st) {
  if (fault_hit(kFaultAlloc)) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  cudaMemPool_t pool = plan_pool();
  if (!pool) return cudaMalloc(p, sz);
  return cudaMallocFromPoolAsync(p, sz, pool, st);
}

namespace {

template <typename T>
static cudaError_t dmalloc(T** p, int64_t n, int64_t* bytes, cudaStream_t st) {
  size_t sz = (size_t)std::max<int64_t>(n, 1) * sizeof(T);
  *bytes += (int64_t)sz;
  return pool_alloc((void**)p, sz, st);
}

}  // namespace

void free_plan_arrays(hegrid_plan* p, cudaStream_t st) {
  void* arrays[] = {p->perm,   p->bin_off, p->cand_off, p->blk_pair_off, p->cand_cnt, p->cand_idx,
                    p->sub_off, p->ent_ck,  p->ent_w,    p->wsum,         p->totals,   p->err_word,
                    p->wtiles};
  for (void* a : arrays)
    if (a) cudaFreeAsync(a, st);
}

// Temporary device buffers of plan_create, released (stream-ordered) on every
// exit path.
struct Scratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s) : st(s) {}
  ~Scratch() {
    for (void* q : ptrs) cudaFreeAsync(q, st);
  }
  template <typename T>
  cudaError_t get(T** p, int64_t n) {
    size_t sz = (size_t)std::max<int64_t>(n, 1) * sizeof(T);
    cudaError_t e = pool_alloc((void**)p, sz, st);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};

// HEALPix-variant layout (host, FP64): the rings that can hold a sample
// within R of a cell (two rings of margin beyond the continuous ring
// coordinate of the padded latitude band) and, in each, the pixels whose
// centres lie within two pixels of the map's RA range widened by Hmax.
// Single IEEE operations apart from products by powers of two, so that any
// contraction leaves the table unchanged.
double hpx_rho(int32_t N, double z) {
  const double Nd = (double)N;
  if (z > 2.0 / 3.0) return Nd * std::sqrt(3.0 * (1.0 - z));
  if (z < -2.0 / 3.0) return 4.0 * Nd - Nd * std::sqrt(3.0 * (1.0 + z));
  return 2.0 * Nd - (3.0 * Nd * z) / 2.0;
}

int64_t hpx_layout(const hegrid_map_geom& g, double R_deg, double R_rad, int32_t N,
                   int32_t* ring0, std::vector<HpxRing>* rings) {
  const double half_rows = 0.5 * (double)(g.ny - 1) * g.dlat_deg;
  const double half_cols = 0.5 * (double)(g.nx - 1) * g.dlon_deg;
  const double lat_lo = g.lat0_deg - half_rows, lat_hi = g.lat0_deg + half_rows;
  const double lat_max = std::max(std::fabs(lat_lo), std::fabs(lat_hi));
  const double Hmax = std::asin(std::sin(R_rad) / std::cos(lat_max * kDeg)) / kDeg;
  const double pa = (g.lon0_deg - half_cols) - Hmax, pb = (g.lon0_deg + half_cols) + Hmax;
  if (pb - pa >= 360.0) return -1;
  const double z0 = std::sin((lat_lo - R_deg) * kDeg), z1 = std::sin((lat_hi + R_deg) * kDeg);
  const int64_t i0 = std::max<int64_t>(1, (int64_t)std::floor(hpx_rho(N, z1)) - 2);
  const int64_t i1 = std::min<int64_t>(4 * (int64_t)N - 1, (int64_t)std::ceil(hpx_rho(N, z0)) + 2);
  int64_t total = 0;
  rings->clear();
  for (int64_t i = i0; i <= i1; ++i) {
    HpxRing e;
    if (i < N) {
      e.n = (int32_t)(4 * i);
      e.half = 1;
    } else if (i > 3 * (int64_t)N) {
      e.n = (int32_t)(4 * (4 * (int64_t)N - i));
      e.half = 1;
    } else {
      e.n = 4 * N;
      e.half = (int32_t)((i - N + 1) & 1);
    }
    const double ua = (pa * (double)e.n) / 360.0 - 0.5 * (double)e.half;
    const double ub = (pb * (double)e.n) / 360.0 - 0.5 * (double)e.half;
    int64_t J0 = (int64_t)std::ceil(ua - 2.0), J1 = (int64_t)std::floor(ub + 2.0);
    int64_t cnt = J1 - J0 + 1;
    if (cnt >= e.n) {
      cnt = e.n;
      J0 = 0;
    }
    e.J0 = (int32_t)J0;
    e.cnt = (int32_t)cnt;
    e.base = total;
    total += cnt;
    rings->push_back(e);
  }
  *ring0 = (int32_t)i0;
  return total;
}

hegrid_status plan_build(hegrid_plan* p, const double* lon, const double* lat,
                         int coords_on_device, cudaStream_t st, int hpx_log2, bool sfl,
                         bool dense_tiles) {
  const int32_t N = (int32_t)p->N;
  const hegrid_map_geom& g = p->geom;
  Scratch sc(st);

  // --- layout of the padded map (a2) -----------------------------------
  const double half_rows = 0.5 * (double)(g.ny - 1) * g.dlat_deg;
  const double lat_max = std::max(std::fabs(g.lat0_deg - half_rows), std::fabs(g.lat0_deg + half_rows));
  if (lat_max + p->R_deg >= 90.0) {
    set_error("map rows come within R of a pole");
    return HEGRID_ERR_UNSUPPORTED;
  }
  const double Hmax = std::asin(std::sin(p->R_rad) / std::cos(lat_max * kDeg)) / kDeg;
  p->pady = (int32_t)std::ceil(p->R_deg / g.dlat_deg) + 1;
  p->padx = (int32_t)std::ceil(Hmax / g.dlon_deg) + 1;
  // Sanson-Flamsteed: per row, the x-ranges of the first and last cells'
  // R-discs (sfl_xrange) set the padding (the oracle's arithmetic)
  std::vector<double> row_ce;  // cos(lat) of each cell row (SFL)
  const double sinR = std::sin(p->R_rad);
  if (sfl) {
    const double xe = 0.5 * (double)(g.nx - 1) * g.dlon_deg;
    double ex = 0.0;
    row_ce.resize(g.ny);
    for (int32_t iy = 0; iy < g.ny; ++iy) {
      const double la = g.lat0_deg + ((double)iy - 0.5 * (double)(g.ny - 1)) * g.dlat_deg;
      const double ce = std::cos(la * kDeg);
      row_ce[iy] = ce;
      double lo, hi;
      sfl_xrange(-xe / ce, la, p->R_deg, sinR, lo, hi);
      ex = std::max(ex, -xe - lo);
      sfl_xrange(xe / ce, la, p->R_deg, sinR, lo, hi);
      ex = std::max(ex, hi - xe);
    }
    p->padx = (int32_t)std::ceil(ex / g.dlon_deg) + 1;
    if ((double)(g.nx + 2 * p->padx) * g.dlon_deg / std::cos(lat_max * kDeg) >= 360.0) {
      set_error("padded map is wider than 360 degrees of RA");
      return HEGRID_ERR_UNSUPPORTED;
    }
  }
  if ((double)(g.nx + 2 * p->padx) * g.dlon_deg >= 360.0) {
    set_error("padded map is wider than 360 degrees of RA");
    return HEGRID_ERR_UNSUPPORTED;
  }
  const int B = p->bin_cells;
  p->nbx = (g.nx + 2 * p->padx + B - 1) / B;
  p->nby = (g.ny + 2 * p->pady + B - 1) / B;
  p->n_bins = (int64_t)p->nbx * p->nby;
  // HEALPix variant: the bins are the table's ring pixels instead
  const bool hpx = hpx_log2 > 0;
  const int32_t nside = hpx ? (int32_t)1 << hpx_log2 : 0;
  int32_t ring0 = 0;
  std::vector<HpxRing> hrings;
  if (hpx) {
    p->n_bins = hpx_layout(g, p->R_deg, p->R_rad, nside, &ring0, &hrings);
    if (p->n_bins < 0) {
      set_error("padded map is wider than 360 degrees of RA");
      return HEGRID_ERR_UNSUPPORTED;
    }
  }
  if (p->n_bins >= (int64_t)0x7fffffff) {
    set_error("too many bins");
    return HEGRID_ERR_UNSUPPORTED;
  }
  p->nbx_b = (g.nx + HG_BX - 1) / HG_BX;
  p->nby_b = (g.ny + HG_BY - 1) / HG_BY;
  p->n_blocks = (int64_t)p->nbx_b * p->nby_b;

  // --- coordinates on the device ---------------------------------------
  const double* dlon = lon;
  const double* dlat = lat;
  if (!coords_on_device) {
    double *a, *b;
    HG_CUDA_TRY(sc.get(&a, N));
    HG_CUDA_TRY(sc.get(&b, N));
    HG_CUDA_TRY(cudaMemcpyAsync(a, lon, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    HG_CUDA_TRY(cudaMemcpyAsync(b, lat, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    dlon = a;
    dlat = b;
  }

  // --- a1 + a2 ------------------------------------------------------------
  uint32_t *key0, *key1;
  int32_t *val0, *val1;
  double *sx, *sy, *sz;
  HG_CUDA_TRY(sc.get(&key0, N));
  HG_CUDA_TRY(sc.get(&key1, N));
  HG_CUDA_TRY(sc.get(&val0, N));
  HG_CUDA_TRY(sc.get(&val1, N));
  HG_CUDA_TRY(sc.get(&sx, N));
  HG_CUDA_TRY(sc.get(&sy, N));
  HG_CUDA_TRY(sc.get(&sz, N));
  KeyParams kp;
  kp.lon0 = g.lon0_deg;
  kp.lat0 = g.lat0_deg;
  kp.dlon = g.dlon_deg;
  kp.dlat = g.dlat_deg;
  kp.rdlon = 1.0 / g.dlon_deg;
  kp.rdlat = 1.0 / g.dlat_deg;
  kp.cx = 0.5 * (double)g.nx + (double)p->padx;
  kp.cy = 0.5 * (double)g.ny + (double)p->pady;
  kp.wx = (double)(g.nx + 2 * p->padx);
  kp.wy = (double)(g.ny + 2 * p->pady);
  kp.bin_cells = B;
  kp.nbx = p->nbx;
  kp.n_bins = (uint32_t)p->n_bins;
  kp.sfl = sfl ? 1 : 0;
  HpxParams hp;
  hp.nside = nside;
  hp.ring0 = ring0;
  hp.n_rings = (int32_t)hrings.size();
  hp.n_bins = (uint32_t)p->n_bins;
  hp.rings = nullptr;
  if (hpx) {
    HpxRing* dr;
    HG_CUDA_TRY(sc.get(&dr, (int64_t)hrings.size()));
    HG_CUDA_TRY(cudaMemcpyAsync(dr, hrings.data(), sizeof(HpxRing) * hrings.size(),
                                cudaMemcpyHostToDevice, st));
    hp.rings = dr;
    k_prep<true><<<(N + 255) / 256, 256, 0, st>>>(N, dlon, dlat, kp, hp, key0, val0);
  } else {
    k_prep<false><<<(N + 255) / 256, 256, 0, st>>>(N, dlon, dlat, kp, hp, key0, val0);
  }
  count_launch();
  HG_CUDA_TRY(launch_status());

  // --- a3: radix sort ------------------------------------------------------
  int bits = 1;
  while (((uint64_t)1 << bits) <= (uint64_t)p->n_bins) ++bits;
  const int passes = (bits + 7) / 8;
  const int32_t n_tiles = (N + kSortTile - 1) / kSortTile;
  const int64_t hist_n = (int64_t)256 * n_tiles;
  int32_t *hist, *hoff, *stmp32;
  HG_CUDA_TRY(sc.get(&hist, hist_n));
  HG_CUDA_TRY(sc.get(&hoff, hist_n + 1));
  HG_CUDA_TRY(sc.get(&stmp32, scan_tmp_elems(hist_n) + 8));
  uint32_t *kin = key0, *kout = key1;
  int32_t *vin = val0, *vout = val1;
  for (int ps = 0; ps < passes; ++ps) {
    k_radix_hist<<<n_tiles, kSortThreads, 0, st>>>(kin, N, 8 * ps, n_tiles, hist);
    count_launch();
    scan_exclusive<int32_t, int32_t>(hist, hist_n, hoff, stmp32, st);
    k_radix_scatter<<<n_tiles, kSortThreads, 0, st>>>(kin, vin, kout, vout, N, 8 * ps, n_tiles,
                                                       hoff);
    count_launch();
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  HG_CUDA_TRY(launch_status());
  int64_t bytes = 0;
  HG_CUDA_TRY(dmalloc(&p->perm, N, &bytes, st));
  HG_CUDA_TRY(dmalloc(&p->bin_off, p->n_bins + 1, &bytes, st));
  HG_CUDA_TRY(cudaMemcpyAsync(p->perm, vin, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st));
  k_bin_offsets<<<(N + 255) / 256, 256, 0, st>>>(kin, N, (uint32_t)p->n_bins, p->bin_off);
  count_launch();
  k_unit_sorted<<<(N + 255) / 256, 256, 0, st>>>(p->perm, N, dlon, dlat, sx, sy, sz);
  count_launch();
  HG_CUDA_TRY(launch_status());

  // --- bin windows (host): of each block, and of each warp's 8 x 4 cell
  // tile within it (the bins that can hold a sample within R of a cell of
  // the rectangle; the block's window is the union of its warps') ------------
  std::vector<int4> hwin((size_t)p->n_blocks * 5);
  const double eps_px = 1e-6;
  const double sR = std::sin(p->R_rad);
  // Sanson-Flamsteed: per cell row, the first and last columns' x-ranges
  // (x_lo grows with the column, so a rectangle's extremes are at its ends)
  std::vector<double> row_lat, row_H, row_cmin, row_cmax;
  if (sfl) {
    row_lat.resize(g.ny);
    row_H.resize(g.ny);
    row_cmin.resize(g.ny);
    row_cmax.resize(g.ny);
    for (int32_t iy = 0; iy < g.ny; ++iy) {
      const double la = g.lat0_deg + ((double)iy - 0.5 * (double)(g.ny - 1)) * g.dlat_deg;
      const double c1 = std::cos((la - p->R_deg) * kDeg), c2 = std::cos((la + p->R_deg) * kDeg);
      row_lat[iy] = la;
      row_H[iy] = std::asin(sR / row_ce[iy]) / kDeg;
      row_cmin[iy] = std::min(c1, c2);
      row_cmax[iy] = (la - p->R_deg <= 0.0 && la + p->R_deg >= 0.0) ? 1.0 : std::max(c1, c2);
    }
  }
  auto window = [&](int ix0, int ix1, int iy0, int iy1) -> int4 {
    ix1 = std::min(ix1, g.nx - 1);
    iy1 = std::min(iy1, g.ny - 1);
    if (ix0 > ix1 || iy0 > iy1) return make_int4(1, 0, 1, 0);  // no cells: empty
    double la0 = g.lat0_deg + ((double)iy0 - 0.5 * (g.ny - 1)) * g.dlat_deg;
    double la1 = g.lat0_deg + ((double)iy1 - 0.5 * (g.ny - 1)) * g.dlat_deg;
    double lmax = std::max(std::fabs(la0), std::fabs(la1));
    double Hb = std::asin(sR / std::cos(lmax * kDeg)) / kDeg;
    double qy_lo = iy0 + p->pady + 0.5 - p->R_deg / g.dlat_deg - eps_px;
    double qy_hi = iy1 + p->pady + 0.5 + p->R_deg / g.dlat_deg + eps_px;
    double qx_lo = ix0 + p->padx + 0.5 - Hb / g.dlon_deg - eps_px;
    double qx_hi = ix1 + p->padx + 0.5 + Hb / g.dlon_deg + eps_px;
    if (sfl) {
      const double x0 = ((double)ix0 - 0.5 * (g.nx - 1)) * g.dlon_deg;
      const double x1 = ((double)ix1 - 0.5 * (g.nx - 1)) * g.dlon_deg;
      double xl = INFINITY, xh = -INFINITY;
      for (int iy = iy0; iy <= iy1; ++iy) {
        const double a = x0 / row_ce[iy] - row_H[iy], b = x1 / row_ce[iy] + row_H[iy];
        xl = std::min(xl, a >= 0.0 ? a * row_cmin[iy] : a * row_cmax[iy]);
        xh = std::max(xh, b >= 0.0 ? b * row_cmax[iy] : b * row_cmin[iy]);
      }
      qx_lo = xl / g.dlon_deg + 0.5 * g.nx + p->padx - eps_px;
      qx_hi = xh / g.dlon_deg + 0.5 * g.nx + p->padx + eps_px;
    }
    int by0 = std::max(0, (int)std::floor(qy_lo) / B);
    int by1 = std::min(p->nby - 1, (int)std::floor(qy_hi) / B);
    int bx0 = std::max(0, (int)std::floor(qx_lo) / B);
    int bx1 = std::min(p->nbx - 1, (int)std::floor(qx_hi) / B);
    return make_int4(by0, by1, bx0, bx1);
  };
  for (int64_t b = 0; b < p->n_blocks; ++b) {
    int bbx = (int)(b % p->nbx_b), bby = (int)(b / p->nbx_b);
    int ix0 = bbx * HG_BX, iy0 = bby * HG_BY;
    hwin[b] = window(ix0, ix0 + HG_BX - 1, iy0, iy0 + HG_BY - 1);
    for (int w = 0; w < 4; ++w) {
      int wx0 = ix0 + (w & 1) * 8, wy0 = iy0 + (w >> 1) * 4;
      hwin[p->n_blocks + 4 * b + w] = window(wx0, wx0 + 7, wy0, wy0 + 3);
    }
  }
  int4* dwin;
  HG_CUDA_TRY(sc.get(&dwin, p->n_blocks * 5));
  HG_CUDA_TRY(cudaMemcpyAsync(dwin, hwin.data(), sizeof(int4) * p->n_blocks * 5,
                              cudaMemcpyHostToDevice, st));
  WinArgs wa;
  wa.win = dwin;
  wa.wwin = dwin + p->n_blocks;
  wa.hwin = nullptr;
  wa.hwwin = nullptr;
  wa.hp = hp;
  // HEALPix windows: the same rectangles as rings (two rings of margin beyond
  // the continuous ring coordinate of their latitude band +- R) and an RA
  // range (the cells' RA +- Hb, rounded outwards to FP32)
  double hpx_pad_deg = 0.0;  // widest pixel of the table, for the FP32 error band
  if (hpx) {
    for (const HpxRing& e : hrings) hpx_pad_deg = std::max(hpx_pad_deg, 360.0 / e.n);
    std::vector<HWin> hh((size_t)p->n_blocks * 5);
    const int32_t r_last = ring0 + (int32_t)hrings.size() - 1;
    auto hwindow = [&](int ix0, int ix1, int iy0, int iy1) -> HWin {
      ix1 = std::min(ix1, g.nx - 1);
      iy1 = std::min(iy1, g.ny - 1);
      if (ix0 > ix1 || iy0 > iy1) return HWin{1, 0, 0.0f, 0.0f};  // no cells: empty
      const double la0 = g.lat0_deg + ((double)iy0 - 0.5 * (g.ny - 1)) * g.dlat_deg;
      const double la1 = g.lat0_deg + ((double)iy1 - 0.5 * (g.ny - 1)) * g.dlat_deg;
      const double lmax = std::max(std::fabs(la0), std::fabs(la1));
      const double Hb = std::asin(sR / std::cos(lmax * kDeg)) / kDeg;
      const double pa = g.lon0_deg + ((double)ix0 - 0.5 * (g.nx - 1)) * g.dlon_deg - Hb;
      const double pb = g.lon0_deg + ((double)ix1 - 0.5 * (g.nx - 1)) * g.dlon_deg + Hb;
      const double zl = std::sin((la0 - p->R_deg) * kDeg), zh = std::sin((la1 + p->R_deg) * kDeg);
      HWin h;
      h.r0 = std::max(ring0, (int32_t)std::floor(hpx_rho(nside, zh)) - 2);
      h.r1 = std::min(r_last, (int32_t)std::ceil(hpx_rho(nside, zl)) + 2);
      h.pa = std::nextafter((float)pa, -INFINITY);
      h.pb = std::nextafter((float)pb, INFINITY);
      return h;
    };
    for (int64_t b = 0; b < p->n_blocks; ++b) {
      int bbx = (int)(b % p->nbx_b), bby = (int)(b / p->nbx_b);
      int ix0 = bbx * HG_BX, iy0 = bby * HG_BY;
      hh[b] = hwindow(ix0, ix0 + HG_BX - 1, iy0, iy0 + HG_BY - 1);
      for (int w = 0; w < 4; ++w) {
        int wx0 = ix0 + (w & 1) * 8, wy0 = iy0 + (w >> 1) * 4;
        hh[p->n_blocks + 4 * b + w] = hwindow(wx0, wx0 + 7, wy0, wy0 + 3);
      }
    }
    HWin* dh;
    HG_CUDA_TRY(sc.get(&dh, p->n_blocks * 5));
    HG_CUDA_TRY(cudaMemcpyAsync(dh, hh.data(), sizeof(HWin) * p->n_blocks * 5,
                                cudaMemcpyHostToDevice, st));
    wa.hwin = dh;
    wa.hwwin = dh + p->n_blocks;
  }

  // --- a4 parameters -------------------------------------------------------
  PairParams pp;
  pp.nx = g.nx;
  pp.ny = g.ny;
  pp.M = p->M;
  pp.nbx_b = p->nbx_b;
  pp.nbx = p->nbx;
  pp.sfl = sfl ? 1 : 0;
  pp.lon0 = g.lon0_deg;
  pp.lat0 = g.lat0_deg;
  pp.dlon = g.dlon_deg;
  pp.dlat = g.dlat_deg;
  {
    double s = std::sin(0.5 * p->R_rad);
    pp.cR2 = 4.0 * s * s;
    // Error band of the FP32 test (relative to c_R^2).  With E the largest
    // |u - u_block| in the window and c the chord, the FP32 chord^2 from the
    // rounded block-local coordinates is within 2^-24 (7 E/c + 8) of the exact
    // value; the band is 2^-20 (8 + 8 E/c), 16x wider.
    double cR = 2.0 * s;
    double wx_cells = HG_BX + 2.0 * (Hmax / g.dlon_deg + 2.0 * B + 1.0);
    double wy_cells = HG_BY + 2.0 * (p->R_deg / g.dlat_deg + 2.0 * B + 1.0);
    if (sfl)  // the padding bounds the sheared discs' x-excess
      wx_cells = HG_BX + 2.0 * (p->padx + 2.0 * B + 1.0);
    if (hpx) {  // windows widened by up to two pixels and three rings each side
      wx_cells = HG_BX + 2.0 * ((Hmax + 4.0 * hpx_pad_deg) / g.dlon_deg + 1.0);
      wy_cells = HG_BY + 2.0 * ((p->R_deg + 4.0 * hpx_pad_deg) / g.dlat_deg + 1.0);
    }
    double E = 0.5 * std::sqrt(wx_cells * wx_cells * g.dlon_deg * g.dlon_deg +
                               wy_cells * wy_cells * g.dlat_deg * g.dlat_deg) * kDeg;
    double band = std::ldexp(8.0 + 8.0 * E / cR, -20);
    pp.lo_thr = std::nextafter((float)(pp.cR2 * (1.0 - band)), 0.0f);
    pp.hi_thr = std::nextafter((float)(pp.cR2 * (1.0 + band)), 1.0f);
    double k = 1.0 / (2.0 * p->sigma_rad * p->sigma_rad);
    pp.k_hi = (float)k;
    pp.k_lo = (float)(k - (double)pp.k_hi);
  }
  // --- a4 upper bounds: slot and entry ranges per block ---------------------
  int64_t *slots_ub, *pairs_ub;
  HG_CUDA_TRY(sc.get(&slots_ub, p->n_blocks + 1));
  HG_CUDA_TRY(sc.get(&pairs_ub, p->n_blocks + 1));
  HG_CUDA_TRY(cudaMemsetAsync(slots_ub + p->n_blocks, 0, sizeof(int64_t), st));
  HG_CUDA_TRY(cudaMemsetAsync(pairs_ub + p->n_blocks, 0, sizeof(int64_t), st));
  {
    BoundParams bp;
    bp.nx = g.nx;
    bp.ny = g.ny;
    bp.nbx_b = p->nbx_b;
    bp.nbx = p->nbx;
    bp.nby = p->nby;
    bp.bin_cells = B;
    bp.padx = p->padx;
    bp.pady = p->pady;
    bp.sfl = sfl ? 1 : 0;
    bp.lon0 = g.lon0_deg;
    bp.lat0 = g.lat0_deg;
    bp.dlat = g.dlat_deg;
    bp.dlon = g.dlon_deg;
    bp.R_deg = p->R_deg;
    bp.sinR = sR;
    bp.eps_px = eps_px;
    if (hpx)
      k_block_bounds<true><<<(unsigned)p->n_blocks, kChunk, 0, st>>>(bp, wa, p->bin_off,
                                                                     slots_ub, pairs_ub);
    else
      k_block_bounds<false><<<(unsigned)p->n_blocks, kChunk, 0, st>>>(bp, wa, p->bin_off,
                                                                      slots_ub, pairs_ub);
    count_launch();
  }
  int64_t* stmp64;
  HG_CUDA_TRY(sc.get(&stmp64, scan_tmp_elems(p->n_blocks + 1) + 8));
  HG_CUDA_TRY(dmalloc(&p->cand_off, p->n_blocks + 1, &bytes, st));
  HG_CUDA_TRY(dmalloc(&p->blk_pair_off, p->n_blocks + 1, &bytes, st));
  // exclusive scans over n+1 entries (last input 0): out[n] is the total
  scan_exclusive<int64_t, int64_t>(slots_ub, p->n_blocks + 1, p->cand_off, stmp64, st);
  scan_exclusive<int64_t, int64_t>(pairs_ub, p->n_blocks + 1, p->blk_pair_off, stmp64, st);
  HG_CUDA_TRY(launch_status());

  // The one host round trip of plan creation: the bounds' totals size the
  // candidate-slot and entry arrays.
  int64_t totals[2];
  HG_CUDA_TRY(cudaMemcpyAsync(&totals[0], p->blk_pair_off + p->n_blocks, sizeof(int64_t),
                              cudaMemcpyDeviceToHost, st));
  HG_CUDA_TRY(cudaMemcpyAsync(&totals[1], p->cand_off + p->n_blocks, sizeof(int64_t),
                              cudaMemcpyDeviceToHost, st));
  HG_CUDA_TRY(cudaStreamSynchronize(st));
  p->P_ub = totals[0];
  p->slots = totals[1];
  if (p->slots > (int64_t)0x7fffffff) {
    set_error("too many candidate slots");
    return HEGRID_ERR_UNSUPPORTED;
  }

  // --- a4 fill + a5 weights ------------------------------------------------
  const int64_t n_sub = p->slots / 32;
  // (+16 bytes: the tensor-core kernel stages entries in 16-byte aligned
  // windows that may reach past the last entry)
  HG_CUDA_TRY(dmalloc(&p->ent_ck, p->P_ub + 8, &bytes, st));
  HG_CUDA_TRY(dmalloc(&p->ent_w, p->P_ub + 4, &bytes, st));
  HG_CUDA_TRY(dmalloc(&p->sub_off, n_sub + 1, &bytes, st));
  HG_CUDA_TRY(dmalloc(&p->wsum, kWsumVariants * p->M, &bytes, st));
  HG_CUDA_TRY(dmalloc(&p->cand_idx, p->slots, &bytes, st));
  HG_CUDA_TRY(dmalloc(&p->cand_cnt, p->n_blocks, &bytes, st));
  HG_CUDA_TRY(dmalloc(&p->totals, 2, &bytes, st));
  HG_CUDA_TRY(dmalloc(&p->err_word, 4, &bytes, st));
  HG_CUDA_TRY(cudaMemsetAsync(p->err_word, 0, 4 * sizeof(int32_t), st));
  HG_CUDA_TRY(cudaMemsetAsync(p->totals, 0, 2 * sizeof(unsigned long long), st));
  HG_CUDA_TRY(cudaMemsetAsync(p->wsum, 0, sizeof(float) * kWsumVariants * p->M, st));
  auto pairs = [&](int32_t blk0, int32_t nb, cudaStream_t s) -> hegrid_status {
    if (nb <= 0) return HEGRID_OK;
    if (hpx)
      k_block_pairs<true><<<(unsigned)nb, kChunk, 0, s>>>(
          pp, wa, p->bin_off, p->perm, sx, sy, sz, p->cand_off, p->blk_pair_off, p->cand_cnt,
          p->cand_idx, p->sub_off, p->ent_ck, p->ent_w, p->wsum, p->totals, blk0);
    else
      k_block_pairs<false><<<(unsigned)nb, kChunk, 0, s>>>(
          pp, wa, p->bin_off, p->perm, sx, sy, sz, p->cand_off, p->blk_pair_off, p->cand_cnt,
          p->cand_idx, p->sub_off, p->ent_ck, p->ent_w, p->wsum, p->totals, blk0);
    count_launch();
    HG_CUDA_TRY(launch_status());
    return HEGRID_OK;
  };
  const int32_t nblk = (int32_t)p->n_blocks;
  if (!dense_tiles) {
    hegrid_status e = pairs(0, nblk, st);
    if (e != HEGRID_OK) return e;
  } else {
    // The dense weight tiles (HEGRID_PLAN_DENSE_TILES): the blocks in two
    // halves, each half's pair kernel and then its tile build on a stream of
    // its own.  The halves' pair kernels share the GPU, the first finishes
    // first, and its (memory-bound) tile build runs in the second's last wave.
    HG_CUDA_TRY(dmalloc(&p->wtiles, tcm_wtile_bytes(p->slots), &bytes, st));
    cudaStream_t s2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    auto release = [&]() {
      if (fork) cudaEventDestroy(fork);
      if (join) cudaEventDestroy(join);
      if (s2) cudaStreamDestroy(s2);  // its resources go once its work is done
    };
    cudaError_t ce = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventRecord(fork, st);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s2, fork, 0);
    if (ce != cudaSuccess) {
      release();
      set_error(std::string("plan_create: ") + cudaGetErrorString(ce));
      return HEGRID_ERR_CUDA;
    }
    const int32_t half = (nblk + 1) / 2;
    const PlanView v = p->view();
    hegrid_status e = pairs(0, half, st);
    if (e == HEGRID_OK) e = pairs(half, nblk - half, s2);
    if (e == HEGRID_OK) e = launch_build_wtiles(v, p->wtiles, st, 0, half);
    if (e == HEGRID_OK) e = launch_build_wtiles(v, p->wtiles, s2, half, nblk - half);
    // st waits for s2's work even after a failed launch, so that the caller's
    // synchronisation of st covers every kernel this call issued
    ce = cudaEventRecord(join, s2);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, join, 0);
    if (ce != cudaSuccess && e == HEGRID_OK) {
      set_error(std::string("plan_create: ") + cudaGetErrorString(ce));
      e = HEGRID_ERR_CUDA;
    }
    release();
    if (e != HEGRID_OK) return e;
  }
  p->P = -1;  // exact totals: read on first use (plan_totals)
  HG_CUDA_TRY(cudaEventCreateWithFlags(&p->ready, cudaEventDisableTiming));
  HG_CUDA_TRY(cudaEventRecord(p->ready, st));
  // scratch is released by ~Scratch, ordered after these kernels on `st`
  p->bytes = bytes;
  return HEGRID_OK;
}

}  // namespace hg

// ===========================================================================
// C ABI: plan lifetime, info, export
// ===========================================================================
extern "C" {

const char* hegrid_last_error(void) { return hg::last_error(); }

int64_t hegrid_launch_count(void) { return hg::launch_count(); }

hegrid_status hegrid_pool_usage(int64_t* used_bytes, int64_t* reserved_bytes) {
  hg::set_error("");
  HG_ARG_CHECK(used_bytes != nullptr || reserved_bytes != nullptr, "both outputs are NULL");
  cudaMemPool_t pool = hg::plan_pool();
  if (!pool) {
    hg::set_error("the library's memory pool could not be created on this device");
    return HEGRID_ERR_CUDA;
  }
  uint64_t used = 0, reserved = 0;
  HG_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  HG_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
  if (used_bytes) *used_bytes = (int64_t)used;
  if (reserved_bytes) *reserved_bytes = (int64_t)reserved;
  return HEGRID_OK;
}

hegrid_status hegrid_plan_create(hegrid_plan** out, int64_t n_samples, const double* lon_deg,
                                 const double* lat_deg, int coords_on_device,
                                 const hegrid_map_geom* geom, const hegrid_kernel* kern,
                                 uint32_t flags, void* stream) {
  hg::set_error("");
  HG_ARG_CHECK(out != nullptr, "out is NULL");
  *out = nullptr;
  HG_ARG_CHECK(lon_deg && lat_deg && geom && kern, "NULL coordinates, geometry or kernel");
  HG_ARG_CHECK(n_samples >= 1 && n_samples < (int64_t)0x7fffffff, "n_samples out of [1, 2^31)");
  HG_ARG_CHECK(geom->nx >= 1 && geom->ny >= 1, "nx, ny must be >= 1");
  HG_ARG_CHECK((int64_t)geom->nx * geom->ny < ((int64_t)1 << 40), "map too large");
  HG_ARG_CHECK(geom->dlon_deg > 0 && geom->dlat_deg > 0, "cell size must be > 0");
  HG_ARG_CHECK(std::isfinite(geom->lon0_deg) && std::isfinite(geom->lat0_deg),
               "map centre must be finite");
  HG_ARG_CHECK(kern->fwhm_deg > 0 && kern->support_sigmas > 0, "FWHM and support must be > 0");
  uint32_t bc = flags & 0xffu;
  const int hpx_log2 = (int)((flags >> 8) & 0x1fu);
  const bool sfl = (flags & HEGRID_PLAN_SFL) != 0;
  const bool dense_tiles = (flags & HEGRID_PLAN_DENSE_TILES) != 0;
  HG_ARG_CHECK((flags >> 15) == 0, "unknown plan_create flag bits");
  HG_ARG_CHECK(hpx_log2 <= 13, "HEALPix nside above 2^13");
  HG_ARG_CHECK(!(sfl && hpx_log2 > 0), "HEALPix binning works on the plain grid only");
  hegrid_plan* p = new hegrid_plan();
  std::memset(p, 0, sizeof(*p));
  p->geom = *geom;
  p->kern = *kern;
  cudaGetDevice(&p->device);
  p->N = n_samples;
  p->M = (int64_t)geom->nx * geom->ny;
  p->bin_cells = bc ? (int32_t)bc : 2;
  double sigma_deg = kern->fwhm_deg / std::sqrt(8.0 * std::log(2.0));
  p->sigma_rad = sigma_deg * hg::kDeg;
  p->R_deg = kern->support_sigmas * sigma_deg;
  p->R_rad = p->R_deg * hg::kDeg;
  if (p->R_deg > 11.0) {
    delete p;
    hg::set_error("kernel radius above 11 degrees is not supported");
    return HEGRID_ERR_UNSUPPORTED;
  }
  hegrid_status s =
      hg::plan_build(p, lon_deg, lat_deg, coords_on_device, (cudaStream_t)stream, hpx_log2, sfl,
                     dense_tiles);
  if (s != HEGRID_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    hg::free_plan_arrays(p, (cudaStream_t)stream);
    cudaStreamSynchronize((cudaStream_t)stream);
    if (p->ready) cudaEventDestroy(p->ready);
    delete p;
    return s;
  }
  *out = p;
  return HEGRID_OK;
}

hegrid_status hegrid_plan_destroy(hegrid_plan* plan) {
  if (!plan) return HEGRID_OK;
  cudaDeviceSynchronize();
  hg::free_plan_arrays(plan, nullptr);
  cudaStreamSynchronize(nullptr);
  if (plan->ready) cudaEventDestroy(plan->ready);
  delete plan;
  return HEGRID_OK;
}

// Exact pairs and used candidate slots, counted by the pair kernel (waits for
// the plan to be built).
static hegrid_status plan_totals(const hegrid_plan* plan, int64_t* P, int64_t* n_cand) {
  HG_CUDA_TRY(cudaEventSynchronize(plan->ready));
  unsigned long long t[2];
  HG_CUDA_TRY(cudaMemcpy(t, plan->totals, sizeof(t), cudaMemcpyDeviceToHost));
  *P = (int64_t)t[0];
  *n_cand = (int64_t)t[1];
  return HEGRID_OK;
}

hegrid_status hegrid_plan_info(const hegrid_plan* plan, int64_t* n_pairs, int64_t* n_bins,
                               int64_t* n_blocks, int64_t* n_cand, int64_t* bytes) {
  HG_ARG_CHECK(plan != nullptr, "plan is NULL");
  int64_t P = 0, nc = 0;
  if (n_pairs || n_cand) {
    hegrid_status st = plan_totals(plan, &P, &nc);
    if (st != HEGRID_OK) return st;
  }
  if (n_pairs) *n_pairs = P;
  if (n_bins) *n_bins = plan->n_bins;
  if (n_blocks) *n_blocks = plan->n_blocks;
  if (n_cand) *n_cand = nc;
  if (bytes) *bytes = plan->bytes;
  return HEGRID_OK;
}

hegrid_status hegrid_plan_export(const hegrid_plan* plan, int32_t* perm, int32_t* bin_off,
                                 int64_t* nb_off, int32_t* nb_idx, float* nb_w, float* weight) {
  HG_ARG_CHECK(plan != nullptr, "plan is NULL");
  HG_CUDA_TRY(cudaDeviceSynchronize());
  if (perm)
    HG_CUDA_TRY(cudaMemcpy(perm, plan->perm, sizeof(int32_t) * plan->N, cudaMemcpyDeviceToHost));
  if (bin_off)
    HG_CUDA_TRY(cudaMemcpy(bin_off, plan->bin_off, sizeof(int32_t) * (plan->n_bins + 1),
                           cudaMemcpyDeviceToHost));
  if (weight)
    HG_CUDA_TRY(cudaMemcpy(weight, plan->wsum, sizeof(float) * plan->M, cudaMemcpyDeviceToHost));
  if (nb_off || nb_idx || nb_w) {
    // Rebuild the CSR by cell (rows = cells) from the blocks' sub-chunk entries.
    int64_t P = 0, nc_used = 0;
    hegrid_status st = plan_totals(plan, &P, &nc_used);
    if (st != HEGRID_OK) return st;
    const int64_t nb = plan->n_blocks, ns = plan->slots / 32, M = plan->M, PU = plan->P_ub;
    std::vector<int64_t> coff(nb + 1), soff(ns + 1);
    std::vector<int32_t> cnt(std::max<int64_t>(nb, 1));
    std::vector<int32_t> cidx(std::max<int64_t>(plan->slots, 1));
    std::vector<uint16_t> ck(std::max<int64_t>(PU, 1));
    std::vector<float> w(std::max<int64_t>(PU, 1));
    HG_CUDA_TRY(cudaMemcpy(coff.data(), plan->cand_off, sizeof(int64_t) * (nb + 1),
                           cudaMemcpyDeviceToHost));
    HG_CUDA_TRY(cudaMemcpy(cnt.data(), plan->cand_cnt, sizeof(int32_t) * nb,
                           cudaMemcpyDeviceToHost));
    HG_CUDA_TRY(cudaMemcpy(soff.data(), plan->sub_off, sizeof(int64_t) * (ns + 1),
                           cudaMemcpyDeviceToHost));
    HG_CUDA_TRY(cudaMemcpy(cidx.data(), plan->cand_idx, sizeof(int32_t) * plan->slots,
                           cudaMemcpyDeviceToHost));
    if (PU) {
      HG_CUDA_TRY(cudaMemcpy(ck.data(), plan->ent_ck, sizeof(uint16_t) * PU, cudaMemcpyDeviceToHost));
      HG_CUDA_TRY(cudaMemcpy(w.data(), plan->ent_w, sizeof(float) * PU, cudaMemcpyDeviceToHost));
    }
    const int nx = plan->geom.nx, nbx_b = plan->nbx_b;
    auto cell_of = [&](int64_t b, int col) -> int64_t {
      int64_t bbx = b % nbx_b, bby = b / nbx_b;
      return (bby * HG_BY + col / HG_BX) * (int64_t)nx + bbx * HG_BX + (col % HG_BX);
    };
    std::vector<int64_t> off(M + 1, 0);
    for (int64_t b = 0; b < nb; ++b)
      for (int64_t e = soff[coff[b] / 32]; e < soff[(coff[b] + cnt[b]) / 32]; ++e) {
        int r, k;
        hg::tile_rk(ck[e], r, k);
        off[cell_of(b, r) + 1]++;
      }
    for (int64_t m = 0; m < M; ++m) off[m + 1] += off[m];
    if (off[M] != P) {
      hg::set_error("plan export: entry count does not match the pair total");
      return HEGRID_ERR_CUDA;
    }
    std::vector<int64_t> cur(off.begin(), off.end() - 1);
    std::vector<std::pair<int32_t, float>> pr(std::max<int64_t>(P, 1));
    for (int64_t b = 0; b < nb; ++b) {
      for (int64_t j = coff[b] / 32; j < (coff[b] + cnt[b]) / 32; ++j) {
        const int64_t loc0 = 32 * j - coff[b];
        for (int64_t e = soff[j]; e < soff[j + 1]; ++e) {
          int r, k;
          hg::tile_rk(ck[e], r, k);
          const int64_t m = cell_of(b, r);
          const int64_t loc = loc0 + k;
          pr[cur[m]++] = {cidx[coff[b] + loc], w[e]};
        }
      }
    }
    for (int64_t m = 0; m < M; ++m) std::sort(pr.begin() + off[m], pr.begin() + off[m + 1]);
    if (nb_off) std::memcpy(nb_off, off.data(), sizeof(int64_t) * (M + 1));
    for (int64_t i = 0; i < P; ++i) {
      if (nb_idx) nb_idx[i] = pr[i].first;
      if (nb_w) nb_w[i] = pr[i].second;
    }
  }
  return HEGRID_OK;
}

hegrid_status hegrid_status_poll(const hegrid_plan* plan) {
  HG_ARG_CHECK(plan != nullptr, "plan is NULL");
  HG_CUDA_TRY(cudaEventSynchronize(plan->ready));
  int32_t w = 0;
  HG_CUDA_TRY(cudaMemcpy(&w, plan->err_word, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (w != 0) {
    hg::set_error("a bounded device-side wait timed out (error word " + std::to_string(w) + ")");
    return HEGRID_ERR_TIMEOUT;
  }
  return HEGRID_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free bin sort.  The same bin key, stable radix sort and bin
// offsets as plan creation, for callers that must not allocate device memory:
// the sort's scratch lives in one fixed file-scope device array.
// ===========================================================================
namespace hg {
namespace {

constexpr int64_t kNoAllocMaxSamples = (int64_t)1 << 19;  // 524,288 samples
constexpr int64_t kNoAllocTiles = (kNoAllocMaxSamples + kSortTile - 1) / kSortTile;
constexpr int64_t kNoAllocHist = 256 * kNoAllocTiles;
constexpr int64_t kNoAllocTmp = 64;
// the scan's partial sums, with the plan path's slack of 8 elements
static_assert(kNoAllocTmp >= scan_tmp_elems(kNoAllocHist) + 8, "scratch too small for the scan");
constexpr size_t kOffKey0 = 0;
constexpr size_t kOffKey1 = kOffKey0 + 4 * kNoAllocMaxSamples;
constexpr size_t kOffVal0 = kOffKey1 + 4 * kNoAllocMaxSamples;
constexpr size_t kOffVal1 = kOffVal0 + 4 * kNoAllocMaxSamples;
constexpr size_t kOffHist = kOffVal1 + 4 * kNoAllocMaxSamples;
constexpr size_t kOffHoff = kOffHist + 4 * kNoAllocHist;
constexpr size_t kOffTmp = kOffHoff + (4 * (kNoAllocHist + 1) + 255) / 256 * 256;
constexpr size_t kNoAllocBytes = kOffTmp + 4 * kNoAllocTmp;  // about 8.5 MB

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[64] = {};

// Device address of the scratch array on the current device (set up once per
// device; host code only sees a stand-in symbol, never the device address).
hegrid_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  HG_CUDA_TRY(cudaGetDevice(&dev));
  HG_ARG_CHECK(dev >= 0 && dev < 64, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    HG_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return HEGRID_OK;
}

}  // namespace
}  // namespace hg

extern "C" hegrid_status hegrid_bin_sort_noalloc(int64_t n_samples, const double* lon_deg,
                                                 const double* lat_deg,
                                                 const hegrid_map_geom* geom,
                                                 const hegrid_kernel* kern, uint32_t flags,
                                                 int32_t* perm_out, int32_t* bin_off_out,
                                                 int64_t bin_off_capacity, int64_t* n_bins_out,
                                                 void* stream) {
  using namespace hg;
  set_error("");
  HG_ARG_CHECK(lon_deg && lat_deg && geom && kern, "NULL coordinates, geometry or kernel");
  HG_ARG_CHECK(perm_out && bin_off_out && n_bins_out, "NULL output");
  HG_ARG_CHECK(n_samples >= 1, "n_samples must be >= 1");
  HG_ARG_CHECK(n_samples <= kNoAllocMaxSamples,
               "n_samples above the allocation-free limit of 524288 samples");
  HG_ARG_CHECK(geom->nx >= 1 && geom->ny >= 1, "nx, ny must be >= 1");
  HG_ARG_CHECK(geom->dlon_deg > 0 && geom->dlat_deg > 0, "cell size must be > 0");
  HG_ARG_CHECK(std::isfinite(geom->lon0_deg) && std::isfinite(geom->lat0_deg),
               "map centre must be finite");
  HG_ARG_CHECK(kern->fwhm_deg > 0 && kern->support_sigmas > 0, "FWHM and support must be > 0");
  HG_ARG_CHECK((flags >> 8) == 0,
               "only plain-grid map bins (HEGRID_PLAN_BIN_CELLS) are sorted here: "
               "HEGRID_PLAN_HEALPIX and HEGRID_PLAN_SFL are not");
  const int B = (flags & 0xffu) ? (int)(flags & 0xffu) : 2;
  const double sigma_deg = kern->fwhm_deg / std::sqrt(8.0 * std::log(2.0));
  const double R_deg = kern->support_sigmas * sigma_deg;
  const double R_rad = R_deg * kDeg;
  if (R_deg > 11.0) {
    set_error("kernel radius above 11 degrees is not supported");
    return HEGRID_ERR_UNSUPPORTED;
  }
  // padded-map layout (the bin key's definition)
  const hegrid_map_geom& g = *geom;
  const double half_rows = 0.5 * (double)(g.ny - 1) * g.dlat_deg;
  const double lat_max =
      std::max(std::fabs(g.lat0_deg - half_rows), std::fabs(g.lat0_deg + half_rows));
  if (lat_max + R_deg >= 90.0) {
    set_error("map rows come within R of a pole");
    return HEGRID_ERR_UNSUPPORTED;
  }
  const double Hmax = std::asin(std::sin(R_rad) / std::cos(lat_max * kDeg)) / kDeg;
  const int32_t pady = (int32_t)std::ceil(R_deg / g.dlat_deg) + 1;
  const int32_t padx = (int32_t)std::ceil(Hmax / g.dlon_deg) + 1;
  if ((double)(g.nx + 2 * padx) * g.dlon_deg >= 360.0) {
    set_error("padded map is wider than 360 degrees of RA");
    return HEGRID_ERR_UNSUPPORTED;
  }
  const int32_t nbx = (g.nx + 2 * padx + B - 1) / B;
  const int32_t nby = (g.ny + 2 * pady + B - 1) / B;
  const int64_t n_bins = (int64_t)nbx * nby;
  *n_bins_out = n_bins;
  HG_ARG_CHECK(n_bins < (int64_t)0x7fffffff, "too many bins");
  HG_ARG_CHECK(bin_off_capacity >= n_bins + 1, "bin_off_out holds fewer than n_bins + 1 entries");

  unsigned char* base = nullptr;
  {
    hegrid_status s = noalloc_scratch(&base);
    if (s != HEGRID_OK) return s;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t N = (int32_t)n_samples;
  uint32_t* key0 = reinterpret_cast<uint32_t*>(base + kOffKey0);
  uint32_t* key1 = reinterpret_cast<uint32_t*>(base + kOffKey1);
  int32_t* val0 = reinterpret_cast<int32_t*>(base + kOffVal0);
  int32_t* val1 = reinterpret_cast<int32_t*>(base + kOffVal1);
  int32_t* hist = reinterpret_cast<int32_t*>(base + kOffHist);
  int32_t* hoff = reinterpret_cast<int32_t*>(base + kOffHoff);
  int32_t* tmp = reinterpret_cast<int32_t*>(base + kOffTmp);

  KeyParams kp;
  kp.lon0 = g.lon0_deg;
  kp.lat0 = g.lat0_deg;
  kp.dlon = g.dlon_deg;
  kp.dlat = g.dlat_deg;
  kp.rdlon = 1.0 / g.dlon_deg;
  kp.rdlat = 1.0 / g.dlat_deg;
  kp.cx = 0.5 * (double)g.nx + (double)padx;
  kp.cy = 0.5 * (double)g.ny + (double)pady;
  kp.wx = (double)(g.nx + 2 * padx);
  kp.wy = (double)(g.ny + 2 * pady);
  kp.bin_cells = B;
  kp.nbx = nbx;
  kp.n_bins = (uint32_t)n_bins;
  kp.sfl = 0;
  HpxParams hp;  // unused by the map-bin key
  std::memset(&hp, 0, sizeof(hp));
  k_prep<false><<<(N + 255) / 256, 256, 0, st>>>(N, lon_deg, lat_deg, kp, hp, key0, val0);
  count_launch();
  int bits = 1;
  while (((uint64_t)1 << bits) <= (uint64_t)n_bins) ++bits;
  const int passes = (bits + 7) / 8;
  const int32_t n_tiles = (N + kSortTile - 1) / kSortTile;
  const int64_t hist_n = (int64_t)256 * n_tiles;
  uint32_t *kin = key0, *kout = key1;
  int32_t *vin = val0, *vout = val1;
  for (int ps = 0; ps < passes; ++ps) {
    k_radix_hist<<<n_tiles, kSortThreads, 0, st>>>(kin, N, 8 * ps, n_tiles, hist);
    count_launch();
    scan_exclusive<int32_t, int32_t>(hist, hist_n, hoff, tmp, st);
    k_radix_scatter<<<n_tiles, kSortThreads, 0, st>>>(kin, vin, kout, vout, N, 8 * ps, n_tiles,
                                                       hoff);
    count_launch();
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  HG_CUDA_TRY(launch_status());
  HG_CUDA_TRY(cudaMemcpyAsync(perm_out, vin, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st));
  k_bin_offsets<<<(N + 255) / 256, 256, 0, st>>>(kin, N, (uint32_t)n_bins, bin_off_out);
  count_launch();
  HG_CUDA_TRY(launch_status());
  return HEGRID_OK;
}
