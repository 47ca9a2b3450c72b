// Oracle for convolution-based gridding (HEGrid, arXiv 2207.04584).
//
// TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct CPU
// statement of what the GPU path computes.  Only the tests, the smoke check and
// the timed CPU baseline of the benchmark may load it; the product path never
// does.  It shares no code with the CUDA library and includes none of its
// headers.
//
// Everything is FP64 (the paper fixes no precision).  Sources:
//   * Eq. 1 (Sec. 2.2): V[g] = (1/W) sum_n V[s_n] w(g; s_n), W = sum_n w(g; s_n).
//   * Algorithm 1 (Sec. 4.1.2): a sample contributes to a cell iff d <= R
//     (inclusive).
//   * Sec. 4.1.1: samples are given a spatial key, sorted by it, and a table of
//     key ranges is built.  The GPU path's default key is a bin of the padded
//     target map (og_bin_keys, written from its definition); its HEALPix
//     variant uses the paper's own RING-scheme pixels (og_hpx_*, written from
//     Gorski et al. 2005's definitions) with a per-ring table of pixel ranges.
// Readings where the paper is silent (kernel shape, distance formula, grid
// geometry, empty cells), in short:
//   * w = exp(-d^2 / (2 sigma^2)), sigma = FWHM / sqrt(8 ln 2), R = support*sigma;
//   * d is the great-circle separation; membership is tested on the haversine
//     h = sin^2(dlat/2) + cos(lat_m) cos(lat_n) sin^2(dlon/2) <= sin^2(R/2);
//   * cell (ix, iy) sits at lon0 + (ix - (nx-1)/2) dlon, lat0 + (iy - (ny-1)/2) dlat;
//   * a cell with W = 0 gets map = NaN.
//
// Parity pins: every function here is pinned by tests/test_oracle_pins.py
// (brute force vs indexed, closed forms along a meridian, isolated-sample
// kernel recovery by the chord formula, constant sky, linearity, convexity,
// wrap and permutation invariance, point-source FWHM); the HEALPix functions by
// tests/test_oracle_hpx.py (centre round trip, equal area, ring sizes, named
// pixels, a layout that keeps every neighbour).
//
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -shared -fPIC.
// -ffp-contract=off keeps the bin key arithmetic to single IEEE operations.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <numeric>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

struct og_geom {
  int32_t nx, ny;
  double lon0, lat0;  // map centre, degrees
  double dlon, dlat;  // cell size, degrees
  int32_t proj;       // 0: plain lon/lat grid; 1: Sanson-Flamsteed (x = (lon - lon0) cos lat)
};

struct og_kernel {
  double fwhm_deg;
  double support;  // truncation radius in units of sigma
};

}  // extern "C"

namespace {

const double kPi = 3.14159265358979323846;
const double kDeg = kPi / 180.0;

// Planted-mistake switch for the pin-strength tests: 0 = the oracle as defined.
// Each nonzero value plants one plausible mistake so the tests can show that
// some pin catches it.  Never set outside those tests.
int g_mutation = 0;

struct Derived {
  double sigma_rad, R_rad, R_deg, hR;
};

Derived derive(const og_kernel* k) {
  Derived d;
  double sigma_deg = k->fwhm_deg / std::sqrt(8.0 * std::log(2.0));
  if (g_mutation == 2) sigma_deg = k->fwhm_deg / 2.0;  // wrong FWHM->sigma
  d.sigma_rad = sigma_deg * kDeg;
  d.R_deg = k->support * sigma_deg;
  d.R_rad = d.R_deg * kDeg;
  double s = std::sin(0.5 * d.R_rad);
  d.hR = s * s;
  return d;
}

// Cell centres.  Plain grid: (lon0 + x, lat0 + y).  Sanson-Flamsteed (the
// sinusoidal projection about lon0, a cos(lat)-scaled grid): the cell's
// projected coordinates x = (lon - lon0) cos(lat), y = lat - lat0 lie on the
// regular grid, so lon = lon0 + x / cos(lat).
// x = (ix - (nx-1)/2) dlon, y = (iy - (ny-1)/2) dlat.
void cell_centre(const og_geom* g, int64_t m, double* lon_deg, double* lat_deg) {
  int64_t ix = m % g->nx, iy = m / g->nx;
  if (g_mutation == 4) std::swap(ix, iy);  // transposed cell index
  const double x = ((double)ix - 0.5 * (double)(g->nx - 1)) * g->dlon;
  *lat_deg = g->lat0 + ((double)iy - 0.5 * (double)(g->ny - 1)) * g->dlat;
  double c = std::cos(*lat_deg * kDeg);
  if (g_mutation == 11) c = 1.0;  // projection's cos(lat) dropped
  *lon_deg = g->proj == 1 ? g->lon0 + x / c : g->lon0 + x;
}

// Sanson-Flamsteed: x-range (degrees of projected x) that holds every point
// within R of the cell at RA offset a_c = lon_c - lon0 and latitude lat_c:
// such points have |lon - lon_c| <= H = asin(sin R / cos lat_c) and lat in
// [lat_c - R, lat_c + R], where cos(lat) lies between the cosines of the
// ends (and 1 if the range holds lat = 0); x = (lon - lon0) cos(lat) is
// extreme at those bounds.
void sfl_xrange(double a_c, double lat_c, double R_deg, double sinR, double* x_lo,
                double* x_hi) {
  const double H = std::asin(sinR / std::cos(lat_c * kDeg)) / kDeg;
  const double c1 = std::cos((lat_c - R_deg) * kDeg), c2 = std::cos((lat_c + R_deg) * kDeg);
  const double cmin = std::min(c1, c2);
  const double cmax = (lat_c - R_deg <= 0.0 && lat_c + R_deg >= 0.0) ? 1.0 : std::max(c1, c2);
  const double a = a_c - H, b = a_c + H;
  *x_lo = a >= 0.0 ? a * cmin : a * cmax;
  *x_hi = b >= 0.0 ? b * cmax : b * cmin;
}

// Haversine of the great-circle separation (radians in, dimensionless out).
double haversine(double lat_m, double lat_n, double dlon) {
  double a = std::sin(0.5 * (lat_n - lat_m));
  double b = std::sin(0.5 * dlon);
  double cm = std::cos(lat_m);
  if (g_mutation == 1) cm = 1.0;  // dropped cos(lat_m) factor
  return a * a + cm * std::cos(lat_n) * b * b;
}

bool inside(double h, double hR) {
  if (g_mutation == 3) return h < hR * (1.0 - 1e-3);  // boundary pulled inward
  return h <= hR;
}

double weight_of(double h, const Derived& d) {
  double hh = std::min(h, 1.0);
  double dist = 2.0 * std::asin(std::sqrt(hh));
  double e = dist * dist / (2.0 * d.sigma_rad * d.sigma_rad);
  if (g_mutation == 5) e = dist / (2.0 * d.sigma_rad);  // d instead of d^2
  return std::exp(-e);
}

int threads_or_default(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

// Wrap degrees into [-180, 180).
double wrap180(double a) {
  double r = std::fmod(a + 180.0, 360.0);
  if (r < 0) r += 360.0;
  return r - 180.0;
}

// ---------------------------------------------------------------------------
// Indexed oracle: its own simple index.  Samples are sorted (stable) into
// declination strips of height R, and inside a strip by the wrapped RA offset
// from the map centre.  A cell scans the strips within +-R of its declination
// and, inside each, the RA window +-asin(sin R / cos lat_m) (the widest RA
// extent of a circle of radius R), then applies the exact haversine test.
// ---------------------------------------------------------------------------
struct Index {
  og_geom g;
  og_kernel k;
  Derived d;
  int64_t n;
  const double* lon;  // caller-owned, degrees
  const double* lat;
  double lat_ref;
  int64_t n_strips;
  std::vector<int64_t> strip_off;  // n_strips + 1
  std::vector<int64_t> order;      // sample indices in (strip, ra) order
  std::vector<double> ra_sorted;   // wrapped RA offset in that order
  std::vector<double> lat_rad, lon_rad;
};

int64_t strip_of(const Index* ix, double lat_deg) {
  double s = std::floor((lat_deg - ix->lat_ref) / ix->d.R_deg);
  if (s < 0) return -1;
  if (s >= (double)ix->n_strips) return ix->n_strips;
  return (int64_t)s;
}

// Collect (n, h) for all samples within R of cell m, ascending n.
void neighbours_of(const Index* ix, int64_t m, std::vector<std::pair<int64_t, double>>* out) {
  out->clear();
  double clon, clat;
  cell_centre(&ix->g, m, &clon, &clat);
  const double latm = clat * kDeg, lonm = clon * kDeg;
  const double slack = 1e-9;
  int64_t s0 = strip_of(ix, clat - ix->d.R_deg - slack);
  int64_t s1 = strip_of(ix, clat + ix->d.R_deg + slack);
  s0 = std::max<int64_t>(s0, 0);
  s1 = std::min<int64_t>(s1, ix->n_strips - 1);
  double cm = std::cos(latm), sR = std::sin(ix->d.R_rad);
  bool full = cm <= sR;  // circle reaches a pole: every RA is possible
  double H = full ? 180.0 : std::asin(sR / cm) / kDeg + slack;
  double a = wrap180(clon - ix->g.lon0);
  auto scan = [&](int64_t s, double lo, double hi) {
    auto b = ix->ra_sorted.begin() + ix->strip_off[s];
    auto e = ix->ra_sorted.begin() + ix->strip_off[s + 1];
    auto p0 = std::lower_bound(b, e, lo);
    auto p1 = std::upper_bound(b, e, hi);
    for (auto p = p0; p < p1; ++p) {
      int64_t j = ix->order[p - ix->ra_sorted.begin()];
      double h = haversine(latm, ix->lat_rad[j], ix->lon_rad[j] - lonm);
      if (inside(h, ix->d.hR)) out->push_back({j, h});
    }
  };
  for (int64_t s = s0; s <= s1; ++s) {
    if (full || H >= 180.0) {
      scan(s, -std::numeric_limits<double>::infinity(), std::numeric_limits<double>::infinity());
      continue;
    }
    scan(s, a - H, a + H);
    if (a - H < -180.0) scan(s, a - H + 360.0, std::numeric_limits<double>::infinity());
    if (a + H >= 180.0) scan(s, -std::numeric_limits<double>::infinity(), a + H - 360.0);
  }
  std::sort(out->begin(), out->end());
}

}  // namespace

extern "C" {

void og_set_mutation(int m) { g_mutation = m; }

// Derived kernel constants: sigma (rad), R (rad), sin^2(R/2).
void og_kernel_constants(const og_kernel* k, double* out3) {
  Derived d = derive(k);
  out3[0] = d.sigma_rad;
  out3[1] = d.R_rad;
  out3[2] = d.hR;
}

void og_cell_centres(const og_geom* g, double* lon_deg, double* lat_deg) {
  int64_t M = (int64_t)g->nx * g->ny;
  for (int64_t m = 0; m < M; ++m) cell_centre(g, m, &lon_deg[m], &lat_deg[m]);
}

// ---------------------------------------------------------------------------
// Brute force: every (cell, sample) pair, O(M*N).  nb_off has M+1 entries.
// ---------------------------------------------------------------------------
int64_t og_bf_count(int64_t n, const double* lon, const double* lat, const og_geom* g,
                    const og_kernel* k, int64_t* nb_off, int nthreads) {
  Derived d = derive(k);
  int64_t M = (int64_t)g->nx * g->ny;
  std::vector<int64_t> cnt(M, 0);
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads_or_default(nthreads))
  for (int64_t m = 0; m < M; ++m) {
    double clon, clat;
    cell_centre(g, m, &clon, &clat);
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) {
      double h = haversine(clat * kDeg, lat[j] * kDeg, (lon[j] - clon) * kDeg);
      if (inside(h, d.hR)) ++c;
    }
    cnt[m] = c;
  }
  nb_off[0] = 0;
  for (int64_t m = 0; m < M; ++m) nb_off[m + 1] = nb_off[m] + cnt[m];
  return nb_off[M];
}

void og_bf_fill(int64_t n, const double* lon, const double* lat, const og_geom* g,
                const og_kernel* k, const int64_t* nb_off, int32_t* nb_idx, double* nb_w,
                int nthreads) {
  Derived d = derive(k);
  int64_t M = (int64_t)g->nx * g->ny;
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads_or_default(nthreads))
  for (int64_t m = 0; m < M; ++m) {
    double clon, clat;
    cell_centre(g, m, &clon, &clat);
    int64_t p = nb_off[m];
    for (int64_t j = 0; j < n; ++j) {
      double h = haversine(clat * kDeg, lat[j] * kDeg, (lon[j] - clon) * kDeg);
      if (inside(h, d.hR)) {
        nb_idx[p] = (int32_t)j;
        nb_w[p] = weight_of(h, d);
        ++p;
      }
    }
  }
}

// Eq. 1 on a given neighbour list: W[m] = sum w, map[m, c] = sum w v / W (NaN if
// W = 0).  values are FP32 [n x ld] (upcast exactly); outputs FP64.
void og_grid_csr(int64_t M, const int64_t* nb_off, const int32_t* nb_idx, const double* nb_w,
                 int64_t C, const float* values, int64_t ld, double* map, double* W,
                 int nthreads) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads_or_default(nthreads))
  for (int64_t m = 0; m < M; ++m) {
    double wsum = 0.0;
    std::vector<double> s(C, 0.0);
    for (int64_t p = nb_off[m]; p < nb_off[m + 1]; ++p) {
      double w = nb_w[p];
      const float* v = values + (int64_t)nb_idx[p] * ld;
      wsum += w;
      for (int64_t c = 0; c < C; ++c) s[c] += w * (double)v[c];
    }
    W[m] = wsum;
    for (int64_t c = 0; c < C; ++c) {
      double r = wsum > 0.0 ? s[c] / wsum : std::numeric_limits<double>::quiet_NaN();
      if (g_mutation == 6 && wsum > 0.0) r = s[c] / (double)(nb_off[m + 1] - nb_off[m]);
      map[m * C + c] = r;
    }
  }
}

// ---------------------------------------------------------------------------
// Indexed oracle.
// ---------------------------------------------------------------------------
void* og_index_create(int64_t n, const double* lon, const double* lat, const og_geom* g,
                      const og_kernel* k) {
  Index* ix = new Index();
  ix->g = *g;
  ix->k = *k;
  ix->d = derive(k);
  ix->n = n;
  ix->lon = lon;
  ix->lat = lat;
  ix->lat_rad.resize(n);
  ix->lon_rad.resize(n);
  double lo = std::numeric_limits<double>::infinity(), hi = -lo;
  for (int64_t j = 0; j < n; ++j) {
    ix->lat_rad[j] = lat[j] * kDeg;
    ix->lon_rad[j] = lon[j] * kDeg;
    lo = std::min(lo, lat[j]);
    hi = std::max(hi, lat[j]);
  }
  if (n == 0) lo = hi = 0.0;
  ix->lat_ref = lo;
  ix->n_strips = (int64_t)std::floor((hi - lo) / ix->d.R_deg) + 1;
  std::vector<int64_t> strip(n);
  std::vector<double> ra(n);
  for (int64_t j = 0; j < n; ++j) {
    strip[j] = strip_of(ix, lat[j]);
    ra[j] = wrap180(lon[j] - g->lon0);
  }
  ix->order.resize(n);
  std::iota(ix->order.begin(), ix->order.end(), 0);
  std::stable_sort(ix->order.begin(), ix->order.end(), [&](int64_t a, int64_t b) {
    if (strip[a] != strip[b]) return strip[a] < strip[b];
    return ra[a] < ra[b];
  });
  ix->ra_sorted.resize(n);
  for (int64_t p = 0; p < n; ++p) ix->ra_sorted[p] = ra[ix->order[p]];
  ix->strip_off.assign(ix->n_strips + 1, 0);
  for (int64_t j = 0; j < n; ++j) ix->strip_off[strip[j] + 1]++;
  for (int64_t s = 0; s < ix->n_strips; ++s) ix->strip_off[s + 1] += ix->strip_off[s];
  return ix;
}

void og_index_destroy(void* h) { delete static_cast<Index*>(h); }

static int64_t cell_at(int64_t i, const int64_t* cells) { return cells ? cells[i] : i; }

// Canonical neighbour CSR (ascending sample index per cell) for ncells cells
// (cells == NULL: all M cells in order).  nb_off has ncells+1 entries.
int64_t og_index_count(void* h, int64_t ncells, const int64_t* cells, int64_t* nb_off,
                       int nthreads) {
  Index* ix = static_cast<Index*>(h);
  std::vector<int64_t> cnt(ncells, 0);
#pragma omp parallel num_threads(threads_or_default(nthreads))
  {
    std::vector<std::pair<int64_t, double>> nb;
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < ncells; ++i) {
      neighbours_of(ix, cell_at(i, cells), &nb);
      cnt[i] = (int64_t)nb.size();
    }
  }
  nb_off[0] = 0;
  for (int64_t i = 0; i < ncells; ++i) nb_off[i + 1] = nb_off[i] + cnt[i];
  return nb_off[ncells];
}

void og_index_fill(void* h, int64_t ncells, const int64_t* cells, const int64_t* nb_off,
                   int32_t* nb_idx, double* nb_w, double* nb_h, int nthreads) {
  Index* ix = static_cast<Index*>(h);
#pragma omp parallel num_threads(threads_or_default(nthreads))
  {
    std::vector<std::pair<int64_t, double>> nb;
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < ncells; ++i) {
      neighbours_of(ix, cell_at(i, cells), &nb);
      int64_t p = nb_off[i];
      for (auto& e : nb) {
        nb_idx[p] = (int32_t)e.first;
        if (nb_w) nb_w[p] = weight_of(e.second, ix->d);
        if (nb_h) nb_h[p] = e.second;
        ++p;
      }
    }
  }
}

// Eq. 1 with per-channel masking (NEXT-4's reading of the paper's "invalid
// data" handling, which it leaves implicit): in channel c a sample whose value
// is not finite contributes to neither sum, so each channel has its own
// W_c[m] = sum of the weights of the cell's samples with a finite value;
// map = S_c / W_c, NaN where W_c = 0.  map and Wc are [ncells x C] FP64.
void og_index_grid_masked(void* h, int64_t ncells, const int64_t* cells, int64_t C,
                          const float* values, int64_t ld, double* map, double* Wc,
                          int nthreads);

// Eq. 1 for ncells cells straight from the index (no stored CSR): map is
// [ncells x C] FP64, W is [ncells].
void og_index_grid(void* h, int64_t ncells, const int64_t* cells, int64_t C, const float* values,
                   int64_t ld, double* map, double* W, int nthreads) {
  Index* ix = static_cast<Index*>(h);
#pragma omp parallel num_threads(threads_or_default(nthreads))
  {
    std::vector<std::pair<int64_t, double>> nb;
    std::vector<double> s(C);
#pragma omp for schedule(dynamic, 4)
    for (int64_t i = 0; i < ncells; ++i) {
      neighbours_of(ix, cell_at(i, cells), &nb);
      std::fill(s.begin(), s.end(), 0.0);
      double wsum = 0.0;
      for (auto& e : nb) {
        double w = weight_of(e.second, ix->d);
        const float* v = values + e.first * ld;
        wsum += w;
        for (int64_t c = 0; c < C; ++c) s[c] += w * (double)v[c];
      }
      W[i] = wsum;
      for (int64_t c = 0; c < C; ++c) {
        double r = wsum > 0.0 ? s[c] / wsum : std::numeric_limits<double>::quiet_NaN();
        if (g_mutation == 6 && wsum > 0.0) r = s[c] / (double)nb.size();
        map[i * C + c] = r;
      }
    }
  }
}

void og_index_grid_masked(void* h, int64_t ncells, const int64_t* cells, int64_t C,
                          const float* values, int64_t ld, double* map, double* Wc,
                          int nthreads) {
  Index* ix = static_cast<Index*>(h);
#pragma omp parallel num_threads(threads_or_default(nthreads))
  {
    std::vector<std::pair<int64_t, double>> nb;
    std::vector<double> s(C), wc(C);
#pragma omp for schedule(dynamic, 4)
    for (int64_t i = 0; i < ncells; ++i) {
      neighbours_of(ix, cell_at(i, cells), &nb);
      std::fill(s.begin(), s.end(), 0.0);
      std::fill(wc.begin(), wc.end(), 0.0);
      for (auto& e : nb) {
        double w = weight_of(e.second, ix->d);
        const float* v = values + e.first * ld;
        for (int64_t c = 0; c < C; ++c) {
          if (!std::isfinite(v[c]) && g_mutation != 10) continue;  // 10: mask ignored
          wc[c] += w;
          s[c] += w * (double)v[c];
        }
      }
      for (int64_t c = 0; c < C; ++c) {
        Wc[i * C + c] = wc[c];
        map[i * C + c] = wc[c] > 0.0 ? s[c] / wc[c] : std::numeric_limits<double>::quiet_NaN();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Bin key of the padded map (the GPU path's replacement for the HEALPix
// pixel index of Sec. 4.1.1), written from its definition:
//   pad_y = ceil(R / dlat) + 1,  pad_x = ceil(Hmax / dlon) + 1, where Hmax is
//   the RA half-width asin(sin R / cos|lat|) at the most poleward cell row;
//   a  = wrap(lon - lon0) into [-180, 180) as a - 360 floor((a + 180) / 360);
//   qx = a / dlon + (nx/2 + pad_x);  qy = (lat - lat0) / dlat + (ny/2 + pad_y);
//   key = floor(qy)/B * nbx + floor(qx)/B  if 0 <= floor(q) < n + 2 pad in
//   both axes, else n_bins (discarded), with nbx = ceil((nx + 2 pad_x) / B).
// All operations are single IEEE operations (no contraction) so that the key
// is reproducible bit for bit.  layout[0..3] = pad_x, pad_y, nbx, nby.
// Returns n_bins, or -1 if the map reaches a pole or wraps onto itself.
// ---------------------------------------------------------------------------
int64_t og_bin_layout(const og_geom* g, const og_kernel* k, int32_t bin_cells, int32_t* layout) {
  Derived d = derive(k);
  double half_rows = 0.5 * (double)(g->ny - 1) * g->dlat;
  double lat_a = std::fabs(g->lat0 - half_rows), lat_b = std::fabs(g->lat0 + half_rows);
  double lat_max = std::max(lat_a, lat_b);
  if (lat_max + d.R_deg >= 90.0) return -1;
  double Hmax = std::asin(std::sin(d.R_rad) / std::cos(lat_max * kDeg)) / kDeg;
  int32_t pad_y = (int32_t)std::ceil(d.R_deg / g->dlat) + 1;
  int32_t pad_x = (int32_t)std::ceil(Hmax / g->dlon) + 1;
  if (g->proj == 1) {
    // the widest x-excess of a first or last column cell's R-disc, over all rows
    const double sinR = std::sin(d.R_rad), xe = 0.5 * (double)(g->nx - 1) * g->dlon;
    double ex = 0.0;
    for (int32_t iy = 0; iy < g->ny; ++iy) {
      const double la = g->lat0 + ((double)iy - 0.5 * (double)(g->ny - 1)) * g->dlat;
      const double ce = std::cos(la * kDeg);
      double lo, hi;
      sfl_xrange(-xe / ce, la, d.R_deg, sinR, &lo, &hi);
      ex = std::max(ex, -xe - lo);
      sfl_xrange(xe / ce, la, d.R_deg, sinR, &lo, &hi);
      ex = std::max(ex, hi - xe);
    }
    pad_x = (int32_t)std::ceil(ex / g->dlon) + 1;
    if ((double)(g->nx + 2 * pad_x) * g->dlon / std::cos(lat_max * kDeg) >= 360.0) return -1;
  }
  if ((double)(g->nx + 2 * pad_x) * g->dlon >= 360.0) return -1;
  int32_t nbx = (g->nx + 2 * pad_x + bin_cells - 1) / bin_cells;
  int32_t nby = (g->ny + 2 * pad_y + bin_cells - 1) / bin_cells;
  if (layout) {
    layout[0] = pad_x;
    layout[1] = pad_y;
    layout[2] = nbx;
    layout[3] = nby;
  }
  return (int64_t)nbx * nby;
}

// key[N] (uint32), perm[N] = sample indices stably sorted by key (discarded
// samples last), bin_off[n_bins + 1] = start of each bin in perm.
int64_t og_bin_keys(int64_t n, const double* lon, const double* lat, const og_geom* g,
                    const og_kernel* k, int32_t bin_cells, uint32_t* key, int32_t* perm,
                    int32_t* bin_off) {
  int32_t lay[4];
  int64_t n_bins = og_bin_layout(g, k, bin_cells, lay);
  if (n_bins < 0) return -1;
  const int64_t wx = g->nx + 2 * lay[0], wy = g->ny + 2 * lay[1];
  const double cx = 0.5 * (double)g->nx + (double)lay[0];
  const double cy = 0.5 * (double)g->ny + (double)lay[1];
  for (int64_t j = 0; j < n; ++j) {
    double a = lon[j] - g->lon0;
    a = a - 360.0 * std::floor((a + 180.0) / 360.0);
    if (g->proj == 1) a = a * std::cos(lat[j] * kDeg);  // projected x
    double qx = a / g->dlon + cx;
    double qy = (lat[j] - g->lat0) / g->dlat + cy;
    double fx = std::floor(qx), fy = std::floor(qy);
    uint32_t kk = (uint32_t)n_bins;
    if (std::isfinite(fx) && std::isfinite(fy) && fx >= 0.0 && fy >= 0.0 && fx < (double)wx &&
        fy < (double)wy) {
      int64_t bx = (int64_t)fx / bin_cells, by = (int64_t)fy / bin_cells;
      kk = (uint32_t)(by * lay[2] + bx);
    }
    key[j] = kk;
  }
  std::vector<int32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  std::memcpy(perm, idx.data(), sizeof(int32_t) * n);
  std::vector<int64_t> cnt(n_bins + 1, 0);
  for (int64_t j = 0; j < n; ++j) cnt[key[j]]++;
  int64_t acc = 0;
  for (int64_t b = 0; b <= n_bins; ++b) {
    bin_off[b] = (int32_t)acc;
    if (b < n_bins) acc += cnt[b];
  }
  return n_bins;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// HEALPix, RING scheme (Gorski et al. 2005, ApJ 622, 759; the paper's
// pixelisation, Sec. 4.1.1), written from the scheme's definitions.  With
// N = nside: 12 N^2 equal-area pixels on 4N - 1 rings of constant latitude,
// numbered from the north pole (i = 1 .. 4N-1).  Polar caps (|z| > 2/3,
// z = sin(lat)): ring i < N holds 4i pixels (mirrored in the south, ring
// 4N - i); the equatorial belt (rings N .. 3N) holds 4N pixels per ring.
// Pixel j of a ring has its centre at phi = (j + s/2) * 360 / n_i degrees with
// s = 1 in the caps and s = (i - N + 1) mod 2 in the belt.  Ring centres:
// z = 1 - i^2 / (3 N^2) in the north cap, z = (4N - 2i) / (3N) in the belt.
//
// ang2pix (point -> ring, pixel in ring), from the same definitions: in the
// belt the pixel edges are the lines t - 3z/4 = const and t + 3z/4 = const in
// (t = phi / 90 deg, z), spaced 1/N, so the two edge indices jp = floor(N (1/2
// + t) - 3Nz/4) and jm = floor(N (1/2 + t) + 3Nz/4) give the ring (from their
// difference) and the pixel (from their sum).  In a cap, within each 90-degree
// face the edges are tp * N sqrt(3 (1 - |z|)) = const and (1 - tp) * N
// sqrt(3 (1 - |z|)) = const (tp = t mod 1); their indices give the ring from
// the pole, and the pixel is floor(t * ring) (cap pixels are exact
// 360 / n_i slices of their ring).
// All arithmetic is single IEEE operations (no contraction): nside is a power
// of two, so the products by N are exact.
// ---------------------------------------------------------------------------
namespace {

struct HpxRing {
  int64_t n;     // pixels in the ring
  int64_t half;  // 1 if the centres are offset by half a pixel
};

HpxRing hpx_ring(int64_t N, int64_t i) {
  if (i < N) return {4 * i, 1};
  if (i > 3 * N) return {4 * (4 * N - i), 1};
  int64_t s = (i - N + 1) & 1;
  if (g_mutation == 7) s ^= 1;  // belt shift on the wrong rings
  return {4 * N, s};
}

// (ring, pixel in ring) of a point: z = sin(lat), t = phi / 90 deg in [0, 4).
void hpx_ang2pix(int64_t N, double z, double t, int64_t* ring, int64_t* pix) {
  const double Nd = (double)N;
  const double az = std::fabs(z);
  if (az <= 2.0 / 3.0) {
    double t1 = Nd * (0.5 + t);
    double t2 = (Nd * 0.75) * z;
    int64_t jp = (int64_t)std::floor(t1 - t2);
    int64_t jm = (int64_t)std::floor(t1 + t2);
    int64_t ir = N + 1 + jp - jm;  // 1 .. 2N+1 from the ring at z = 2/3
    int64_t kshift = 1 - (ir & 1);
    if (g_mutation == 9) kshift = ir & 1;  // pixel shift on the wrong rings
    int64_t ip = (jp + jm - N + kshift + 1) / 2;
    ip = ((ip % (4 * N)) + 4 * N) % (4 * N);
    *ring = N - 1 + ir;
    *pix = ip;
    return;
  }
  double tp = t - std::floor(t);
  double tmp = Nd * std::sqrt(3.0 * (1.0 - az));
  if (g_mutation == 8) tmp = Nd * std::sqrt(3.0 * (1.0 + az));  // wrong cap edge spacing
  int64_t jp = (int64_t)std::floor(tp * tmp);
  int64_t jm = (int64_t)std::floor((1.0 - tp) * tmp);
  int64_t ir = jp + jm + 1;  // ring from the nearest pole, 1 .. N
  if (ir > N) ir = N;
  int64_t ip = (int64_t)std::floor(t * (double)ir);
  if (ip >= 4 * ir) ip = 4 * ir - 1;
  *ring = z > 0.0 ? ir : 4 * N - ir;
  *pix = ip;
}

// Continuous ring coordinate of z (ring centres at integers), for ring
// ranges; a pixel of ring i lies between the centres of rings i - 1 and
// i + 1, so the pixels holding points with z in [z0, z1] are in rings
// floor(rho(z1)) - 1 .. ceil(rho(z0)) + 1.
double hpx_rho(int64_t N, double z) {
  const double Nd = (double)N;
  if (z > 2.0 / 3.0) return Nd * std::sqrt(3.0 * (1.0 - z));
  if (z < -2.0 / 3.0) return 4.0 * Nd - Nd * std::sqrt(3.0 * (1.0 + z));
  return 2.0 * Nd - (3.0 * Nd * z) / 2.0;
}

}  // namespace

extern "C" {

void og_hpx_ang2pix(int64_t nside, int64_t n, const double* z, const double* phi_deg,
                    int64_t* ring, int64_t* pix, int64_t* ipix) {
  const int64_t N = nside;
  for (int64_t k = 0; k < n; ++k) {
    double a = phi_deg[k] - 360.0 * std::floor(phi_deg[k] / 360.0);
    int64_t i, j;
    hpx_ang2pix(N, z[k], a / 90.0, &i, &j);
    // pixels before ring i: 2 i (i - 1) in the north cap, then 4N per ring
    int64_t before;
    if (i <= N) {
      before = 2 * i * (i - 1);
    } else if (i <= 3 * N) {
      before = 2 * N * (N - 1) + (i - N) * 4 * N;
    } else {
      int64_t ii = 4 * N - i;  // south cap, counted from the south pole
      before = 12 * N * N - 2 * ii * (ii + 1);
    }
    ring[k] = i;
    pix[k] = j;
    ipix[k] = before + j;
  }
}

// Centres of all 12 nside^2 pixels in ring order (z and phi in degrees).
void og_hpx_centres(int64_t nside, double* z, double* phi_deg) {
  const int64_t N = nside;
  const double Nd = (double)N;
  int64_t k = 0;
  for (int64_t i = 1; i <= 4 * N - 1; ++i) {
    HpxRing r = hpx_ring(N, i);
    double zi;
    if (i < N)
      zi = 1.0 - (double)(i * i) / (3.0 * Nd * Nd);
    else if (i > 3 * N)
      zi = -(1.0 - (double)((4 * N - i) * (4 * N - i)) / (3.0 * Nd * Nd));
    else
      zi = (double)(4 * N - 2 * i) / (3.0 * Nd);
    for (int64_t j = 0; j < r.n; ++j, ++k) {
      z[k] = zi;
      phi_deg[k] = ((double)j + 0.5 * (double)r.half) * 360.0 / (double)r.n;
    }
  }
}

// Bin layout of the HEALPix variant (the LUT of Sec. 4.1.1 restricted to the
// padded map): the rings whose pixels can hold a sample within R of a cell,
// and in each ring the pixels whose centres lie within 2 pixels of the
// map's RA range widened by Hmax (a pixel's RA extent is its centre +- half
// a pixel).  table[4 r + 0..3] = n_i, J0 (first pixel, unwrapped), cnt,
// half for ring ring0 + r; bins are numbered ring by ring, pixel (j - J0) mod
// n_i inside a ring.  Returns n_bins (-1: the map reaches a pole or wraps).
int64_t og_hpx_layout(const og_geom* g, const og_kernel* k, int64_t nside, int64_t* ring0,
                      int64_t* n_rings, int64_t* table) {
  Derived d = derive(k);
  const int64_t N = nside;
  double half_rows = 0.5 * (double)(g->ny - 1) * g->dlat;
  double half_cols = 0.5 * (double)(g->nx - 1) * g->dlon;
  double lat_lo = g->lat0 - half_rows, lat_hi = g->lat0 + half_rows;
  double lat_max = std::max(std::fabs(lat_lo), std::fabs(lat_hi));
  if (lat_max + d.R_deg >= 90.0) return -1;
  double Hmax = std::asin(std::sin(d.R_rad) / std::cos(lat_max * kDeg)) / kDeg;
  double pa = (g->lon0 - half_cols) - Hmax, pb = (g->lon0 + half_cols) + Hmax;
  if (pb - pa >= 360.0) return -1;
  double z0 = std::sin((lat_lo - d.R_deg) * kDeg), z1 = std::sin((lat_hi + d.R_deg) * kDeg);
  int64_t i0 = std::max<int64_t>(1, (int64_t)std::floor(hpx_rho(N, z1)) - 2);
  int64_t i1 = std::min<int64_t>(4 * N - 1, (int64_t)std::ceil(hpx_rho(N, z0)) + 2);
  int64_t total = 0;
  for (int64_t i = i0; i <= i1; ++i) {
    HpxRing r = hpx_ring(N, i);
    double ua = (pa * (double)r.n) / 360.0 - 0.5 * (double)r.half;
    double ub = (pb * (double)r.n) / 360.0 - 0.5 * (double)r.half;
    int64_t J0 = (int64_t)std::ceil(ua - 2.0), J1 = (int64_t)std::floor(ub + 2.0);
    int64_t cnt = J1 - J0 + 1;
    if (cnt >= r.n) {
      cnt = r.n;
      J0 = 0;
    }
    if (table) {
      int64_t* e = table + 4 * (i - i0);
      e[0] = r.n;
      e[1] = J0;
      e[2] = cnt;
      e[3] = r.half;
    }
    total += cnt;
  }
  if (ring0) *ring0 = i0;
  if (n_rings) *n_rings = i1 - i0 + 1;
  return total;
}

// HEALPix-variant bin keys: z = sin(lat), phi = lon wrapped into [0, 360);
// key = (bins of the rings before) + (j - J0) mod n_i, or n_bins when the
// ring or pixel is outside the layout.  perm / bin_off as og_bin_keys.
int64_t og_hpx_keys(int64_t n, const double* lon, const double* lat, const og_geom* g,
                    const og_kernel* k, int64_t nside, uint32_t* key, int32_t* perm,
                    int32_t* bin_off) {
  int64_t i0 = 0, nr = 0;
  int64_t n_bins = og_hpx_layout(g, k, nside, &i0, &nr, nullptr);
  if (n_bins < 0) return -1;
  std::vector<int64_t> tab(4 * nr), base(nr);
  og_hpx_layout(g, k, nside, &i0, &nr, tab.data());
  int64_t acc = 0;
  for (int64_t r = 0; r < nr; ++r) {
    base[r] = acc;
    acc += tab[4 * r + 2];
  }
  for (int64_t q = 0; q < n; ++q) {
    double z = std::sin(lat[q] * kDeg);
    double a = lon[q] - 360.0 * std::floor(lon[q] / 360.0);
    int64_t i, j;
    hpx_ang2pix(nside, z, a / 90.0, &i, &j);
    uint32_t kk = (uint32_t)n_bins;
    if (i >= i0 && i < i0 + nr) {
      const int64_t* e = tab.data() + 4 * (i - i0);
      int64_t jr = ((j - e[1]) % e[0] + e[0]) % e[0];
      if (jr < e[2]) kk = (uint32_t)(base[i - i0] + jr);
    }
    key[q] = kk;
  }
  std::vector<int32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  std::memcpy(perm, idx.data(), sizeof(int32_t) * n);
  std::vector<int64_t> cnt(n_bins + 1, 0);
  for (int64_t q = 0; q < n; ++q) cnt[key[q]]++;
  int64_t run = 0;
  for (int64_t b = 0; b <= n_bins; ++b) {
    bin_off[b] = (int32_t)run;
    if (b < n_bins) run += cnt[b];
  }
  return n_bins;
}

}  // extern "C"
