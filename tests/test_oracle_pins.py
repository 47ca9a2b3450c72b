"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-derives the oracle's own formula chain (haversine -> asin ->
Gaussian).  Each pin uses an independent route: brute force, a meridian
closed form, the chord formula for the separation, invariants of Eq. 1
(constant sky, linearity, convexity), symmetries (RA wrap, sample order) and
the Gaussian-convolution closed form for a point source.  The last test plants
a mistake in the oracle and checks that some pin fails.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2207_04584_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ARCMIN = 1.0 / 60.0


def _small_case(seed, n=1500, nx=20, ny=16, lon0=45.0, lat0=20.0, cell=ARCMIN, fwhm=3 * ARCMIN,
                C=3, spread=1.3):
    rng = np.random.default_rng(seed)
    half_x = 0.5 * nx * cell * spread
    half_y = 0.5 * ny * cell * spread
    lon = lon0 + rng.uniform(-half_x, half_x, n)
    lat = lat0 + rng.uniform(-half_y, half_y, n)
    geom = {"nx": nx, "ny": ny, "lon0": lon0, "lat0": lat0, "dlon": cell, "dlat": cell}
    values = rng.normal(1.0, 2.0, (n, C)).astype(np.float32)
    return lon % 360.0, lat, geom, fwhm, values


def _centres(geom):
    """Cell centres from the map geometry (computed here, not by the oracle)."""
    m = np.arange(geom["nx"] * geom["ny"])
    ix, iy = m % geom["nx"], m // geom["nx"]
    lon = geom["lon0"] + (ix - 0.5 * (geom["nx"] - 1)) * geom["dlon"]
    lat = geom["lat0"] + (iy - 0.5 * (geom["ny"] - 1)) * geom["dlat"]
    return lon, lat


def _unit(lon_deg, lat_deg):
    a, d = np.radians(lon_deg), np.radians(lat_deg)
    return np.stack([np.cos(d) * np.cos(a), np.cos(d) * np.sin(a), np.sin(d)], axis=-1)


# --------------------------------------------------------------------------
# pins (each raises AssertionError when the oracle is wrong)
# --------------------------------------------------------------------------
def pin_bruteforce_vs_indexed(seed=1, lon0=45.0, wrtol=5e-12):
    lon, lat, geom, fwhm, values = _small_case(seed, lon0=lon0)
    bf = oracle.neighbours_bruteforce(lon, lat, geom, fwhm)
    ix = oracle.Index(lon, lat, geom, fwhm)
    io = ix.neighbours()
    assert np.array_equal(bf[0], io[0]), "neighbour counts differ"
    assert np.array_equal(bf[1], io[1]), "neighbour indices differ"
    # the two routes round the RA difference differently: weights agree to FP64
    assert np.allclose(bf[2], io[2], rtol=wrtol, atol=0), "weights differ"
    m1, w1 = oracle.grid_csr(*bf, values)
    m2, w2 = ix.grid(values)
    assert np.allclose(m1, m2, rtol=1e-11, atol=1e-11, equal_nan=True)
    assert np.allclose(w1, w2, rtol=wrtol, atol=0)


def pin_meridian_golden():
    case = json.load(open(os.path.join(GOLDEN, "meridian_case.json")))
    g = case["cell"]
    fwhm = case["fwhm_arcmin"] * ARCMIN
    sigma_deg = fwhm / math.sqrt(8.0 * math.log(2.0))
    k = np.array(case["k_sigma"])
    lon = np.full(len(k), g["lon0"])
    lat = g["lat0"] + k * sigma_deg
    values = np.array(case["values"], np.float32)[:, None]
    off, idx, w = oracle.neighbours_bruteforce(lon, lat, g, fwhm, case["support"])
    want_w = np.array(case["expected_weight"])
    got_w = np.zeros(len(k))
    got_w[idx] = w
    assert np.allclose(got_w, want_w, rtol=1e-12, atol=1e-15), (got_w, want_w)
    keep = want_w > 0
    want_map = float(np.sum(want_w[keep] * values[keep, 0]) / np.sum(want_w[keep]))
    m, Wm = oracle.grid_csr(off, idx, w, values)
    assert abs(m[0, 0] - want_map) <= 1e-12 * abs(want_map)
    assert abs(Wm[0] - want_w.sum()) <= 1e-12 * want_w.sum()


def pin_isolated_sample(seed=3):
    """One sample, value 1: the weight map is the kernel itself (chord formula)."""
    rng = np.random.default_rng(seed)
    geom = {"nx": 24, "ny": 20, "lon0": 200.0, "lat0": 55.0, "dlon": 0.5 * ARCMIN,
            "dlat": 0.5 * ARCMIN}
    fwhm = 2.9 * ARCMIN
    sig, R, _ = oracle.kernel_constants(fwhm, 3.0)
    for _ in range(3):
        lon = np.array([200.0 + rng.uniform(-4, 4) * ARCMIN])
        lat = np.array([55.0 + rng.uniform(-3, 3) * ARCMIN])
        values = np.array([[1.0, 5.0]], np.float32)
        off, idx, w = oracle.neighbours_bruteforce(lon, lat, geom, fwhm)
        m, Wm = oracle.grid_csr(off, idx, w, values)
        clon, clat = _centres(geom)
        chord = np.linalg.norm(_unit(clon, clat) - _unit(lon, lat)[0], axis=1)
        d = 2.0 * np.arcsin(chord / 2.0)
        inside = d <= R
        near = np.abs(d / R - 1.0) < 1e-9
        want = np.where(inside, np.exp(-d * d / (2 * sig * sig)), 0.0)
        ok = ~near
        assert np.allclose(Wm[ok], want[ok], rtol=5e-12, atol=0), "kernel shape / radius"
        has = Wm > 0
        assert np.allclose(m[has, 0], 1.0, rtol=4e-16) and np.allclose(m[has, 1], 5.0, rtol=4e-16)
        assert np.all(np.isnan(m[~has]))
        assert np.all(has[inside & ok]) and not np.any(has[~inside & ok])


def pin_constant_sky():
    wl = W.config1(with_values=False, n=6000, nx=60, ny=60)
    ix = oracle.Index(wl["lon"], wl["lat"], wl["geom"], wl["fwhm_deg"])
    v = np.full((len(wl["lon"]), 2), 3.7, np.float32)
    m, Wm = ix.grid(v)
    has = Wm > 0
    assert has.sum() > 1000
    k = float(np.float32(3.7))
    assert np.all(np.abs(m[has] - k) <= 8 * np.finfo(np.float64).eps * k)
    assert np.all(np.isnan(m[~has]))


def pin_linearity(seed=5):
    lon, lat, geom, fwhm, values = _small_case(seed, C=2)
    rng = np.random.default_rng(seed + 1)
    a, b = 0.75, -2.5  # exactly representable, products exact in FP64 upcast
    v2 = (a * values[:, 0].astype(np.float64) + b * values[:, 1]).astype(np.float32)
    # use exactly representable combos: scale values so that the float32 combo is exact
    base = np.round(values * 64) / 64
    v2 = (a * base[:, 0] + b * base[:, 1]).astype(np.float32)
    vals = np.concatenate([base.astype(np.float32), v2[:, None]], axis=1)
    perm = rng.permutation(3)
    ix = oracle.Index(lon, lat, geom, fwhm)
    m, Wm = ix.grid(vals)
    has = Wm > 0
    lhs = m[has, 2]
    rhs = a * m[has, 0] + b * m[has, 1]
    scale = np.max(np.abs(m[has]))
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * scale
    mp, _ = ix.grid(np.ascontiguousarray(vals[:, perm]))
    assert np.array_equal(mp[has], m[has][:, perm])


def pin_convexity(seed=6):
    lon, lat, geom, fwhm, values = _small_case(seed, C=4)
    off, idx, w = oracle.neighbours_bruteforce(lon, lat, geom, fwhm)
    m, Wm = oracle.grid_csr(off, idx, w, values)
    for cell in range(len(off) - 1):
        a, b = off[cell], off[cell + 1]
        if b == a:
            continue
        v = values[idx[a:b]].astype(np.float64)
        lo, hi = v.min(axis=0), v.max(axis=0)
        tol = 1e-12 * np.maximum(np.abs(lo), np.abs(hi))
        assert np.all(m[cell] >= lo - tol) and np.all(m[cell] <= hi + tol)


def pin_wrap_invariance(seed=7):
    # field straddling RA = 0: lon0 = 0.05 deg
    lon, lat, geom, fwhm, values = _small_case(seed, lon0=0.05)
    ix1 = oracle.Index(lon, lat, geom, fwhm)
    ix2 = oracle.Index(lon + 360.0, lat, geom, fwhm)
    a = ix1.neighbours(with_h=True)
    b = ix2.neighbours(with_h=True)
    _, _, hR = oracle.kernel_constants(fwhm, 3.0)
    if not (np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])):
        # any difference must sit in the FP64 tie band around h = sin^2(R/2)
        sa = set(zip(np.repeat(np.arange(len(a[0]) - 1), np.diff(a[0])), a[1]))
        sb = set(zip(np.repeat(np.arange(len(b[0]) - 1), np.diff(b[0])), b[1]))
        assert len(sa ^ sb) <= 2
    m1, _ = ix1.grid(values)
    m2, _ = ix2.grid(values)
    assert np.allclose(m1, m2, rtol=1e-10, atol=1e-10, equal_nan=True)
    # indexed oracle straddling RA=0 must equal brute force
    # (RA differences across 0/360 are rounded at the 360-degree scale: the two
    # FP64 routes then agree to ~1e-11 in the weights)
    pin_bruteforce_vs_indexed(seed=seed, lon0=0.05, wrtol=1e-10)


def pin_permutation_invariance(seed=8):
    lon, lat, geom, fwhm, values = _small_case(seed)
    rng = np.random.default_rng(seed)
    p = rng.permutation(len(lon))
    ix1 = oracle.Index(lon, lat, geom, fwhm)
    ix2 = oracle.Index(lon[p], lat[p], geom, fwhm)
    a = ix1.neighbours()
    b = ix2.neighbours()
    assert np.array_equal(a[0], b[0])
    inv = np.argsort(p)  # new index j holds old sample p[j]
    for cell in range(len(a[0]) - 1):
        s, e = a[0][cell], a[0][cell + 1]
        old = np.sort(p[b[1][s:e]])
        assert np.array_equal(old, a[1][s:e])
    m1, _ = ix1.grid(values)
    m2, _ = ix2.grid(np.ascontiguousarray(values[p]))
    assert np.allclose(m1, m2, rtol=1e-12, atol=1e-12, equal_nan=True)
    del inv


def pin_point_source_fwhm():
    """Gaussian source * truncated Gaussian kernel: second moments add.

    For a 2-D Gaussian kernel truncated at r = 3 sigma the radial second moment
    is 2 sigma^2 (1 - 5.5 e^-4.5) / (1 - e^-4.5) (closed form); with dense
    uniform sampling the normalised gridding is the convolution with that
    kernel, so the map's per-axis variance is s_src^2 + s_k^2 (1-5.5e^-4.5)/(1-e^-4.5).
    """
    rng = np.random.default_rng(11)
    cell = 0.5 * ARCMIN
    nx = ny = 64
    lon0, lat0 = 10.0, 0.0  # equator: RA and Dec offsets are both arc lengths
    half = 0.5 * nx * cell + 0.1
    n = 120000
    lon = lon0 + rng.uniform(-half, half, n)
    lat = lat0 + rng.uniform(-half, half, n)
    fwhm_k = 3.0 * ARCMIN
    fwhm_s = 2.0 * ARCMIN
    ss = fwhm_s / math.sqrt(8 * math.log(2))
    sk = fwhm_k / math.sqrt(8 * math.log(2))
    r2 = (lon - lon0) ** 2 + (lat - lat0) ** 2
    v = np.exp(-0.5 * r2 / ss ** 2).astype(np.float32)[:, None]
    geom = {"nx": nx, "ny": ny, "lon0": lon0, "lat0": lat0, "dlon": cell, "dlat": cell}
    ix = oracle.Index(lon, lat, geom, fwhm_k)
    m, Wm = ix.grid(v)
    clon, clat = _centres(geom)
    img = m[:, 0]
    x = clon - lon0
    var_x = np.sum(img * x * x) / np.sum(img)
    e = math.exp(-4.5)
    want = ss ** 2 + sk ** 2 * (1 - 5.5 * e) / (1 - e)
    assert abs(var_x / want - 1.0) < 0.02, (var_x, want)


PINS = [pin_bruteforce_vs_indexed, pin_meridian_golden, pin_isolated_sample, pin_constant_sky,
        pin_linearity, pin_convexity, pin_wrap_invariance, pin_permutation_invariance,
        pin_point_source_fwhm]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    oracle.set_mutation(0)
    pin()


# --------------------------------------------------------------------------
# bin key / sort / offsets of the padded map
# --------------------------------------------------------------------------
@pytest.mark.parametrize("bin_cells", [1, 2, 4])
def test_bin_keys_sort_and_offsets(bin_cells):
    wl = W.config1(with_values=False)
    key, perm, off = oracle.bin_keys(wl["lon"], wl["lat"], wl["geom"], wl["fwhm_deg"],
                                     bin_cells=bin_cells)
    n_bins, lay = oracle.bin_layout(wl["geom"], wl["fwhm_deg"], bin_cells=bin_cells)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    sk = key[perm]
    assert np.array_equal(off, np.searchsorted(sk, np.arange(n_bins + 1), side="left"))
    # each kept sample lies in its bin (checked away from bin edges by a
    # different evaluation order of the pixel coordinate)
    g = wl["geom"]
    padx, pady, nbx, nby = lay
    a = (wl["lon"] - g["lon0"] + 180.0) % 360.0 - 180.0
    qx = (a + (0.5 * g["nx"] + padx) * g["dlon"]) / g["dlon"]
    qy = (wl["lat"] - g["lat0"] + (0.5 * g["ny"] + pady) * g["dlat"]) / g["dlat"]
    kept = key < n_bins
    bx, by = key[kept] % nbx, key[kept] // nbx
    fx, fy = qx[kept] / bin_cells, qy[kept] / bin_cells
    far = (np.abs(fx - np.round(fx)) > 1e-9) & (np.abs(fy - np.round(fy)) > 1e-9)
    assert np.all((np.floor(fx) == bx)[far]) and np.all((np.floor(fy) == by)[far])


def test_bin_padding_holds_every_neighbour():
    """Every sample within R of a cell is kept by the padded-map key."""
    lon, lat, geom, fwhm, _ = _small_case(21, n=3000, spread=2.5)
    off, idx, _ = oracle.neighbours_bruteforce(lon, lat, geom, fwhm)
    key, _, _ = oracle.bin_keys(lon, lat, geom, fwhm, bin_cells=2)
    n_bins, _ = oracle.bin_layout(geom, fwhm, bin_cells=2)
    assert np.all(key[np.unique(idx)] < n_bins)
    assert np.any(key == n_bins)  # the spread field does put samples outside


def test_bin_layout_rejects_pole_and_wrap():
    fwhm = 3 * ARCMIN
    assert oracle.bin_layout({"nx": 10, "ny": 10, "lon0": 0.0, "lat0": 89.95, "dlon": ARCMIN,
                              "dlat": ARCMIN}, fwhm)[0] == -1
    assert oracle.bin_layout({"nx": 400, "ny": 10, "lon0": 0.0, "lat0": 0.0, "dlon": 1.0,
                              "dlat": ARCMIN}, fwhm)[0] == -1


# --------------------------------------------------------------------------
# pin strength: each planted mistake is caught by at least one pin
# --------------------------------------------------------------------------
MUTATIONS = {1: "dropped cos(lat_m)", 2: "wrong FWHM->sigma", 3: "boundary pulled in",
             4: "transposed cell index", 5: "d instead of d^2", 6: "normalised by count"}


@pytest.mark.parametrize("mutation", sorted(MUTATIONS), ids=list(MUTATIONS.values()))
def test_planted_mistake_is_caught(mutation):
    caught = []
    try:
        oracle.set_mutation(mutation)
        for pin in [pin_meridian_golden, pin_isolated_sample, pin_constant_sky,
                    pin_point_source_fwhm]:
            try:
                pin()
            except AssertionError:
                caught.append(pin.__name__)
    finally:
        oracle.set_mutation(0)
    assert caught, f"no pin caught mutation {MUTATIONS[mutation]}"
