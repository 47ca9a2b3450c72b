"""Pins of the oracle's Sanson-Flamsteed map (the sinusoidal projection about
lon0: cells on a regular grid of x = (lon - lon0) cos(lat), y = lat - lat0).
The cell centres are pinned by what the projection fixes: the middle row is
the plain grid's only where cos(lat0) = 1 (the equator), and along any row
neighbouring centres are dlon apart on the sky (the projection keeps lengths
along parallels) while the plain grid's are dlon cos(lat) apart; a sample at
a cell centre recovers its value there; the padded-map bins keep every
brute-force neighbour of a wide, high-latitude, sheared map; brute force and
the indexed oracle agree on it.  A planted mistake (cos(lat) dropped) is
caught."""
import math

import numpy as np
import pytest

import oracle

ARCMIN = 1.0 / 60.0


def _gc_deg(lon1, lat1, lon2, lat2):
    p1, p2 = np.radians(lat1), np.radians(lat2)
    h = np.sin((p2 - p1) / 2) ** 2 + np.cos(p1) * np.cos(p2) * np.sin(np.radians(lon2 - lon1) / 2) ** 2
    return np.degrees(2 * np.arcsin(np.sqrt(h)))


def pin_row_spacing_is_dlon_on_the_sky():
    geom = {"nx": 60, "ny": 40, "lon0": 200.0, "lat0": 55.0, "dlon": 2 * ARCMIN,
            "dlat": 2 * ARCMIN, "proj": "sfl"}
    lon, lat = oracle.cell_centres(geom)
    lon = lon.reshape(40, 60)
    lat = lat.reshape(40, 60)
    d = _gc_deg(lon[:, :-1], lat[:, :-1], lon[:, 1:], lat[:, 1:])
    # along a parallel the sky spacing of points dlon/cos(lat) apart in RA is
    # dlon up to the parallel's curvature (relative ~(dlon tan(lat))^2 / 24)
    assert np.max(np.abs(d / geom["dlon"] - 1.0)) < 1e-6
    plain = dict(geom, proj="car")
    lp, bp = oracle.cell_centres(plain)
    dp = _gc_deg(lp.reshape(40, 60)[:, :-1], bp.reshape(40, 60)[:, :-1],
                 lp.reshape(40, 60)[:, 1:], bp.reshape(40, 60)[:, 1:])
    assert np.min(np.abs(dp / geom["dlon"] - 1.0)) > 0.3  # cos(lat) ~ 0.5 .. 0.6 there
    # the middle column sits on lon0 in every row
    assert np.allclose(lon[:, 29:31].mean(axis=1), 200.0, atol=1e-9)


def pin_equator_row_matches_plain_grid():
    geom = {"nx": 11, "ny": 3, "lon0": 10.0, "lat0": 0.0, "dlon": ARCMIN, "dlat": ARCMIN}
    a, b = oracle.cell_centres(dict(geom, proj="sfl"))
    c, d = oracle.cell_centres(geom)
    mid = slice(11, 22)
    assert np.allclose(a[mid], c[mid], atol=1e-12) and np.array_equal(b, d)


def pin_sample_at_cell_centre():
    geom = {"nx": 9, "ny": 7, "lon0": 30.0, "lat0": 62.0, "dlon": 20 * ARCMIN,
            "dlat": 20 * ARCMIN, "proj": "sfl"}
    lon, lat = oracle.cell_centres(geom)
    m = 3 * 9 + 7
    v = np.array([[2.5]], np.float32)
    out, W = oracle.Index(lon[m:m + 1], lat[m:m + 1], geom, 3 * ARCMIN).grid(v)
    assert out[m, 0] == pytest.approx(2.5) and W[m] == pytest.approx(1.0)
    assert np.sum(W > 0) == 1


def _wide_case(seed=41, n=6000):
    rng = np.random.default_rng(seed)
    geom = {"nx": 240, "ny": 30, "lon0": 0.5, "lat0": 58.0, "dlon": 3 * ARCMIN,
            "dlat": 3 * ARCMIN, "proj": "sfl"}
    lat = geom["lat0"] + rng.uniform(-0.9, 0.9, n)
    x = rng.uniform(-6.5, 6.5, n)
    lon = (geom["lon0"] + x / np.cos(np.radians(lat))) % 360.0
    return lon, lat, geom, 10 * ARCMIN


def pin_padding_and_index_on_sheared_map():
    lon, lat, geom, fwhm = _wide_case()
    off, idx, w = oracle.neighbours_bruteforce(lon, lat, geom, fwhm)
    ioff, iidx, iw = oracle.Index(lon, lat, geom, fwhm).neighbours()
    assert np.array_equal(off, ioff) and np.array_equal(idx, iidx)
    assert np.max(np.abs(w - iw)) <= 5e-12
    key, perm, boff = oracle.bin_keys(lon, lat, geom, fwhm, bin_cells=2)
    n_bins, lay = oracle.bin_layout(geom, fwhm, bin_cells=2)
    assert np.all(key[np.unique(idx)] < n_bins)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    # the edge columns' discs need more than the plain grid's RA padding
    n_plain, lay_plain = oracle.bin_layout(dict(geom, proj="car"), fwhm, bin_cells=2)
    assert lay[0] > lay_plain[0] * math.cos(math.radians(58.9))


PINS = [pin_row_spacing_is_dlon_on_the_sky, pin_equator_row_matches_plain_grid,
        pin_sample_at_cell_centre, pin_padding_and_index_on_sheared_map]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    oracle.set_mutation(0)
    pin()


def test_planted_mistake_is_caught():
    caught = []
    try:
        oracle.set_mutation(11)  # the projection's cos(lat) dropped
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                caught.append(pin.__name__)
    finally:
        oracle.set_mutation(0)
    assert caught
