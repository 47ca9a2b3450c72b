"""Pins of the oracle's per-channel masking (NaN or Inf values contribute to
neither sum of their channel, so each channel has its own W_c): a non-finite
value of sample k in channel c gives the map of the data with sample k deleted
in that channel and leaves the other channels as they were; the masked sums
over the brute-force neighbour lists (computed here with numpy) agree; a
channel with no finite value is NaN with W_c = 0; a planted mistake (the mask
ignored) is caught."""
import numpy as np
import pytest

import oracle

ARCMIN = 1.0 / 60.0


def _case(seed=31, n=2500, C=4):
    rng = np.random.default_rng(seed)
    geom = {"nx": 24, "ny": 18, "lon0": 150.0, "lat0": 35.0, "dlon": ARCMIN, "dlat": ARCMIN}
    lon = geom["lon0"] + rng.uniform(-0.25, 0.25, n)
    lat = geom["lat0"] + rng.uniform(-0.19, 0.19, n)
    v = rng.normal(1.0, 2.0, (n, C)).astype(np.float32)
    return lon, lat, geom, 3.0 * ARCMIN, v


def pin_nan_equals_deletion():
    lon, lat, geom, fwhm, v = _case()
    rng = np.random.default_rng(5)
    k = rng.choice(len(lon), 60, replace=False)
    vm = v.copy()
    vm[k, 1] = np.nan
    vm[k[:20], 3] = np.inf
    got, Wc = oracle.Index(lon, lat, geom, fwhm).grid_masked(vm)
    full, W = oracle.Index(lon, lat, geom, fwhm).grid(v)
    keep1 = np.setdiff1d(np.arange(len(lon)), k)
    keep3 = np.setdiff1d(np.arange(len(lon)), k[:20])
    d1, W1 = oracle.Index(lon[keep1], lat[keep1], geom, fwhm).grid(v[keep1])
    d3, W3 = oracle.Index(lon[keep3], lat[keep3], geom, fwhm).grid(v[keep3])
    for c, ref, Wr in ((0, full, W), (1, d1, W1), (2, full, W), (3, d3, W3)):
        np.testing.assert_array_equal(np.isnan(got[:, c]), np.isnan(ref[:, c]))
        ok = ~np.isnan(ref[:, c])
        np.testing.assert_allclose(got[ok, c], ref[ok, c], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(Wc[:, c], Wr, rtol=1e-12, atol=0)


def pin_masked_sums_on_bruteforce_lists():
    lon, lat, geom, fwhm, v = _case(seed=32)
    v[::7, 0] = np.nan
    v[::5, 2] = -np.inf
    off, idx, w = oracle.neighbours_bruteforce(lon, lat, geom, fwhm)
    got, Wc = oracle.Index(lon, lat, geom, fwhm).grid_masked(v)
    M = len(off) - 1
    for c in range(v.shape[1]):
        fin = np.isfinite(v[idx, c])
        wv = np.where(fin, w, 0.0)
        cell = np.repeat(np.arange(M), np.diff(off))
        Wr = np.bincount(cell, weights=wv, minlength=M)
        Sr = np.bincount(cell, weights=np.where(fin, w * np.nan_to_num(v[idx, c].astype(np.float64),
                                                                       posinf=0, neginf=0), 0.0),
                         minlength=M)
        with np.errstate(invalid="ignore", divide="ignore"):
            ref = np.where(Wr > 0, Sr / Wr, np.nan)
        np.testing.assert_array_equal(np.isnan(got[:, c]), np.isnan(ref))
        ok = ~np.isnan(ref)
        np.testing.assert_allclose(got[ok, c], ref[ok], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(Wc[:, c], Wr, rtol=1e-10, atol=1e-15)


def pin_all_masked_channel():
    lon, lat, geom, fwhm, v = _case(seed=33, C=3)
    v[:, 2] = np.nan
    got, Wc = oracle.Index(lon, lat, geom, fwhm).grid_masked(v)
    assert np.all(np.isnan(got[:, 2])) and np.all(Wc[:, 2] == 0)
    assert np.any(np.isfinite(got[:, 0]))


PINS = [pin_nan_equals_deletion, pin_masked_sums_on_bruteforce_lists, pin_all_masked_channel]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    oracle.set_mutation(0)
    pin()


def test_planted_mistake_is_caught():
    caught = []
    try:
        oracle.set_mutation(10)  # the mask ignored
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                caught.append(pin.__name__)
    finally:
        oracle.set_mutation(0)
    assert caught
