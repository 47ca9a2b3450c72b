"""Pins of the oracle's HEALPix ring scheme (the paper's pixelisation,
Sec. 4.1.1; Gorski et al. 2005) and of the HEALPix-variant bin layout, each
against what the scheme's definitions fix: pixel centres map back to their own
pixel, pixels are equal in area, rings hold 4i (caps) or 4N (belt) pixels,
named pixels of nside = 1, and the layout keeps every sample that lies within
R of a map cell.  Planted mistakes in the oracle are each caught."""
import math

import numpy as np
import pytest

import oracle
from paper_2207_04584_gb300 import workloads as W

ARCMIN = 1.0 / 60.0


def pin_centres_round_trip():
    for N in (1, 2, 4, 8, 16, 64):
        z, phi = oracle.hpx_centres(N)
        _, _, ip = oracle.hpx_ang2pix(N, z, phi)
        assert np.array_equal(ip, np.arange(12 * N * N)), N


def pin_equal_area():
    """Uniform points on the sphere fall evenly into the 12 N^2 pixels (chi^2 per
    pixel near 1; a misplaced pixel edge moves a finite area between pixels)."""
    rng = np.random.default_rng(11)
    n = 2_000_000
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 360.0, n)
    for N in (2, 4, 8):
        _, _, ip = oracle.hpx_ang2pix(N, z, phi)
        c = np.bincount(ip, minlength=12 * N * N)
        assert c.size == 12 * N * N
        mean = n / (12 * N * N)
        chi2 = float(((c - mean) ** 2 / mean).sum()) / (12 * N * N)
        assert chi2 < 1.3, (N, chi2)


def pin_ring_sizes_and_heights():
    for N in (1, 2, 4, 8):
        z, phi = oracle.hpx_centres(N)
        zs, counts = np.unique(-z, return_counts=True)  # rings from the north
        zs = -zs
        want = [4 * i if i < N else (4 * N if i <= 3 * N else 4 * (4 * N - i))
                for i in range(1, 4 * N)]
        assert list(counts) == want, N
        # z = 2/3 at ring N (the cap/belt edge), 0 at ring 2N, -2/3 at ring 3N
        assert zs[N - 1] == pytest.approx(2.0 / 3.0, abs=1e-15)
        assert zs[2 * N - 1] == pytest.approx(0.0, abs=1e-15)
        assert zs[3 * N - 1] == pytest.approx(-2.0 / 3.0, abs=1e-15)


def pin_named_pixels_nside1():
    z = np.array([0.0, 0.99, -0.99, 0.0])
    phi = np.array([0.0, 10.0, 350.0, 91.0])
    ring, pix, ip = oracle.hpx_ang2pix(1, z, phi)
    # (z=0, phi=0): centre of the first equatorial pixel; near the north pole at
    # phi=10: pixel 0; near the south pole at phi=350: the last pixel; the
    # equator just past 90 deg: the second equatorial pixel
    assert list(ip) == [4, 0, 11, 5]
    assert list(ring) == [2, 1, 3, 2]


def pin_layout_keeps_every_neighbour():
    """Each sample within R of a cell gets a key inside the layout, and its key
    decodes to its own (ring, pixel)."""
    rng = np.random.default_rng(23)
    n = 4000
    geom = {"nx": 40, "ny": 30, "lon0": 359.8, "lat0": 41.2, "dlon": ARCMIN, "dlat": ARCMIN}
    fwhm = 3.0 * ARCMIN
    lon = geom["lon0"] + rng.uniform(-0.5, 0.5, n)
    lat = geom["lat0"] + rng.uniform(-0.45, 0.45, n)
    off, idx, _ = oracle.neighbours_bruteforce(lon, lat, geom, fwhm)
    for nside in (256, 1024, 4096):
        key, perm, boff = oracle.hpx_keys(lon, lat, geom, fwhm, nside=nside)
        n_bins, ring0, tab = oracle.hpx_layout(geom, fwhm, nside=nside)
        assert np.all(key[np.unique(idx)] < n_bins), nside
        assert np.array_equal(perm, np.argsort(key, kind="stable"))
        assert np.array_equal(boff, np.searchsorted(key[perm], np.arange(n_bins + 1)))
        base = np.concatenate([[0], np.cumsum(tab[:, 2])])
        kept = np.nonzero(key < n_bins)[0]
        r = np.searchsorted(base, key[kept], side="right") - 1
        jr = key[kept] - base[r]
        j = (tab[r, 1] + jr) % tab[r, 0]
        ring, pix, _ = oracle.hpx_ang2pix(nside, np.sin(np.radians(lat[kept])), lon[kept])
        assert np.array_equal(ring, ring0 + r) and np.array_equal(pix, j), nside


PINS = [pin_centres_round_trip, pin_equal_area, pin_ring_sizes_and_heights,
        pin_named_pixels_nside1, pin_layout_keeps_every_neighbour]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    oracle.set_mutation(0)
    pin()


def test_layout_spans_cap_edge_and_rejects_pole():
    """The simulated survey's map (Dec 31-51) straddles z = 2/3 (Dec 41.8): its
    layout holds cap rings (4i pixels) and belt rings (4N)."""
    wl = W.sim_survey(n=1000, with_values=False)
    n_bins, ring0, tab = oracle.hpx_layout(wl["geom"], wl["fwhm_deg"], nside=4096)
    N = 4096
    rings = ring0 + np.arange(len(tab))
    assert np.any(rings < N) and np.any(rings > N)
    assert np.array_equal(tab[:, 0], np.where(rings < N, 4 * rings, 4 * N))
    assert n_bins == tab[:, 2].sum()
    with pytest.raises(ValueError):
        oracle.hpx_layout({"nx": 10, "ny": 10, "lon0": 0.0, "lat0": 89.95, "dlon": ARCMIN,
                           "dlat": ARCMIN}, 3 * ARCMIN)


MUTATIONS = {7: "belt centre shift on the wrong rings", 8: "wrong cap edge spacing",
             9: "belt pixel shift on the wrong rings"}


@pytest.mark.parametrize("mutation", sorted(MUTATIONS), ids=list(MUTATIONS.values()))
def test_planted_mistake_is_caught(mutation):
    caught = []
    try:
        oracle.set_mutation(mutation)
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                caught.append(pin.__name__)
    finally:
        oracle.set_mutation(0)
    assert caught, f"no pin caught mutation {MUTATIONS[mutation]}"
