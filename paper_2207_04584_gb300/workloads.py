"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no gridding arithmetic: it only draws sample positions
(uniform fields and FAST-like 19-beam drift scans, Sec. 2.1) and a sky model
(Gaussian point sources with spectra, a spectral baseline, per-beam offsets
and white noise).  Both the CUDA path and the oracle consume what it returns.

Every generator is deterministic in its seed (numpy PCG64).  Config ``k`` of
the benchmark family uses seed ``SEED_BASE + k``.

The paper's datasets (simulated HDF5 files and FAST observations, Table 2)
are not available; these inputs stand in for them with FAST's scan geometry
(19 beams at 5.74 arcmin spacing, rotated by 23.4 degrees, drifting in RA at
the sidereal rate, Sec. 2.1).
"""
from __future__ import annotations

import concurrent.futures as _cf
import math
import os

import numpy as np

SEED_BASE = 2207045840
ARCMIN = 1.0 / 60.0
ARCSEC = 1.0 / 3600.0


# --------------------------------------------------------------------------
# positions
# --------------------------------------------------------------------------
def uniform_positions(rng, n, lon_range, lat_range):
    lon = rng.uniform(lon_range[0], lon_range[1], n)
    lat = rng.uniform(lat_range[0], lat_range[1], n)
    return lon, lat


def hex19_offsets(spacing_deg, rotation_deg):
    """(dx, dy) offsets in degrees of a 19-beam hexagonal receiver."""
    pts = []
    for q in range(-2, 3):
        for r in range(-2, 3):
            if abs(q) <= 2 and abs(r) <= 2 and abs(q + r) <= 2:
                pts.append((spacing_deg * (q + 0.5 * r), spacing_deg * (r * math.sqrt(3.0) / 2.0)))
    pts = np.array(pts)
    t = math.radians(rotation_deg)
    rot = np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
    return pts @ rot.T


def drift_scan(rng, centre, size_deg, n_passes=7, spacing_arcmin=5.74, rotation_deg=23.4,
               ra_step_arcmin=0.25, jitter_arcsec=2.0, max_samples=None):
    """FAST-like drift scan covering a ``size_deg`` square field.

    Each pass is a set of Dec strips; in a strip the 19 beams drift along RA in
    steps of ``ra_step_arcmin`` (1 s of sidereal drift at 15 arcsec of RA per
    second).  Passes are offset in Dec by 1/n_passes of the track spacing.
    Returns lon, lat (degrees, float64) and the beam id of each sample.
    """
    lon_c, lat_c = centre
    half = 0.5 * size_deg
    off = hex19_offsets(spacing_arcmin * ARCMIN, rotation_deg)
    dy = off[:, 1]
    span = dy.max() - dy.min()
    track = span / 18.0                      # mean Dec spacing between tracks
    strip_step = span + track                # strips tile the Dec axis
    n_ra = int(round(size_deg / (ra_step_arcmin * ARCMIN)))
    ra_t = lon_c - half + (np.arange(n_ra) + 0.5) * ra_step_arcmin * ARCMIN
    lons, lats, beams = [], [], []
    for p in range(n_passes):
        dec0 = lat_c - half - dy.min() + p * track / n_passes
        s = 0
        while dec0 + s * strip_step + dy.min() < lat_c + half:
            base = dec0 + s * strip_step
            for b in range(19):
                la = base + dy[b]
                if la < lat_c - half or la >= lat_c + half:
                    continue
                lo = ra_t + off[b, 0] / math.cos(math.radians(la))
                keep = (lo >= lon_c - half) & (lo < lon_c + half)
                k = int(keep.sum())
                lons.append(lo[keep] + rng.normal(0.0, jitter_arcsec * ARCSEC, k))
                lats.append(np.full(k, la) + rng.normal(0.0, jitter_arcsec * ARCSEC, k))
                beams.append(np.full(k, b, np.int8))
            s += 1
    lon = np.concatenate(lons)
    lat = np.concatenate(lats)
    beam = np.concatenate(beams)
    if max_samples is not None and len(lon) > max_samples:
        sel = np.sort(rng.choice(len(lon), max_samples, replace=False))
        lon, lat, beam = lon[sel], lat[sel], beam[sel]
    return lon, lat, beam


# --------------------------------------------------------------------------
# sky model
# --------------------------------------------------------------------------
def _threads():
    return max(1, min(16, os.cpu_count() or 1))


def _fill_noise(values, seed, sigma, row_offset_fn=None):
    """values[:] = sigma * N(0,1) (+ per-row offsets), chunked over threads."""
    n = values.shape[0]
    nchunk = max(1, min(64, n // 4096 + 1))
    bounds = np.linspace(0, n, nchunk + 1).astype(np.int64)
    seeds = np.random.SeedSequence(seed).spawn(nchunk)

    def work(i):
        a, b = int(bounds[i]), int(bounds[i + 1])
        if b <= a:
            return
        g = np.random.Generator(np.random.PCG64(seeds[i]))
        blk = values[a:b]
        g.standard_normal(out=blk, dtype=np.float32)
        blk *= np.float32(sigma)
        if row_offset_fn is not None:
            blk += row_offset_fn(a, b)

    with _cf.ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(work, range(nchunk)))


def add_sources(values, lon, lat, src_lon, src_lat, src_fwhm_deg, spectra, cut_sigmas=5.0):
    """values[n, :] += profile_s(n) * spectra[s, :] for Gaussian sources.

    The source profile is a flat-sky Gaussian (RA offsets scaled by cos Dec);
    it is truncated at ``cut_sigmas``.  Channel blocks are filled by threads.
    """
    sig = src_fwhm_deg / math.sqrt(8.0 * math.log(2.0))
    order = np.argsort(lat, kind="stable")
    lat_s = lat[order]
    rad = cut_sigmas * sig
    foot = []
    for s in range(len(src_lon)):
        a = np.searchsorted(lat_s, src_lat[s] - rad)
        b = np.searchsorted(lat_s, src_lat[s] + rad, side="right")
        if b <= a:
            continue
        idx = order[a:b]
        dx = (lon[idx] - src_lon[s]) * math.cos(math.radians(src_lat[s]))
        dy = lat[idx] - src_lat[s]
        r2 = dx * dx + dy * dy
        keep = r2 <= rad * rad
        if not keep.any():
            continue
        foot.append((s, idx[keep], np.exp(-0.5 * r2[keep] / (sig * sig)).astype(np.float32)))
    C = values.shape[1]
    nblk = max(1, min(_threads(), C // 16))
    edges = np.linspace(0, C, nblk + 1).astype(np.int64)

    def work(i):
        c0, c1 = int(edges[i]), int(edges[i + 1])
        if c1 <= c0:
            return
        for s, idx, prof in foot:
            values[idx, c0:c1] += prof[:, None] * spectra[s, c0:c1][None, :]

    with _cf.ThreadPoolExecutor(nblk) as ex:
        list(ex.map(work, range(nblk)))


def one_over_f(rng, C, amplitude=1.0, mean=1.0):
    """A 1/f-like baseline along the channel axis (shared by all samples)."""
    if C == 1:
        return np.array([mean], np.float32)
    f = np.fft.rfftfreq(C)
    spec = rng.normal(size=len(f)) + 1j * rng.normal(size=len(f))
    spec[1:] /= np.sqrt(f[1:])
    spec[0] = 0.0
    x = np.fft.irfft(spec, n=C)
    x = x / (np.std(x) + 1e-30) * amplitude * 0.1
    return (mean + x).astype(np.float32)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def _geom(nx, ny, lon0, lat0, cell_deg):
    return {"nx": int(nx), "ny": int(ny), "lon0": float(lon0), "lat0": float(lat0),
            "dlon": float(cell_deg), "dlat": float(cell_deg)}


def config1(seed=SEED_BASE + 1, n=20000, C=4, nx=120, ny=120, with_values=True):
    """Plain FP32, tiny: uniform samples in a 2x2 deg field at (180, 30)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lon, lat = uniform_positions(rng, n, (179.0, 181.0), (29.0, 31.0))
    wl = {"name": "config1-uniform-tiny", "lon": lon, "lat": lat,
          "geom": _geom(nx, ny, 180.0, 30.0, ARCMIN), "fwhm_deg": 3.0 * ARCMIN, "support": 3.0}
    if with_values:
        ns = 20
        src_lon = rng.uniform(179.0, 181.0, ns)
        src_lat = rng.uniform(29.0, 31.0, ns)
        amp = np.exp(rng.uniform(math.log(0.1), math.log(10.0), ns))
        spectra = (amp[:, None] * rng.uniform(0.5, 1.5, (ns, C))).astype(np.float32)
        values = np.empty((n, C), np.float32)
        _fill_noise(values, int(rng.integers(2**62)), 0.05)
        add_sources(values, lon, lat, src_lon, src_lat, 3.0 * ARCMIN, spectra)
        wl["values"] = values
    return wl


def config2(seed=SEED_BASE + 2, C=1024, size_deg=5.0, cell_arcmin=0.5, n_passes=7,
            n_sources=2000, with_values=True, out=None, max_samples=None):
    """FAST-like 19-beam drift scan over a 5x5 deg field at (30, 41), FP32 values.

    ``out`` (optional) is a preallocated float32 [N, C] (e.g. pinned host
    memory); pass ``with_values=False`` first to learn N.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    centre = (30.0, 41.0)
    lon, lat, beam = drift_scan(rng, centre, size_deg, n_passes=n_passes, max_samples=max_samples)
    npx = int(round(size_deg / (cell_arcmin * ARCMIN)))
    wl = {"name": "config2-fast-drift", "lon": lon, "lat": lat, "beam": beam,
          "geom": _geom(npx, npx, centre[0], centre[1], cell_arcmin * ARCMIN),
          "fwhm_deg": 2.9 * ARCMIN, "support": 3.0}
    if not with_values:
        return wl
    n = len(lon)
    vrng = np.random.Generator(np.random.PCG64(seed + 1000))
    half = 0.5 * size_deg
    src_lon = vrng.uniform(centre[0] - half, centre[0] + half, n_sources)
    src_lat = vrng.uniform(centre[1] - half, centre[1] + half, n_sources)
    amp = np.exp(vrng.uniform(math.log(0.1), math.log(10.0), n_sources))
    beta = vrng.uniform(-2.0, 1.0, n_sources)
    nu = np.linspace(1.0, 1.5, C) / 1.25
    spectra = (amp[:, None] * nu[None, :] ** beta[:, None]).astype(np.float32)
    baseline = one_over_f(vrng, C)
    beam_off = vrng.normal(0.0, 0.1, 19).astype(np.float32)
    values = out if out is not None else np.empty((n, C), np.float32)
    assert values.shape == (n, C) and values.dtype == np.float32

    def offsets(a, b):
        return baseline[None, :] + beam_off[beam[a:b]][:, None]

    _fill_noise(values, int(vrng.integers(2**62)), 0.02, offsets)
    add_sources(values, lon, lat, src_lon, src_lat, 2.9 * ARCMIN, spectra)
    wl["values"] = values
    return wl


def config3(seed=SEED_BASE + 3, C=16384, with_values=True):
    """Precision variant: config-1 positions and map, C channels of smooth spectra."""
    base = config1(with_values=False)
    wl = dict(base)
    wl["name"] = "config3-precision"
    if not with_values:
        return wl
    rng = np.random.Generator(np.random.PCG64(seed))
    lon, lat = base["lon"], base["lat"]
    ns = 20
    src_lon = rng.uniform(179.0, 181.0, ns)
    src_lat = rng.uniform(29.0, 31.0, ns)
    amp = np.exp(rng.uniform(math.log(0.1), math.log(10.0), ns))
    x = np.linspace(-1.0, 1.0, C)
    c1 = rng.normal(0, 0.3, ns)
    c2 = rng.normal(0, 0.2, ns)
    spectra = (amp[:, None] * np.exp(c1[:, None] * x[None, :] + c2[:, None] * x[None, :] ** 2)
               ).astype(np.float32)
    values = np.empty((len(lon), C), np.float32)
    _fill_noise(values, int(rng.integers(2**62)), 0.05)
    add_sources(values, lon, lat, src_lon, src_lat, 3.0 * ARCMIN, spectra)
    wl["values"] = values
    return wl


def config4_fields(seed=SEED_BASE + 4, n_fields=64, max_bytes=150e9, n_range=(1e4, 2e6),
                   side_choices=(64, 128, 256, 512, 1024), c_range=(64, 4096)):
    """Parameters of the batched uneven fields (no samples drawn yet).

    Each field's device footprint is estimated (values at their stored width,
    the FP32 map, about 7 bytes per in-radius pair for the plan's weight
    entries and candidate lists, 40 bytes per sample for the rest of the
    plan); while the total exceeds max_bytes the largest field is drawn anew
    (seeded), so the set is found in a few draws.
    """
    rng = np.random.Generator(np.random.PCG64(seed))

    def draw():
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        side = int(side_choices[int(rng.integers(len(side_choices)))])
        cell = float(rng.choice([0.5, 1.0])) * ARCMIN
        lc2 = rng.uniform(math.log2(c_range[0]), math.log2(c_range[1]))
        C = int(2 ** int(round(lc2)))
        dtype = "f32" if rng.uniform() < 0.5 else "bf16"
        fwhm = rng.uniform(2.9, 6.0) * ARCMIN
        pattern = ["drift", "raster", "uniform"][int(rng.integers(3))]
        lon0 = float(rng.uniform(10.0, 350.0))
        lat0 = float(rng.uniform(-60.0, 60.0))
        eb = 4 if dtype == "f32" else 2
        pairs_est = n * math.pi * (3 * fwhm / 2.3548) ** 2 / (cell * cell)
        est = n * C * eb + side * side * C * 4 + pairs_est * 7 + n * 40
        return {"n": n, "side": side, "cell_deg": cell, "C": C, "dtype": dtype,
                "fwhm_deg": fwhm, "pattern": pattern, "lon0": lon0, "lat0": lat0,
                "seed": int(rng.integers(2**62)), "bytes_est": est}

    fields = [draw() for _ in range(n_fields)]
    while sum(f["bytes_est"] for f in fields) > max_bytes:
        big = max(range(n_fields), key=lambda i: fields[i]["bytes_est"])
        fields[big] = draw()
    return fields, sum(f["bytes_est"] for f in fields)


def field_samples(f, with_values=True):
    """Samples of one config-4 field (positions over the map, values FP32)."""
    rng = np.random.Generator(np.random.PCG64(f["seed"]))
    side, cell = f["side"], f["cell_deg"]
    size = side * cell
    centre = (f["lon0"], f["lat0"])
    n = f["n"]
    if f["pattern"] == "uniform":
        lon, lat = uniform_positions(rng, n, (centre[0] - size / 2, centre[0] + size / 2),
                                     (centre[1] - size / 2, centre[1] + size / 2))
        beam = np.zeros(n, np.int8)
    elif f["pattern"] == "raster":
        rows = max(1, int(math.sqrt(n)))
        cols = max(1, n // rows)
        yy, xx = np.meshgrid(np.linspace(-0.5, 0.5, rows, endpoint=False),
                             np.linspace(-0.5, 0.5, cols, endpoint=False), indexing="ij")
        lon = centre[0] + size * xx.ravel() + rng.normal(0, 2 * ARCSEC, rows * cols)
        lat = centre[1] + size * yy.ravel() + rng.normal(0, 2 * ARCSEC, rows * cols)
        beam = np.zeros(len(lon), np.int8)
    else:
        lon, lat, beam = drift_scan(rng, centre, size, n_passes=max(1, min(7, n // 20000 + 1)),
                                    max_samples=n)
    wl = {"name": f"field-{f['pattern']}", "lon": lon, "lat": lat, "beam": beam,
          "geom": _geom(side, side, centre[0], centre[1], cell), "fwhm_deg": f["fwhm_deg"],
          "support": 3.0, "dtype": f["dtype"]}
    if with_values:
        C = f["C"]
        values = np.empty((len(lon), C), np.float32)
        _fill_noise(values, int(rng.integers(2**62)), 0.05)
        ns = 20
        src_lon = rng.uniform(centre[0] - size / 2, centre[0] + size / 2, ns)
        src_lat = rng.uniform(centre[1] - size / 2, centre[1] + size / 2, ns)
        amp = np.exp(rng.uniform(math.log(0.1), math.log(10.0), ns))
        spectra = (amp[:, None] * rng.uniform(0.5, 1.5, (ns, C))).astype(np.float32)
        add_sources(values, lon, lat, src_lon, src_lat, f["fwhm_deg"], spectra)
        wl["values"] = values
    return wl


def config5(seed=SEED_BASE + 5, size_deg=3.3, cell_arcmin=0.5, n_passes=None, target_n=1_000_000):
    """Full-band streaming positions: 19-beam drift over 3.3x3.3 deg at (30, 41).

    Values are drawn per chunk with :func:`config5_chunk`.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    centre = (30.0, 41.0)
    if n_passes is None:
        probe, _, _ = drift_scan(rng, centre, size_deg, n_passes=1)
        n_passes = max(1, int(math.ceil(target_n / max(1, len(probe)))))
        rng = np.random.Generator(np.random.PCG64(seed))
    lon, lat, beam = drift_scan(rng, centre, size_deg, n_passes=n_passes, max_samples=target_n)
    npx = int(round(size_deg / (cell_arcmin * ARCMIN)))
    return {"name": "config5-fullband", "lon": lon, "lat": lat, "beam": beam,
            "geom": _geom(npx, npx, centre[0], centre[1], cell_arcmin * ARCMIN),
            "fwhm_deg": 2.9 * ARCMIN, "support": 3.0}


def config5_chunk(wl, k, C_chunk=4096, seed=SEED_BASE + 5, n_sources=300, out=None):
    """Channel chunk ``k`` (FP32) of the config-5 spectra; sources share positions."""
    lon, lat, beam = wl["lon"], wl["lat"], wl["beam"]
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    g = wl["geom"]
    half = 0.5 * g["nx"] * g["dlon"]
    src_lon = rng.uniform(g["lon0"] - half, g["lon0"] + half, n_sources)
    src_lat = rng.uniform(g["lat0"] - half, g["lat0"] + half, n_sources)
    amp = np.exp(rng.uniform(math.log(0.1), math.log(10.0), n_sources))
    beta = rng.uniform(-2.0, 1.0, n_sources)
    crng = np.random.Generator(np.random.PCG64(seed + 100 + k))
    nu = (1.0 + 0.5 * (k * C_chunk + np.arange(C_chunk)) / (16 * C_chunk)) / 1.25
    spectra = (amp[:, None] * nu[None, :] ** beta[:, None]).astype(np.float32)
    baseline = one_over_f(crng, C_chunk)
    beam_off = rng.normal(0.0, 0.1, 19).astype(np.float32)
    values = out if out is not None else np.empty((len(lon), C_chunk), np.float32)

    def offsets(a, b):
        return baseline[None, :] + beam_off[beam[a:b]][:, None]

    _fill_noise(values, int(crng.integers(2**62)), 0.02, offsets)
    add_sources(values, lon, lat, src_lon, src_lat, 2.9 * ARCMIN, spectra)
    return values


def sim_survey(seed=SEED_BASE + 6, n=19_000_000, C=50, n_sources=1000, with_values=True,
               out=None, lon_span=60.0):
    """The simulated survey of Sec. 5 (Table 2): a 60 x 20 deg map centred on (30, 41),
    ``n`` samples (1.5e7 - 1.9e7 in Tables 3 and 4) of ``C`` = 50 channels, 180 arcsec beam.

    Sample positions are uniform in (lon, lat) over the map; the map has 1 arcmin cells
    (3600 x 1200) and the gridding kernel's FWHM is the beam's.  The positions are i.i.d.,
    so the first ``k`` samples of this set are a ``k``-sample draw of the same workload
    (the benchmark times prefixes of one 1.9e7-sample set).
    Values: Gaussian point sources of the beam's width with power-law spectra, a 1/f-like
    spectral baseline and white noise.  ``out`` (optional) is a preallocated float32
    [n, C] (e.g. pinned host memory).  ``lon_span`` < 60 keeps the first ``lon_span``
    degrees of RA (a smaller field at the same density when ``n`` is scaled with it).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    centre = (0.5 * lon_span, 41.0)
    lon, lat = uniform_positions(rng, n, (0.0, lon_span), (31.0, 51.0))
    beam_deg = 180.0 * ARCSEC
    wl = {"name": "sim-survey-60x20", "lon": lon, "lat": lat,
          "geom": _geom(int(round(lon_span * 60)), 1200, centre[0], centre[1], ARCMIN),
          "fwhm_deg": beam_deg, "support": 3.0}
    if not with_values:
        return wl
    vrng = np.random.Generator(np.random.PCG64(seed + 1000))
    src_lon = vrng.uniform(0.0, lon_span, n_sources)
    src_lat = vrng.uniform(31.0, 51.0, n_sources)
    amp = np.exp(vrng.uniform(math.log(0.1), math.log(10.0), n_sources))
    beta = vrng.uniform(-2.0, 1.0, n_sources)
    nu = np.linspace(1.0, 1.5, C) / 1.25
    spectra = (amp[:, None] * nu[None, :] ** beta[:, None]).astype(np.float32)
    baseline = one_over_f(vrng, C)
    values = out if out is not None else np.empty((n, C), np.float32)
    assert values.shape == (n, C) and values.dtype == np.float32
    _fill_noise(values, int(vrng.integers(2**62)), 0.02, lambda a, b: baseline[None, :])
    add_sources(values, lon, lat, src_lon, src_lat, beam_deg, spectra)
    wl["values"] = values
    return wl
