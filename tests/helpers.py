"""Comparison helpers shared by the GPU parity tests (no method arithmetic
beyond the error metric and a haversine used only to classify tie pairs)."""
import numpy as np


def map_error(got, ref, W, rel_mask=1e-3):
    """Per-channel error: max |got - ref| / RMS(ref) over cells with W >= rel_mask * max W.

    Returns (max over channels, median over channels, mask)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    W = np.asarray(W, np.float64)
    mask = W >= rel_mask * W.max()
    rms = np.sqrt(np.mean(ref[mask] ** 2, axis=0))
    e = np.max(np.abs(got[mask] - ref[mask]), axis=0) / rms
    return float(e.max()), float(np.median(e)), mask


def pair_set(off, idx):
    cells = np.repeat(np.arange(len(off) - 1), np.diff(off))
    return set(zip(cells.tolist(), np.asarray(idx).tolist()))


def haversine_h(lon_m, lat_m, lon_n, lat_n):
    a = np.radians(lat_n - lat_m)
    b = np.radians(lon_n - lon_m)
    return np.sin(a / 2) ** 2 + np.cos(np.radians(lat_m)) * np.cos(np.radians(lat_n)) * \
        np.sin(b / 2) ** 2


def centres(geom, cells=None):
    """Cell centres (used only to classify tie pairs): the plain grid, or the
    Sanson-Flamsteed grid (lon = lon0 + x / cos(lat)) for geom["proj"] == "sfl"."""
    m = np.arange(geom["nx"] * geom["ny"]) if cells is None else np.asarray(cells)
    ix, iy = m % geom["nx"], m // geom["nx"]
    x = (ix - 0.5 * (geom["nx"] - 1)) * geom["dlon"]
    lat = geom["lat0"] + (iy - 0.5 * (geom["ny"] - 1)) * geom["dlat"]
    if str(geom.get("proj", "")).lower() == "sfl":
        return geom["lon0"] + x / np.cos(np.radians(lat)), lat
    return geom["lon0"] + x, lat


def csr_diff_in_tie_band(off_a, idx_a, off_b, idx_b, lon, lat, geom, hR, cells=None, tau=1e-9):
    """Pairs present in one CSR and not the other; assert each lies within the
    relative tie band |h/hR - 1| <= tau.  Returns the number of such pairs."""
    sa, sb = pair_set(off_a, idx_a), pair_set(off_b, idx_b)
    diff = sa ^ sb
    if diff:
        d = np.array(sorted(diff))
        cm = d[:, 0] if cells is None else np.asarray(cells)[d[:, 0]]
        clon, clat = centres(geom, cm)
        h = haversine_h(clon, clat, lon[d[:, 1]], lat[d[:, 1]])
        bad = np.abs(h / hR - 1.0) > tau
        assert not bad.any(), f"{bad.sum()} membership differences outside the tie band"
    return len(diff)
