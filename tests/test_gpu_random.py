"""Seeded randomized GPU parity against the oracle: each case draws a map
(size, cell, centre anywhere between -70 and +70 deg of Dec, RA near 0 / 360
or anywhere), a kernel width, a sample pattern (uniform over a field larger or
smaller than the map, or clustered), a channel count spanning every
tensor-core tile width, a bin edge or a HEALPix nside, and the map geometry
(plain or Sanson-Flamsteed), then checks the neighbour CSR (modulo the FP64 tie band),
the weights and the maps of the FP32 and split tensor-core forms."""
import math

import numpy as np
import pytest

import oracle
from helpers import csr_diff_in_tie_band, map_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ARCMIN = 1.0 / 60.0
TOL = {"fp32": 1e-5, "tc_split": 5e-5}


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_04584_gb300 import build
    build.build()
    from paper_2207_04584_gb300 import hegrid
    hegrid.lib()
    return hegrid


def _draw(seed):
    rng = np.random.default_rng(7000 + seed)
    nx, ny = int(rng.integers(5, 70)), int(rng.integers(5, 50))
    cell = float(rng.choice([0.25, 0.5, 1.0, 2.0])) * ARCMIN
    lat0 = float(rng.uniform(-70, 70))
    lon0 = float(rng.choice([0.0, 359.9, rng.uniform(0, 360)]))
    fwhm = float(rng.uniform(1.5, 5.0)) * cell * 2.0
    sfl = bool(rng.uniform() < 0.3)
    C = int(rng.choice([1, 3, 8, 40, 64, 65, 128, 129, 200, 260]))
    bins = int(rng.integers(1, 5))
    spread = float(rng.uniform(0.6, 1.6))
    n = int(rng.integers(200, 8000))
    if rng.uniform() < 0.3:  # clustered: a few dense spots
        k = int(rng.integers(1, 6))
        cx = rng.uniform(-0.5, 0.5, k) * nx * cell
        cy = rng.uniform(-0.5, 0.5, k) * ny * cell
        j = rng.integers(0, k, n)
        x = cx[j] + rng.normal(0, 2 * cell, n)
        y = cy[j] + rng.normal(0, 2 * cell, n)
    else:
        x = rng.uniform(-0.5, 0.5, n) * nx * cell * spread
        y = rng.uniform(-0.5, 0.5, n) * ny * cell * spread
    lat = np.clip(lat0 + y, -89.0, 89.0)
    lon = lon0 + (x / np.cos(np.radians(lat)) if sfl else x)
    values = rng.normal(1.0, 2.0, (n, C)).astype(np.float32)
    geom = {"nx": nx, "ny": ny, "lon0": lon0, "lat0": lat0, "dlon": cell, "dlat": cell}
    hpx = 0 if sfl or rng.uniform() < 0.7 else int(rng.integers(10, 14))
    return lon % 360.0, lat, geom, fwhm, values, sfl, bins, hpx


@pytest.mark.parametrize("seed", range(32))
def test_random_case(H, seed):
    lon, lat, geom, fwhm, values, sfl, bins, hpx = _draw(seed)
    N, C = values.shape
    M = geom["nx"] * geom["ny"]
    og = dict(geom, proj="sfl") if sfl else geom
    flags = H.HEGRID_PLAN_BIN_CELLS(bins) | (H.HEGRID_PLAN_SFL if sfl else 0)
    if hpx:
        flags = H.HEGRID_PLAN_HEALPIX(hpx)
    s = torch.cuda.current_stream().cuda_stream
    ld = (C + 3) // 4 * 4
    vp = np.zeros((N, ld), np.float32)
    vp[:, :C] = values
    plan = H.hegrid_plan_create(N, lon, lat, 0, geom, fwhm, 3.0, flags, s)
    try:
        info = H.hegrid_plan_info(plan)
        off = np.zeros(M + 1, np.int64)
        idx = np.zeros(info["n_pairs"], np.int32)
        w = np.zeros(info["n_pairs"], np.float32)
        H.hegrid_plan_export(plan, None, None, off, idx, w, None)
        v = torch.from_numpy(vp).cuda()
        maps = {}
        for mode, md in (("fp32", H.HEGRID_MODE_FP32), ("tc_split", H.HEGRID_MODE_TC_SPLIT)):
            out = torch.full((M, C), -7.0, device="cuda")
            H.hegrid_grid(plan, v, H.HEGRID_F32, C, ld, out, C, None, md, s)
            torch.cuda.synchronize()
            maps[mode] = out.cpu().numpy()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    ix = oracle.Index(lon, lat, og, fwhm)
    ooff, oidx, ow = ix.neighbours()
    _, _, hR = oracle.kernel_constants(fwhm)
    nd = csr_diff_in_tie_band(off, idx, ooff, oidx, lon, lat, og, hR)
    if nd == 0:
        assert np.array_equal(off, ooff) and np.array_equal(idx, oidx)
        if len(w):
            assert np.max(np.abs(w.astype(np.float64) / ow - 1.0)) <= 5e-7
    ref, Wref = ix.grid(values)
    for mode, got in maps.items():
        assert np.array_equal(np.isnan(got), np.isnan(ref)), mode
        if Wref.max() > 0:
            err, _, _ = map_error(got, ref, Wref)
            assert err <= TOL[mode], (seed, mode, err, dict(C=C, sfl=sfl, bins=bins, hpx=hpx,
                                                            **geom))
    assert not math.isnan(float(info["n_pairs"]))
