"""GPU parity of the Sanson-Flamsteed map geometry (HEGRID_PLAN_SFL) against
the oracle: bin permutation and offsets bit for bit, the neighbour CSR
(modulo the FP64 tie band) and the weights, and the maps of the FP32 and
split tensor-core forms, on a wide sheared map at high latitude across RA 0,
a dense field across RA 0, and a map straddling the equator."""
import numpy as np
import pytest

import oracle
from helpers import csr_diff_in_tie_band, map_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ARCMIN = 1.0 / 60.0
TOL = {"fp32": 1e-5, "tc_split": 5e-5}
WEIGHT_RTOL = 5e-7


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_04584_gb300 import build
    build.build()
    from paper_2207_04584_gb300 import hegrid
    hegrid.lib()
    return hegrid


def _field(name):
    rng = np.random.default_rng({"wide": 41, "dense": 42, "equator": 43}[name])
    if name == "wide":
        geom = {"nx": 240, "ny": 30, "lon0": 0.5, "lat0": 58.0, "dlon": 3 * ARCMIN,
                "dlat": 3 * ARCMIN}
        n, fwhm, xs, ys = 8000, 10 * ARCMIN, 6.5, 0.9
    elif name == "dense":
        geom = {"nx": 64, "ny": 48, "lon0": 359.7, "lat0": 63.0, "dlon": ARCMIN,
                "dlat": ARCMIN}
        n, fwhm, xs, ys = 40000, 3 * ARCMIN, 0.6, 0.45
    else:
        geom = {"nx": 90, "ny": 60, "lon0": 140.0, "lat0": 0.2, "dlon": ARCMIN, "dlat": ARCMIN}
        n, fwhm, xs, ys = 30000, 3 * ARCMIN, 0.8, 0.55
    lat = geom["lat0"] + rng.uniform(-ys, ys, n)
    x = rng.uniform(-xs, xs, n)
    lon = (geom["lon0"] + x / np.cos(np.radians(lat))) % 360.0
    values = rng.normal(1.0, 2.0, (n, 8)).astype(np.float32)
    return lon, lat, geom, fwhm, values


@pytest.mark.parametrize("name", ["wide", "dense", "equator"])
def test_sfl_plan_and_maps(H, name):
    lon, lat, geom, fwhm, values = _field(name)
    N, M = len(lon), geom["nx"] * geom["ny"]
    og = dict(geom, proj="sfl")
    s = torch.cuda.current_stream().cuda_stream
    plan = H.hegrid_plan_create(N, lon, lat, 0, geom, fwhm, 3.0, H.HEGRID_PLAN_SFL, s)
    try:
        info = H.hegrid_plan_info(plan)
        perm = np.zeros(N, np.int32)
        boff = np.zeros(info["n_bins"] + 1, np.int32)
        off = np.zeros(M + 1, np.int64)
        idx = np.zeros(info["n_pairs"], np.int32)
        w = np.zeros(info["n_pairs"], np.float32)
        H.hegrid_plan_export(plan, perm, boff, off, idx, w, None)
        maps = {}
        v = torch.from_numpy(values).cuda()
        for mode, md in (("fp32", H.HEGRID_MODE_FP32), ("tc_split", H.HEGRID_MODE_TC_SPLIT)):
            out = torch.full((M, 8), -7.0, device="cuda")
            H.hegrid_grid(plan, v, H.HEGRID_F32, 8, 8, out, 8, None, md, s)
            torch.cuda.synchronize()
            maps[mode] = out.cpu().numpy()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    _, operm, obin = oracle.bin_keys(lon, lat, og, fwhm, bin_cells=2)
    assert np.array_equal(boff, obin)
    assert np.array_equal(perm, operm)
    ix = oracle.Index(lon, lat, og, fwhm)
    ooff, oidx, ow = ix.neighbours()
    _, _, hR = oracle.kernel_constants(fwhm)
    nd = csr_diff_in_tie_band(off, idx, ooff, oidx, lon, lat, og, hR)
    if nd == 0:
        assert np.array_equal(off, ooff) and np.array_equal(idx, oidx)
        assert np.max(np.abs(w.astype(np.float64) / ow - 1.0)) <= WEIGHT_RTOL
    ref, Wref = ix.grid(values)
    for mode, got in maps.items():
        err, _, _ = map_error(got, ref, Wref)
        assert err <= TOL[mode], (mode, err)
        assert np.array_equal(np.isnan(got), np.isnan(ref))


def test_sfl_flag_checks(H):
    lon, lat, geom, fwhm, _ = _field("equator")
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(H.HegridError):
        H.hegrid_plan_create(len(lon), lon, lat, 0, geom, fwhm, 3.0,
                             H.HEGRID_PLAN_SFL | H.HEGRID_PLAN_HEALPIX(12), s)
    with pytest.raises(H.HegridError):
        H.hegrid_plan_create(len(lon), lon, lat, 0, geom, fwhm, 3.0, 1 << 15, s)
