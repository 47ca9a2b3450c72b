"""GPU parity of the HEALPix binning variant (the paper's own pixelisation,
Sec. 4.1.1) against the oracle: the HEALPix keys, their stable sort and the
table offsets bit for bit; the pairs, weights and maps the same as with map
bins (the binning changes only the candidate search); maps within the
tolerances of the default path.  Fields in the equatorial belt, across the
cap edge z = 2/3 (Dec 41.8), in the south, and across RA = 0."""
import numpy as np
import pytest

import oracle
from helpers import csr_diff_in_tie_band, map_error
from paper_2207_04584_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tc_split": 5e-5}
ARCMIN = 1.0 / 60.0


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_04584_gb300 import build
    build.build()
    from paper_2207_04584_gb300 import hegrid
    hegrid.lib()
    return hegrid


def _plan(H, wl, flags):
    s = torch.cuda.current_stream().cuda_stream
    return H.hegrid_plan_create(len(wl["lon"]), np.ascontiguousarray(wl["lon"]),
                                np.ascontiguousarray(wl["lat"]), 0, wl["geom"], wl["fwhm_deg"],
                                3.0, flags, s)


def _export(H, plan, N, M):
    info = H.hegrid_plan_info(plan)
    perm = np.zeros(N, np.int32)
    bin_off = np.zeros(info["n_bins"] + 1, np.int32)
    off = np.zeros(M + 1, np.int64)
    idx = np.zeros(info["n_pairs"], np.int32)
    w = np.zeros(info["n_pairs"], np.float32)
    wsum = np.zeros(M, np.float32)
    H.hegrid_plan_export(plan, perm, bin_off, off, idx, w, wsum)
    return info, perm, bin_off, off, idx, w, wsum


def _field(seed, n, nx, ny, lon0, lat0, cell=ARCMIN, fwhm=3 * ARCMIN, spread=1.2, C=6):
    rng = np.random.default_rng(seed)
    lon = lon0 + rng.uniform(-0.5 * nx * cell * spread, 0.5 * nx * cell * spread, n)
    lat = lat0 + rng.uniform(-0.5 * ny * cell * spread, 0.5 * ny * cell * spread, n)
    values = rng.normal(1.0, 2.0, (n, C)).astype(np.float32)
    return {"lon": lon % 360.0, "lat": lat, "values": values, "fwhm_deg": fwhm,
            "geom": {"nx": nx, "ny": ny, "lon0": lon0, "lat0": lat0, "dlon": cell, "dlat": cell}}


FIELDS = {
    "belt": (1, dict(n=20000, nx=70, ny=50, lon0=120.0, lat0=20.0)),
    "cap_edge": (2, dict(n=30000, nx=60, ny=90, lon0=200.0, lat0=41.8)),
    "south_cap": (3, dict(n=20000, nx=40, ny=60, lon0=300.0, lat0=-55.0)),
    "ra_zero": (4, dict(n=20000, nx=80, ny=30, lon0=0.3, lat0=41.0)),
}


@pytest.mark.parametrize("name", sorted(FIELDS))
@pytest.mark.parametrize("k", [10, 12, 13])
def test_hpx_keys_pairs_weights(H, name, k):
    seed, kw = FIELDS[name]
    wl = _field(seed, **kw)
    g = wl["geom"]
    N, M = len(wl["lon"]), g["nx"] * g["ny"]
    plan = _plan(H, wl, H.HEGRID_PLAN_HEALPIX(k))
    try:
        info, perm, bin_off, off, idx, w, wsum = _export(H, plan, N, M)
    finally:
        H.hegrid_plan_destroy(plan)
    # keys, stable sort and table offsets: bit for bit
    _, operm, obin = oracle.hpx_keys(wl["lon"], wl["lat"], g, wl["fwhm_deg"], nside=1 << k)
    assert info["n_bins"] == len(obin) - 1
    assert np.array_equal(bin_off, obin)
    assert np.array_equal(perm, operm)
    # the pairs: those of the oracle (modulo the FP64 tie band), and exactly the
    # pairs and weights of the map-bin plan
    ix = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"])
    ooff, oidx, ow = ix.neighbours()
    _, _, hR = oracle.kernel_constants(wl["fwhm_deg"])
    csr_diff_in_tie_band(off, idx, ooff, oidx, wl["lon"], wl["lat"], g, hR)
    plan = _plan(H, wl, 0)
    try:
        _, _, _, boff, bidx, bw, bwsum = _export(H, plan, N, M)
    finally:
        H.hegrid_plan_destroy(plan)
    assert np.array_equal(off, boff) and np.array_equal(idx, bidx)
    assert np.array_equal(w, bw)
    assert np.allclose(wsum, bwsum, rtol=2e-6, atol=0)


@pytest.mark.parametrize("mode", ["fp32", "tc_split"])
def test_hpx_maps_survey_cut(H, mode):
    """A 2 x 20 deg cut of the simulated survey (Dec 31-51, across the cap
    edge) at its density, gridded through the HEALPix variant at nside 4096."""
    wl = W.sim_survey(n=470_000, C=8, lon_span=2.0)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    s = torch.cuda.current_stream().cuda_stream
    md = H.HEGRID_MODE_FP32 if mode == "fp32" else H.HEGRID_MODE_TC_SPLIT
    plan = _plan(H, wl, H.HEGRID_PLAN_HEALPIX(12))
    try:
        v = torch.from_numpy(wl["values"]).cuda()
        out = torch.full((M, 8), -7.0, device="cuda")
        wout = torch.full((M,), -7.0, device="cuda")
        H.hegrid_grid(plan, v, H.HEGRID_F32, 8, 8, out, 8, wout, md, s)
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(wl["values"])
    got = out.cpu().numpy()
    err, _, _ = map_error(got, ref, Wref)
    assert err <= TOL[mode], err
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.allclose(wout.cpu().numpy(), Wref, rtol=2e-5, atol=0)


def test_hpx_flag_checks(H):
    wl = _field(9, n=100, nx=10, ny=10, lon0=10.0, lat0=10.0)
    with pytest.raises(H.HegridError):
        _plan(H, wl, H.HEGRID_PLAN_HEALPIX(14))  # nside above 2^13
    with pytest.raises(H.HegridError):
        _plan(H, wl, 1 << 15)  # an unknown flag bit
    lon = torch.from_numpy(np.ascontiguousarray(wl["lon"])).cuda()
    lat = torch.from_numpy(np.ascontiguousarray(wl["lat"])).cuda()
    perm = torch.empty(100, dtype=torch.int32, device="cuda")
    off = torch.empty(1 << 16, dtype=torch.int32, device="cuda")
    with pytest.raises(H.HegridError):
        H.hegrid_bin_sort_noalloc(100, lon, lat, wl["geom"], wl["fwhm_deg"], 3.0, perm, off,
                                  off.numel(), H.HEGRID_PLAN_HEALPIX(12),
                                  torch.cuda.current_stream().cuda_stream)
