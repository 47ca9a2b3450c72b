"""GPU parity of the CUDA path against the FP64 oracle (through the C ABI).

Integer structures (bin permutation, bin offsets, neighbour CSR) are compared
bit for bit; a membership difference is allowed only inside the FP64 tie band
around d = R.  Weights are compared per pair (FP32 from FP64 separations:
a few ulp).  Maps use the error metric: max over channels of
max |gpu - oracle| / RMS(oracle) on cells with W >= 1e-3 max W, with the
tolerance 1e-5 for the FP32 path and 5e-5 for the split tensor-core path.
"""
import numpy as np
import pytest

import oracle
from helpers import csr_diff_in_tie_band, map_error
from paper_2207_04584_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_SPLIT = 5e-5
WEIGHT_RTOL = 5e-7  # ~4 ulp of FP32
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


def _plan(H, wl, flags=0):
    s = torch.cuda.current_stream().cuda_stream
    return H.hegrid_plan_create(len(wl["lon"]), np.ascontiguousarray(wl["lon"]),
                                np.ascontiguousarray(wl["lat"]), 0, wl["geom"], wl["fwhm_deg"],
                                wl.get("support", 3.0), flags, s)


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


def _grid(H, plan, values, M, mode, dtype=None, ld=None):
    dev = torch.device("cuda")
    v = values if isinstance(values, torch.Tensor) else torch.from_numpy(values)
    v = v.to(dev)
    C = v.shape[1] if ld is None else ld
    nch = values.shape[1]
    out = torch.full((M, nch), -7.0, device=dev)
    wout = torch.full((M,), -7.0, device=dev)
    dt = H.HEGRID_F32 if dtype is None else dtype
    H.hegrid_grid(plan, v, dt, nch, v.shape[1] if ld is None else ld, out, nch, wout, mode,
                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    H.hegrid_status_poll(plan)
    del C
    return out.cpu().numpy(), wout.cpu().numpy()


def _case(seed, n=3000, nx=37, ny=21, lon0=45.0, lat0=20.0, cell=ARCMIN, fwhm=3 * ARCMIN, C=5,
          spread=1.3):
    rng = np.random.default_rng(seed)
    lon = lon0 + rng.uniform(-0.5 * nx * cell * spread, 0.5 * nx * cell * spread, n)
    lat = lat0 + rng.uniform(-0.5 * ny * cell * spread, 0.5 * ny * cell * spread, n)
    values = rng.normal(1.0, 2.0, (n, C)).astype(np.float32)
    return {"lon": lon % 360.0, "lat": lat, "values": values, "fwhm_deg": fwhm, "support": 3.0,
            "geom": {"nx": nx, "ny": ny, "lon0": lon0, "lat0": lat0, "dlon": cell, "dlat": cell}}


def check_plan(H, wl, bin_cells=2):
    N = len(wl["lon"])
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    plan = _plan(H, wl, flags=bin_cells if bin_cells != 2 else 0)
    try:
        info, perm, bin_off, off, idx, w, wsum = _export(H, plan, N, M)
    finally:
        H.hegrid_plan_destroy(plan)
    # a2/a3: bit-exact against the oracle's key, stable sort and offsets
    _, operm, obin = oracle.bin_keys(wl["lon"], wl["lat"], g, wl["fwhm_deg"], wl["support"],
                                     bin_cells)
    assert np.array_equal(perm, operm)
    assert np.array_equal(bin_off, obin)
    # a4: CSR bit-exact modulo the tie band
    ix = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"], wl["support"])
    ooff, oidx, ow = ix.neighbours()
    _, _, hR = oracle.kernel_constants(wl["fwhm_deg"], wl["support"])
    nd = csr_diff_in_tie_band(off, idx, ooff, oidx, wl["lon"], wl["lat"], g, hR)
    if nd == 0:
        assert np.array_equal(off, ooff) and np.array_equal(idx, oidx)
        # a5: weights per pair, and W
        rel = np.abs(w.astype(np.float64) / ow - 1.0)
        assert rel.max() <= WEIGHT_RTOL, rel.max()
        Wo = np.add.reduceat(ow, ooff[:-1]) if len(ow) else np.zeros(M)
        Wo[np.diff(ooff) == 0] = 0.0
        has = Wo > 0
        assert np.all(wsum[~has] == 0)
        assert np.max(np.abs(wsum[has] / Wo[has] - 1.0)) <= 2e-6
    return info


@pytest.mark.parametrize("seed,kw", [
    (1, {}),
    (2, {"nx": 16, "ny": 8}),                         # exactly one block
    (3, {"nx": 50, "ny": 9, "lon0": 0.1}),            # straddles RA = 0
    (4, {"nx": 20, "ny": 30, "lat0": -62.0}),         # southern, high |Dec|
    (5, {"n": 1, "nx": 5, "ny": 5}),                  # a single sample
    (6, {"n": 2000, "spread": 4.0}),                  # most samples off the map
    (7, {"cell": 0.5 * ARCMIN, "fwhm": 2.9 * ARCMIN}),
    # dense: a staged chunk's entries overflow the pair kernel's weight buffer,
    # so W is summed over several spans of candidate groups
    (8, {"n": 20000, "nx": 48, "ny": 24, "cell": 0.5 * ARCMIN, "fwhm": 2.9 * ARCMIN,
         "spread": 1.1}),
])
def test_plan_matches_oracle(H, seed, kw):
    check_plan(H, _case(seed, **kw))


def test_plan_keys_on_bin_edges(H):
    """Samples on the exact FP64 bin edges of the key expression and a few ulp
    either side (where floor(RN(RN(x / d) + c)) must come from the correctly
    rounded quotient), and on the RA wrap at lon0 +- 180 deg."""
    wl = _case(21, n=0, nx=37, ny=21)
    g = wl["geom"]
    rng = np.random.default_rng(22)
    lons, lats = [], []
    for k in range(-8, g["nx"] + 8):  # RA edges near and across the map
        e = g["lon0"] + (k - 0.5 * g["nx"]) * g["dlon"]
        for u in range(-3, 4):
            x = e
            for _ in range(abs(u)):
                x = np.nextafter(x, np.inf if u > 0 else -np.inf)
            lons.append(x)
            lats.append(g["lat0"] + rng.uniform(-0.4, 0.4) * g["ny"] * g["dlat"])
    for k in range(-8, g["ny"] + 8):  # Dec edges
        e = g["lat0"] + (k - 0.5 * g["ny"]) * g["dlat"]
        for u in range(-3, 4):
            y = e
            for _ in range(abs(u)):
                y = np.nextafter(y, np.inf if u > 0 else -np.inf)
            lats.append(y)
            lons.append(g["lon0"] + rng.uniform(-0.4, 0.4) * g["nx"] * g["dlon"])
    for d in (180.0, -180.0):  # the RA wrap of the key (off the map)
        e = g["lon0"] + d
        for u in range(-3, 4):
            x = e
            for _ in range(abs(u)):
                x = np.nextafter(x, np.inf if u > 0 else -np.inf)
            lons.append(x)
            lats.append(g["lat0"])
    wl["lon"] = np.asarray(lons, np.float64)
    wl["lat"] = np.asarray(lats, np.float64)
    wl["values"] = np.ones((len(lons), 1), np.float32)
    for bin_cells in (1, 2, 3):
        check_plan(H, wl, bin_cells=bin_cells)


@pytest.mark.parametrize("bin_cells", [1, 4, 7])
def test_plan_bin_sizes(H, bin_cells):
    check_plan(H, _case(11, nx=33, ny=17), bin_cells=bin_cells)


def test_plan_config1(H):
    info = check_plan(H, W.config1())
    assert info["n_pairs"] > 900000


@pytest.mark.parametrize("C", [1, 5, 128, 300])
def test_grid_f32_matches_oracle(H, C):
    wl = _case(21, n=6000, nx=40, ny=24, C=C)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    ld = (C + 3) // 4 * 4
    vals = np.zeros((len(wl["lon"]), ld), np.float32)
    vals[:, :C] = wl["values"]
    plan = _plan(H, wl)
    try:
        v = torch.from_numpy(vals).cuda()
        out = torch.full((M, C), -7.0, device="cuda")
        wout = torch.full((M,), -7.0, device="cuda")
        H.hegrid_grid(plan, v, H.HEGRID_F32, C, ld, out, C, wout, H.HEGRID_MODE_FP32,
                      torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    got, gw = out.cpu().numpy(), wout.cpu().numpy()
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(wl["values"])
    err, _, _ = map_error(got, ref, Wref)
    assert err <= TOL_F32, err
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.allclose(gw, Wref, rtol=2e-6, atol=0)


def test_grid_f32_config1(H):
    wl = W.config1()
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    plan = _plan(H, wl)
    try:
        got, gw = _grid(H, plan, wl["values"], M, H.HEGRID_MODE_FP32)
    finally:
        H.hegrid_plan_destroy(plan)
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(wl["values"])
    err, med, _ = map_error(got, ref, Wref)
    assert err <= TOL_F32, err
    assert np.array_equal(np.isnan(got), np.isnan(ref))


def test_constant_sky_f32(H):
    wl = W.config1(with_values=False)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    v = np.full((len(wl["lon"]), 4), 3.7, np.float32)
    plan = _plan(H, wl)
    try:
        got, gw = _grid(H, plan, v, M, H.HEGRID_MODE_FP32)
    finally:
        H.hegrid_plan_destroy(plan)
    has = gw > 0
    assert np.max(np.abs(got[has] / np.float32(3.7) - 1.0)) <= 1e-6
    assert np.all(np.isnan(got[~has]))


def test_padded_ld_and_offset_map(H):
    """ld_values > C and ld_map > C leave the padding columns untouched."""
    wl = _case(31, n=4000, nx=20, ny=20, C=6)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    vals = np.full((len(wl["lon"]), 12), np.nan, np.float32)
    vals[:, :6] = wl["values"]
    plan = _plan(H, wl)
    try:
        v = torch.from_numpy(vals).cuda()
        out = torch.full((M, 9), -7.0, device="cuda")
        H.hegrid_grid(plan, v, H.HEGRID_F32, 6, 12, out, 9, None, H.HEGRID_MODE_FP32,
                      torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    finally:
        H.hegrid_plan_destroy(plan)
    got = out.cpu().numpy()
    assert np.all(got[:, 6:] == -7.0)
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(wl["values"])
    err, _, _ = map_error(got[:, :6], ref, Wref)
    assert err <= TOL_F32


def test_invalid_arguments(H):
    wl = _case(41, n=100, nx=8, ny=8)
    plan = _plan(H, wl)
    try:
        v = torch.zeros((100, 5), device="cuda")
        out = torch.zeros((64, 5), device="cuda")
        with pytest.raises(H.HegridError) as e:  # ld*4 not a multiple of 16
            H.hegrid_grid(plan, v, H.HEGRID_F32, 5, 5, out, 5, None, H.HEGRID_MODE_FP32)
        assert e.value.status == H.HEGRID_ERR_INVALID_ARG
        with pytest.raises(H.HegridError) as e:  # FP32 mode needs F32 values
            H.hegrid_grid(plan, v, H.HEGRID_BF16, 5, 8, out, 5, None, H.HEGRID_MODE_FP32)
        assert e.value.status == H.HEGRID_ERR_UNSUPPORTED
    finally:
        H.hegrid_plan_destroy(plan)
    polar = _case(42, n=100, nx=8, ny=8, lat0=89.99)
    with pytest.raises(H.HegridError) as e:
        _plan(H, polar)
    assert e.value.status == H.HEGRID_ERR_UNSUPPORTED
