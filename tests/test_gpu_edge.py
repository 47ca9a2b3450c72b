"""GPU edge cases of the grid kernels against the oracle: chunks whose weight
entries overflow the shared-memory staging (a kernel many cells wide), cell
blocks with no candidates at all (a sparse field), a field across RA = 0."""
import numpy as np
import pytest

import oracle
from helpers import map_error

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


def _run(H, lon, lat, values, geom, fwhm, mode):
    M = geom["nx"] * geom["ny"]
    C = values.shape[1]
    s = torch.cuda.current_stream().cuda_stream
    md = H.HEGRID_MODE_FP32 if mode == "fp32" else H.HEGRID_MODE_TC_SPLIT
    plan = H.hegrid_plan_create(len(lon), lon, lat, 0, geom, fwhm, 3.0, 0, s)
    try:
        v = torch.from_numpy(values).cuda()
        out = torch.full((M, C), -7.0, device="cuda")
        wout = torch.full((M,), -7.0, device="cuda")
        H.hegrid_grid(plan, v, H.HEGRID_F32, C, C, out, C, wout, md, s)
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    ref, Wref = oracle.Index(lon, lat, geom, fwhm).grid(values)
    got = out.cpu().numpy()
    err, _, _ = map_error(got, ref, Wref)
    assert err <= TOL[mode], err
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.allclose(wout.cpu().numpy(), Wref, rtol=2e-5, atol=0)
    return got


@pytest.mark.parametrize("mode", ["fp32", "tc_split"])
def test_wide_kernel_overflows_entry_staging(H, mode):
    """R is ~15 cells, so every candidate reaches all 128 cells of its block:
    4,096 entries per 32-candidate chunk, beyond the staged entry windows."""
    rng = np.random.default_rng(901)
    cell = 0.25 * ARCMIN
    geom = {"nx": 48, "ny": 24, "lon0": 120.0, "lat0": -20.0, "dlon": cell, "dlat": cell}
    n = 6000
    lon = 120.0 + rng.uniform(-0.75, 0.75, n) * 48 * cell
    lat = -20.0 + rng.uniform(-0.75, 0.75, n) * 24 * cell
    values = rng.normal(0.5, 1.0, (n, 12)).astype(np.float32)
    _run(H, lon, lat, values, geom, 3.0 * ARCMIN, mode)


@pytest.mark.parametrize("mode", ["fp32", "tc_split"])
def test_sparse_field_has_empty_blocks(H, mode):
    """Two small clusters in a large map: most cell blocks have no candidate
    and their cells must come out NaN with W = 0."""
    rng = np.random.default_rng(902)
    cell = 1.0 * ARCMIN
    geom = {"nx": 96, "ny": 64, "lon0": 210.0, "lat0": 35.0, "dlon": cell, "dlat": cell}
    a = rng.normal(0.0, 3.0 * ARCMIN, (1500, 2)) + [210.0 - 30 * ARCMIN, 35.0 + 15 * ARCMIN]
    b = rng.normal(0.0, 2.0 * ARCMIN, (1000, 2)) + [210.0 + 25 * ARCMIN, 35.0 - 20 * ARCMIN]
    pts = np.concatenate([a, b])
    values = rng.normal(1.0, 0.5, (len(pts), 20)).astype(np.float32)
    got = _run(H, pts[:, 0].copy(), pts[:, 1].copy(), values, geom, 3.0 * ARCMIN, mode)
    assert np.isnan(got[:, 0]).mean() > 0.8


@pytest.mark.parametrize("mode", ["fp32", "tc_split"])
def test_field_across_ra_zero(H, mode):
    rng = np.random.default_rng(903)
    cell = 0.5 * ARCMIN
    geom = {"nx": 64, "ny": 32, "lon0": 0.05, "lat0": 10.0, "dlon": cell, "dlat": cell}
    n = 8000
    lon = (0.05 + rng.uniform(-0.6, 0.6, n) * 64 * cell) % 360.0
    lat = 10.0 + rng.uniform(-0.6, 0.6, n) * 32 * cell
    values = rng.normal(2.0, 1.0, (n, 8)).astype(np.float32)
    _run(H, lon, lat, values, geom, 2.5 * ARCMIN, mode)


@pytest.mark.parametrize("mode", ["fp32", "tc_split"])
def test_no_sample_reaches_the_map(H, mode):
    """Every sample lies far from the map: no pairs at all, every block empty;
    the map is NaN everywhere and W is 0 (plain and masked calls)."""
    rng = np.random.default_rng(905)
    geom = {"nx": 40, "ny": 20, "lon0": 100.0, "lat0": 10.0, "dlon": ARCMIN, "dlat": ARCMIN}
    n = 500
    lon = 150.0 + rng.uniform(-1, 1, n)
    lat = -30.0 + rng.uniform(-1, 1, n)
    values = rng.normal(size=(n, 8)).astype(np.float32)
    M = geom["nx"] * geom["ny"]
    s = torch.cuda.current_stream().cuda_stream
    md = H.HEGRID_MODE_FP32 if mode == "fp32" else H.HEGRID_MODE_TC_SPLIT
    plan = H.hegrid_plan_create(n, lon, lat, 0, geom, 3 * ARCMIN, 3.0, 0, s)
    try:
        assert H.hegrid_plan_info(plan)["n_pairs"] == 0
        v = torch.from_numpy(values).cuda()
        out = torch.zeros((M, 8), device="cuda")
        wout = torch.full((M,), -7.0, device="cuda")
        H.hegrid_grid(plan, v, H.HEGRID_F32, 8, 8, out, 8, wout, md, s)
        out2 = torch.zeros((M, 8), device="cuda")
        wc = torch.full((M, 8), -7.0, device="cuda")
        H.hegrid_grid_masked(plan, v, H.HEGRID_F32, 8, 8, out2, 8, wc, md, s)
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    assert torch.isnan(out).all() and (wout == 0).all()
    assert torch.isnan(out2).all() and (wc == 0).all()
