"""The benchmarked configuration itself against the oracle: the FAST-like
drift scan (19 beams, 5 x 5 deg at (30, 41), N = 1,940,838 samples, C = 1024
FP32 channels, a 600 x 600 map at 0.5', FWHM 2.9') through both grid forms in
the launch configuration the benchmark times (device coordinates, dense
1024-channel rows: four 256-channel tensor-core tiles, eight 128-channel FP32
tiles).  Eq. 1 is checked on every 20th map row plus the map's edge rows and
columns (about 19,000 cells, every channel), the weight map on the same cells,
and the plan's pair count against the oracle's count over the whole map."""
import numpy as np
import pytest

import oracle
from helpers import map_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tc_split": 5e-5, "tc_split_dense_a": 5e-5, "tc_split_prescaled": 5e-5}


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_04584_gb300 import build
    build.build()
    from paper_2207_04584_gb300 import hegrid
    hegrid.lib()
    return hegrid


@pytest.fixture(scope="module")
def drift():
    from paper_2207_04584_gb300 import workloads as W
    wl = W.config2()
    g = wl["geom"]
    nx, ny = g["nx"], g["ny"]
    rows = np.unique(np.concatenate([np.arange(0, ny, 20), [1, ny - 2, ny - 1]]))
    cols = np.array([0, 1, nx - 2, nx - 1])
    cells = np.unique(np.concatenate([
        (rows[:, None] * nx + np.arange(nx)[None, :]).ravel(),
        (np.arange(ny)[:, None] * nx + cols[None, :]).ravel()]))
    ix = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"])
    ref, Wref = ix.grid(wl["values"], cells=cells)
    _, P = ix.count()
    return wl, cells, ref, Wref, P


@pytest.fixture(scope="module")
def plan(H, drift):
    wl = drift[0]
    s = torch.cuda.current_stream().cuda_stream
    lon_d = torch.from_numpy(np.ascontiguousarray(wl["lon"])).cuda()
    lat_d = torch.from_numpy(np.ascontiguousarray(wl["lat"])).cuda()
    p = H.hegrid_plan_create(len(wl["lon"]), lon_d, lat_d, 1, wl["geom"], wl["fwhm_deg"], 3.0,
                             0, s)
    yield p
    H.hegrid_plan_destroy(p)


@pytest.mark.parametrize("mode", ["fp32", "tc_split", "tc_split_dense_a", "tc_split_prescaled"])
def test_drift_scan_full_size(H, drift, plan, mode):
    """Both forms; the split form also with dense A tiles (the kernel the
    benchmark's autotuner keeps) and through the prescaled call the benchmark
    step makes (channel maxima computed apart)."""
    wl, cells, ref, Wref, P = drift
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    N, C = wl["values"].shape
    assert (N, C) == (1940838, 1024)
    s = torch.cuda.current_stream().cuda_stream
    md = H.HEGRID_MODE_FP32 if mode == "fp32" else H.HEGRID_MODE_TC_SPLIT
    H.hegrid_plan_set_tuning(plan, H.HEGRID_MODE_TC_SPLIT, 0, 0, 0,
                             3 if mode in ("tc_split_dense_a", "tc_split_prescaled") else 1)
    v = torch.from_numpy(wl["values"]).cuda()
    out = torch.full((M, C), -7.0, device="cuda")
    wout = torch.full((M,), -7.0, device="cuda")
    if mode == "tc_split_prescaled":
        chmax = torch.empty(C, dtype=torch.int32, device="cuda")
        H.hegrid_chan_maxima(v, H.HEGRID_F32, N, C, C, chmax, H.HEGRID_MAXIMA_BESIDE, s)
        H.hegrid_grid_prescaled(plan, v, H.HEGRID_F32, C, C, chmax, out, C, wout, md, s)
    else:
        H.hegrid_grid(plan, v, H.HEGRID_F32, C, C, out, C, wout, md, s)
    torch.cuda.synchronize()
    H.hegrid_status_poll(plan)
    idx = torch.from_numpy(cells).cuda()
    got = out[idx].cpu().numpy()
    gw = wout[idx].cpu().numpy()
    del out, v
    err, med, mask = map_error(got, ref, Wref)
    print(f"drift scan {mode}: {len(cells)} cells x {C} channels, max {err:.3e} "
          f"median {med:.3e}")
    assert err <= TOL[mode], err
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    has = Wref > 0
    assert np.max(np.abs(gw[has] / Wref[has] - 1.0)) <= 2e-5
    assert np.all(gw[~has] == 0)
    info = H.hegrid_plan_info(plan)
    # the oracle's pair count over the whole map (the tie band allows a few)
    assert abs(info["n_pairs"] - P) <= 8, (info["n_pairs"], P)
    assert mask.sum() > 15000
