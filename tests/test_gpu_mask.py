"""GPU parity of per-channel masking (hegrid_grid_masked) against the oracle:
NaN and +-Inf values scattered over the channels, a channel with no finite
value, a sample with no finite value; FP32 and split tensor-core forms, FP32
and BF16 values.  Error metric per channel: max |gpu - oracle| / RMS(oracle)
over the cells whose W_c is at least 1e-3 of the channel's largest."""
import numpy as np
import pytest

import oracle

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


def _case(seed=71, n=8000, C=24):
    rng = np.random.default_rng(seed)
    geom = {"nx": 40, "ny": 30, "lon0": 75.0, "lat0": 25.0, "dlon": ARCMIN, "dlat": ARCMIN}
    lon = geom["lon0"] + rng.uniform(-0.4, 0.4, n)
    lat = geom["lat0"] + rng.uniform(-0.3, 0.3, n)
    v = rng.normal(1.0, 2.0, (n, C)).astype(np.float32)
    bad = rng.uniform(size=(n, C)) < 0.05
    v[bad] = np.nan
    v[rng.choice(n, 40), rng.choice(C, 40)] = np.inf
    v[rng.choice(n, 40), rng.choice(C, 40)] = -np.inf
    v[:, 5] = np.nan          # a channel with no finite value
    v[17, :] = np.nan         # a sample with no finite value
    v[::3, 9] = np.nan        # a channel with a third of its samples masked
    return lon, lat, geom, 3.0 * ARCMIN, v


def _err(got, ref, Wc):
    e = []
    for c in range(ref.shape[1]):
        if Wc[:, c].max() <= 0:
            continue
        m = Wc[:, c] >= 1e-3 * Wc[:, c].max()
        rms = np.sqrt(np.mean(ref[m, c] ** 2))
        e.append(np.max(np.abs(got[m, c] - ref[m, c])) / rms)
    return max(e)


@pytest.mark.parametrize("mode", ["fp32", "tc_split"])
@pytest.mark.parametrize("kind", ["f32", "bf16"])
def test_masked_matches_oracle(H, mode, kind):
    if mode == "fp32" and kind == "bf16":
        pytest.skip("the FP32 form takes FP32 values")
    lon, lat, geom, fwhm, v = _case()
    n, C = v.shape
    M = geom["nx"] * geom["ny"]
    s = torch.cuda.current_stream().cuda_stream
    if kind == "bf16":
        vt = torch.from_numpy(v).to(torch.bfloat16)
        ld = (C + 7) // 8 * 8
        dv = torch.zeros((n, ld), dtype=torch.bfloat16, device="cuda")
        dv[:, :C] = vt.cuda()
        up = vt.float().numpy()
        dt = H.HEGRID_BF16
    else:
        ld = C
        dv = torch.from_numpy(v).cuda()
        up = v
        dt = H.HEGRID_F32
    md = H.HEGRID_MODE_FP32 if mode == "fp32" else H.HEGRID_MODE_TC_SPLIT
    plan = H.hegrid_plan_create(n, lon, lat, 0, geom, fwhm, 3.0, 0, s)
    try:
        out = torch.full((M, C), -7.0, device="cuda")
        wc = torch.full((M, C), -7.0, device="cuda")
        H.hegrid_grid_masked(plan, dv, dt, C, ld, out, C, wc, md, s)
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    ref, Wref = oracle.Index(lon, lat, geom, fwhm).grid_masked(np.ascontiguousarray(up))
    got, gwc = out.cpu().numpy(), wc.cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.all(np.isnan(got[:, 5])) and np.all(gwc[:, 5] == 0)
    err = _err(got, ref, Wref)
    assert err <= TOL[mode], err
    has = Wref > 0
    assert np.all(gwc[~has] == 0)
    assert np.max(np.abs(gwc[has] / Wref[has] - 1.0)) <= (2e-6 if mode == "fp32" else 5e-5)


def test_masked_without_invalid_values_is_the_plain_map(H):
    rng = np.random.default_rng(72)
    lon, lat, geom, fwhm, _ = _case()
    v = rng.normal(1.0, 2.0, (len(lon), 8)).astype(np.float32)
    M = geom["nx"] * geom["ny"]
    s = torch.cuda.current_stream().cuda_stream
    plan = H.hegrid_plan_create(len(lon), lon, lat, 0, geom, fwhm, 3.0, 0, s)
    try:
        dv = torch.from_numpy(v).cuda()
        a = torch.empty((M, 8), device="cuda")
        b = torch.empty((M, 8), device="cuda")
        w = torch.empty(M, device="cuda")
        H.hegrid_grid(plan, dv, H.HEGRID_F32, 8, 8, a, 8, w, H.HEGRID_MODE_FP32, s)
        H.hegrid_grid_masked(plan, dv, H.HEGRID_F32, 8, 8, b, 8, None, H.HEGRID_MODE_FP32, s)
        torch.cuda.synchronize()
    finally:
        H.hegrid_plan_destroy(plan)
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(a)
    # the mask pass gives W_c / W = 1 up to the FP32 sum of the weights
    np.testing.assert_allclose(b[ok], a[ok], rtol=2e-6, atol=1e-6)
