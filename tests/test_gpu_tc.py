"""GPU parity of the tcgen05 tensor-core path against the FP64 oracle.

Tolerances (error metric of the FP32 tests): split form 5e-5; the single
BF16 form is reported and only bounded loosely.  For BF16/FP16-stored values
the oracle runs on the stored values upcast exactly, so the error measures the
computation only.
"""
import numpy as np
import pytest

import oracle
from helpers import map_error
from paper_2207_04584_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SPLIT = 5e-5
TOL_SINGLE = 3e-2
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


def _plan(H, wl, kernel=0, flags=0):
    """A plan whose tensor-core calls run `kernel` (0: default, 1: cell-major,
    2: channel-major, 3: cell-major with dense A tiles)."""
    p = H.hegrid_plan_create(len(wl["lon"]), np.ascontiguousarray(wl["lon"]),
                             np.ascontiguousarray(wl["lat"]), 0, wl["geom"], wl["fwhm_deg"],
                             wl.get("support", 3.0), flags,
                             torch.cuda.current_stream().cuda_stream)
    if kernel:
        H.hegrid_plan_set_tuning(p, H.HEGRID_MODE_TC_SPLIT, 0, 0, 0, kernel)
    return p


def _run(H, plan, vdev, dtype, C, ld, M, mode):
    out = torch.full((M, C), -7.0, device="cuda")
    wout = torch.full((M,), -7.0, device="cuda")
    H.hegrid_grid(plan, vdev, dtype, C, ld, out, C, wout, mode,
                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    H.hegrid_status_poll(plan)
    return out.cpu().numpy(), wout.cpu().numpy()


def _case(seed, n=6000, nx=40, ny=24, C=5, lon0=45.0, lat0=20.0, cell=ARCMIN, fwhm=3 * ARCMIN):
    rng = np.random.default_rng(seed)
    lon = lon0 + rng.uniform(-0.65 * nx * cell, 0.65 * nx * cell, n)
    lat = lat0 + rng.uniform(-0.65 * ny * cell, 0.65 * ny * cell, n)
    values = (rng.normal(1.0, 2.0, (n, C))).astype(np.float32)
    return {"lon": lon % 360.0, "lat": lat, "values": values, "fwhm_deg": fwhm, "support": 3.0,
            "geom": {"nx": nx, "ny": ny, "lon0": lon0, "lat0": lat0, "dlon": cell, "dlat": cell}}


def _padded(values, mult):
    n, C = values.shape
    ld = (C + mult - 1) // mult * mult
    v = np.zeros((n, ld), values.dtype)
    v[:, :C] = values
    return v, ld


@pytest.mark.parametrize("mode,tol", [("split", TOL_SPLIT), ("single", TOL_SINGLE)])
def test_tc_f32_config1(H, mode, tol):
    wl = W.config1()
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    md = H.HEGRID_MODE_TC_SPLIT if mode == "split" else H.HEGRID_MODE_TC
    plan = _plan(H, wl)
    try:
        got, gw = _run(H, plan, torch.from_numpy(wl["values"]).cuda(), H.HEGRID_F32, 4, 4, M, md)
    finally:
        H.hegrid_plan_destroy(plan)
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(wl["values"])
    err, med, _ = map_error(got, ref, Wref)
    print(f"tc {mode} config1: max err {err:.3e} median {med:.3e}")
    assert err <= tol, err
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    has = Wref > 0
    wtol = 2e-5 if mode == "split" else 1e-2
    assert np.max(np.abs(gw[has] / Wref[has] - 1.0)) <= wtol


@pytest.mark.parametrize("kernel", [1, 2, 3])
@pytest.mark.parametrize("C", [1, 5, 64, 65, 100, 128, 129, 256, 257, 300])
def test_tc_split_ragged_channels(H, C, kernel):
    """Every channel-tile width (64, 128, 256 cell-major; 128 channel-major)
    and its edges, ragged and full."""
    wl = _case(51, C=C)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    v, ld = _padded(wl["values"], 4)
    plan = _plan(H, wl, kernel)
    try:
        got, _ = _run(H, plan, torch.from_numpy(v).cuda(), H.HEGRID_F32, C, ld, M,
                      H.HEGRID_MODE_TC_SPLIT)
    finally:
        H.hegrid_plan_destroy(plan)
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(wl["values"])
    err, _, _ = map_error(got, ref, Wref)
    assert err <= TOL_SPLIT, err
    assert np.array_equal(np.isnan(got), np.isnan(ref))


@pytest.mark.parametrize("kind", ["bf16", "f16", "bf16x2"])
def test_tc_stored_dtypes(H, kind):
    wl = _case(61, C=24)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    vt = torch.from_numpy(wl["values"])
    if kind == "bf16":
        dv = vt.to(torch.bfloat16)
        ref_vals = dv.float().numpy()
        dt = H.HEGRID_BF16
    elif kind == "f16":
        dv = vt.to(torch.float16)
        ref_vals = dv.float().numpy()
        dt = H.HEGRID_F16
    else:
        hi = vt.to(torch.bfloat16)
        lo = (vt - hi.float()).to(torch.bfloat16)
        dv = torch.stack([hi, lo], dim=-1).contiguous().view(torch.int32)
        ref_vals = wl["values"]
        dt = H.HEGRID_BF16X2
    plan = _plan(H, wl)
    try:
        got, _ = _run(H, plan, dv.contiguous().cuda(), dt, 24, 24, M, H.HEGRID_MODE_TC_SPLIT)
    finally:
        H.hegrid_plan_destroy(plan)
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(
        np.ascontiguousarray(ref_vals))
    err, _, _ = map_error(got, ref, Wref)
    print(f"tc split {kind}: max err {err:.3e}")
    assert err <= TOL_SPLIT, err


def test_tc_constant_sky(H):
    wl = W.config1(with_values=False)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    v = np.full((len(wl["lon"]), 8), 3.7, np.float32)
    plan = _plan(H, wl)
    try:
        got, gw = _run(H, plan, torch.from_numpy(v).cuda(), H.HEGRID_F32, 8, 8, M,
                       H.HEGRID_MODE_TC_SPLIT)
    finally:
        H.hegrid_plan_destroy(plan)
    has = gw > 0
    assert np.max(np.abs(got[has] / np.float32(3.7) - 1.0)) <= 2e-5
    assert np.all(np.isnan(got[~has]))


def test_tc_matches_fp32_path(H):
    """The two GPU forms agree with each other as well as with the oracle."""
    wl = _case(71, n=8000, nx=48, ny=40, C=64)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    plan = _plan(H, wl)
    try:
        vd = torch.from_numpy(wl["values"]).cuda()
        a, wa = _run(H, plan, vd, H.HEGRID_F32, 64, 64, M, H.HEGRID_MODE_FP32)
        b, wb = _run(H, plan, vd, H.HEGRID_F32, 64, 64, M, H.HEGRID_MODE_TC_SPLIT)
    finally:
        H.hegrid_plan_destroy(plan)
    err, _, _ = map_error(b, a.astype(np.float64), wa)
    assert err <= TOL_SPLIT


def test_tc_config3_precision_table(H):
    """Config 3: 16,384 channels on the config-1 geometry, per-dtype error."""
    wl = W.config3()
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    C = wl["values"].shape[1]
    vt = torch.from_numpy(wl["values"])
    plan = _plan(H, wl)
    ix = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"])
    rng = np.random.default_rng(3)
    cells = np.sort(rng.choice(M, 600, replace=False))
    res = {}
    try:
        for kind, dv, dt, md, refv in [
            ("bf16", vt.to(torch.bfloat16), H.HEGRID_BF16, H.HEGRID_MODE_TC_SPLIT, None),
            ("bf16-single", vt.to(torch.bfloat16), H.HEGRID_BF16, H.HEGRID_MODE_TC, None),
            ("f16", vt.to(torch.float16), H.HEGRID_F16, H.HEGRID_MODE_TC_SPLIT, None),
            ("f32-split", vt, H.HEGRID_F32, H.HEGRID_MODE_TC_SPLIT, wl["values"]),
        ]:
            out = torch.empty((M, C), device="cuda")
            H.hegrid_grid(plan, dv.contiguous().cuda(), dt, C, C, out, C, None, md,
                          torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            got = out[torch.from_numpy(cells).cuda()].cpu().numpy()
            if refv is None:
                refv = dv.float().numpy()
            ref, Wref = ix.grid(np.ascontiguousarray(refv), cells=cells)
            err, med, _ = map_error(got, ref, Wref)
            res[kind] = (err, med)
            del out
    finally:
        H.hegrid_plan_destroy(plan)
    print("config3 per-dtype error (max, median):", res)
    assert res["bf16"][0] <= TOL_SPLIT
    assert res["f16"][0] <= TOL_SPLIT
    assert res["f32-split"][0] <= TOL_SPLIT


@pytest.mark.parametrize("scale", [1e6, 1e-5, 1e30, 1e-30])
def test_tc_split_out_of_fp16_range(H, scale):
    """Values far outside FP16's range are brought into it by the per-channel
    power-of-two scale (every channel scaled alike here)."""
    wl = _case(81, C=16)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    vals = (wl["values"].astype(np.float64) * scale).astype(np.float32)
    plan = _plan(H, wl)
    try:
        got, _ = _run(H, plan, torch.from_numpy(vals).cuda(), H.HEGRID_F32, 16, 16, M,
                      H.HEGRID_MODE_TC_SPLIT)
    finally:
        H.hegrid_plan_destroy(plan)
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(vals)
    err, _, _ = map_error(got, ref, Wref)
    print(f"values x {scale}: {err:.3e}")
    assert err <= TOL_SPLIT, err


def test_tc_split_huge_outliers(H):
    """A few samples 1e5 times brighter than the rest set their channels' scales,
    so every other value sits ~17 binades below its channel's largest.

    Cells that touch a huge sample are dominated by it: they are checked
    relative to their own magnitude.  Every other cell must meet the split
    tolerance."""
    wl = _case(82, C=16)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    vals = wl["values"].copy()
    rng = np.random.default_rng(5)
    hot = rng.choice(len(vals), 40, replace=False)
    vals[hot] *= 1e5
    plan = _plan(H, wl)
    try:
        got, _ = _run(H, plan, torch.from_numpy(vals).cuda(), H.HEGRID_F32, 16, 16, M,
                      H.HEGRID_MODE_TC_SPLIT)
    finally:
        H.hegrid_plan_destroy(plan)
    ix = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"])
    ref, Wref = ix.grid(vals)
    off, idx, _ = ix.neighbours()
    cells = np.repeat(np.arange(M), np.diff(off))
    hot_cell = np.zeros(M, bool)
    hot_cell[cells[np.isin(idx, hot)]] = True
    cold = ~hot_cell & (Wref > 0)
    err, _, _ = map_error(got[cold], ref[cold], Wref[cold])
    assert err <= TOL_SPLIT, err
    h = hot_cell & (Wref >= 1e-3 * Wref.max())
    rel = np.abs(got[h] - ref[h]) / np.abs(ref[h]).max(axis=0)
    assert rel.max() <= 2.0 ** -18, rel.max()


@pytest.mark.parametrize("C", [40, 120])
def test_tc_narrow_tiles_bf16_and_batch(H, C):
    """The 64- and 128-channel tiles on BF16 values, and a batch mixing all
    three tile widths in one call (one launch per width)."""
    wl = _case(61, C=C)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    vb = torch.from_numpy(wl["values"]).to(torch.bfloat16)
    ld = (C + 7) // 8 * 8
    vdev = torch.zeros((len(wl["lon"]), ld), dtype=torch.bfloat16, device="cuda")
    vdev[:, :C] = vb.cuda()
    up = vb.float().numpy()
    plan = _plan(H, wl)
    try:
        got, _ = _run(H, plan, vdev, H.HEGRID_BF16, C, ld, M, H.HEGRID_MODE_TC_SPLIT)
        # the same plan three times in one batch, at 40/120/300 channels
        wide = np.ascontiguousarray(np.tile(wl["values"], (1, -(-300 // C)))[:, :300])
        outs, args = [], []
        for c in (40, 120, 300):
            v = torch.from_numpy(_padded(wide[:, :c], 4)[0]).cuda()
            o = torch.full((M, c), -7.0, device="cuda")
            outs.append((v, o, c))
            args.append({"values": v, "dtype": H.HEGRID_F32, "n_channels": c,
                         "ld_values": v.shape[1], "map_out": o, "ld_map": c, "weight_out": None,
                         "mode": H.HEGRID_MODE_TC_SPLIT})
        H.hegrid_grid_batched([plan] * 3, args, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    ix = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"])
    ref, Wref = ix.grid(np.ascontiguousarray(up))
    err, _, _ = map_error(got, ref, Wref)
    assert err <= TOL_SPLIT, err
    ref3, W3 = ix.grid(wide)
    for v, o, c in outs:
        err, _, _ = map_error(o.cpu().numpy(), ref3[:, :c], W3)
        assert err <= TOL_SPLIT, (c, err)


def _stored(kind, vals, H):
    """(device tensor, dtype, ld, values the oracle sees) for values stored as `kind`."""
    n, C = vals.shape
    vt = torch.from_numpy(vals)
    if kind == "f32":
        v, ld = _padded(vals, 4)
        return torch.from_numpy(v).cuda(), H.HEGRID_F32, ld, vals
    if kind in ("bf16", "f16"):
        ld = (C + 7) // 8 * 8
        tdt = torch.bfloat16 if kind == "bf16" else torch.float16
        dv = torch.zeros((n, ld), dtype=tdt)
        dv[:, :C] = vt.to(tdt)
        return dv.cuda(), (H.HEGRID_BF16 if kind == "bf16" else H.HEGRID_F16), ld, \
            np.ascontiguousarray(dv[:, :C].float().numpy())
    hi = vt.to(torch.bfloat16)
    lo = (vt - hi.float()).to(torch.bfloat16)
    ld = (C + 3) // 4 * 4
    pair = torch.zeros((n, ld, 2), dtype=torch.bfloat16)
    pair[:, :C, 0] = hi
    pair[:, :C, 1] = lo
    stored = (hi.double() + lo.double()).numpy()  # exact: hi + lo is an FP32 value
    return pair.view(torch.int32).reshape(n, ld).cuda(), H.HEGRID_BF16X2, ld, \
        np.ascontiguousarray(stored.astype(np.float32))


@pytest.mark.parametrize("kernel", [1, 2, 3])
@pytest.mark.parametrize("kind", ["f32", "bf16x2", "bf16", "f16"])
@pytest.mark.parametrize("C", [50, 100, 300])
def test_tc_split_mixed_channel_scales(H, kind, C, kernel):
    """Eq. 1 holds per channel: a faint channel must keep the split form's
    accuracy relative to its own RMS when it shares a channel tile (64, 128 or
    256 wide, by C) with channels many decades brighter.  Channel c is scaled
    by 10^(c mod 11 - 6) (10^(c mod 7 - 4) for FP16 storage, whose range is
    narrower), so every tile mixes 1e-6 .. 1e4 (1e-4 .. 1e2)."""
    wl = _case(91 + C, n=6000, C=C)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    e = (np.arange(C) % 7 - 4) if kind == "f16" else (np.arange(C) % 11 - 6)
    vals = (wl["values"].astype(np.float64) * 10.0 ** e[None, :]).astype(np.float32)
    dv, dt, ld, seen = _stored(kind, vals, H)
    plan = _plan(H, wl, kernel)
    try:
        got, gw = _run(H, plan, dv, dt, C, ld, M, H.HEGRID_MODE_TC_SPLIT)
    finally:
        H.hegrid_plan_destroy(plan)
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(seen)
    err, med, _ = map_error(got, ref, Wref)
    print(f"mixed scales {kind} C={C}: max {err:.3e} median {med:.3e}")
    assert err <= TOL_SPLIT, err
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    has = Wref > 0
    assert np.max(np.abs(gw[has] / Wref[has] - 1.0)) <= 2e-5


@pytest.mark.parametrize("C", [100, 300])
@pytest.mark.parametrize("kind", ["f32", "bf16x2", "bf16", "f16"])
@pytest.mark.parametrize("mode", ["split", "single"])
def test_channel_major_equals_cell_major(H, C, kind, mode):
    """The channel-major kernel (values as the MMA's A operand in tensor memory,
    weights from the plan's dense tiles) forms the same products as the
    cell-major kernel and adds them in the same segments; only the tensor
    core's internal summation order differs with the MMA shape.  So the maps
    agree to a few units of FP32 rounding relative to each channel's RMS,
    with the same NaN pattern, and the weight maps (the plan's) are equal; a
    repeated cell-major call is bit-identical to the first."""
    wl = _case(71 + C, n=9000, nx=56, ny=32, C=C)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    dv, dt, ld, _ = _stored(kind, wl["values"], H)
    md = H.HEGRID_MODE_TC_SPLIT if mode == "split" else H.HEGRID_MODE_TC
    maps = []
    plan = _plan(H, wl)
    try:
        for kernel in (1, 2, 1):
            H.hegrid_plan_set_tuning(plan, md, -4, 16, 0, kernel)
            maps.append(_run(H, plan, dv, dt, C, ld, M, md))
    finally:
        H.hegrid_plan_destroy(plan)
    (a, wa), (b, wb), (c, wc) = maps
    assert np.array_equal(a, c, equal_nan=True)
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(a[:, 0])
    rms = np.sqrt(np.mean(a[ok].astype(np.float64) ** 2, axis=0))
    diff = np.max(np.abs(a[ok].astype(np.float64) - b[ok]), axis=0) / rms
    assert diff.max() <= 2e-6, diff.max()
    assert np.array_equal(wa, wb) and np.array_equal(wa, wc)


@pytest.mark.parametrize("C", [40, 100, 300])
@pytest.mark.parametrize("kind", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("mode", ["split", "single"])
@pytest.mark.parametrize("tiles", ["first call", "plan flag"])
def test_dense_a_tiles_equal_built_a_tiles(H, C, kind, mode, tiles):
    """The cell-major kernel with its A tiles copied from the plan's dense
    weight tiles (kernel 3) multiplies exactly the A tiles its A builders would
    assemble from the entries (kernel 1), at every channel-tile width (64 with
    two sub-chunks per chunk, 128, 256), whether the tiles were built by the
    first call that needs them or by plan creation (HEGRID_PLAN_DENSE_TILES):
    maps and weight maps equal bit for bit."""
    wl = _case(131 + C, n=9000, nx=56, ny=32, C=C)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    dv, dt, ld, _ = _stored(kind, wl["values"], H)
    md = H.HEGRID_MODE_TC_SPLIT if mode == "split" else H.HEGRID_MODE_TC
    plan = _plan(H, wl, flags=H.HEGRID_PLAN_DENSE_TILES if tiles == "plan flag" else 0)
    try:
        H.hegrid_plan_set_tuning(plan, md, -4, 16, 0, 1)
        a, wa = _run(H, plan, dv, dt, C, ld, M, md)
        H.hegrid_plan_set_tuning(plan, md, -4, 16, 0, 3)
        b, wb = _run(H, plan, dv, dt, C, ld, M, md)
    finally:
        H.hegrid_plan_destroy(plan)
    assert np.array_equal(a, b, equal_nan=True)
    assert np.array_equal(wa, wb)


@pytest.mark.parametrize("binning", ["map bins", "healpix", "sfl"])
@pytest.mark.parametrize("kernel", [2, 3])
def test_plan_written_tiles_equal_first_call_tiles(H, binning, kernel):
    """Dense weight tiles written by plan creation (HEGRID_PLAN_DENSE_TILES:
    the pair kernel in two halves on two streams, each half's tiles built after
    it) give the same maps, bit for bit, as the tiles the first grid call
    builds, under each binning and for both kernels that read them; the flag
    adds the tiles' bytes to the plan's device memory."""
    wl = _case(171, n=9000, nx=56, ny=32, C=148)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    base = {"map bins": 0, "healpix": H.HEGRID_PLAN_HEALPIX(12), "sfl": H.HEGRID_PLAN_SFL}[binning]
    vd = torch.from_numpy(wl["values"]).cuda()
    res = []
    for flags in (base, base | H.HEGRID_PLAN_DENSE_TILES):
        plan = _plan(H, wl, kernel, flags)
        try:
            info = H.hegrid_plan_info(plan)
            res.append(_run(H, plan, vd, H.HEGRID_F32, 148, 148, M, H.HEGRID_MODE_TC_SPLIT)
                       + (info,))
            assert H.hegrid_status_poll(plan) == H.HEGRID_OK
        finally:
            H.hegrid_plan_destroy(plan)
    (a, wa, ia), (b, wb, ib) = res
    assert np.array_equal(a, b, equal_nan=True)
    assert np.array_equal(wa, wb)
    assert ib["bytes"] > ia["bytes"]
    og = dict(g, proj="sfl") if binning == "sfl" else g
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], og, wl["fwhm_deg"]).grid(wl["values"])
    err, _, _ = map_error(b, ref, Wref)
    assert err <= TOL_SPLIT, err


def test_plan_tiles_split_launch_matches_single_launch_plan(H):
    """With HEGRID_PLAN_DENSE_TILES the pair kernel runs as two launches (the
    block halves, on two streams): the exported plan (CSR, weights, W) equals
    the plan of one launch bit for bit, on an odd block count."""
    wl = _case(181, n=7000, nx=72, ny=40, C=4)  # 5 x 5 blocks of 16 x 8 cells
    out = []
    for flags in (0, H.HEGRID_PLAN_DENSE_TILES):
        plan = _plan(H, wl, 0, flags)
        try:
            info = H.hegrid_plan_info(plan)
            N = len(wl["lon"])
            M = wl["geom"]["nx"] * wl["geom"]["ny"]
            nb_off = np.zeros(M + 1, np.int64)
            nb_idx = np.zeros(info["n_pairs"], np.int32)
            nb_w = np.zeros(info["n_pairs"], np.float32)
            wgt = np.zeros(M, np.float32)
            H.hegrid_plan_export(plan, None, None, nb_off, nb_idx, nb_w, wgt)
            out.append((info["n_blocks"], nb_off, nb_idx, nb_w, wgt))
        finally:
            H.hegrid_plan_destroy(plan)
    assert out[0][0] == 25 and out[1][0] == 25
    for x, y in zip(out[0][1:], out[1][1:]):
        assert np.array_equal(x, y)
