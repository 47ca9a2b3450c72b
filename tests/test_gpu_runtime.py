"""GPU tests of the batching and streaming runtime (many fields in one
persistent launch, the CUDA-graph batch, host-chunk streaming with
copy/compute overlap) against single-field calls and the oracle."""
import numpy as np
import pytest

import oracle
from helpers import map_error
from paper_2207_04584_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_SPLIT = 5e-5


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_04584_gb300 import build
    build.build()
    from paper_2207_04584_gb300 import hegrid
    hegrid.lib()
    return hegrid


def _fields(n_fields=6, seed=W.SEED_BASE + 204):
    """A scaled-down config-4 batch: uneven N, map sizes, channels (tensor-core
    tiles of every width: 64, 128 and 256 channels), dtypes."""
    fields, _ = W.config4_fields(seed=seed, n_fields=n_fields, max_bytes=4e9,
                                 n_range=(2e3, 3e4), side_choices=(24, 40, 64),
                                 c_range=(4, 512))
    return [W.field_samples(f) for f in fields]


def _plan(H, wl):
    return H.hegrid_plan_create(len(wl["lon"]), np.ascontiguousarray(wl["lon"]),
                                np.ascontiguousarray(wl["lat"]), 0, wl["geom"], wl["fwhm_deg"],
                                3.0, 0, torch.cuda.current_stream().cuda_stream)


def _dev_values(wl, dtype_name):
    v = torch.from_numpy(wl["values"])
    C = v.shape[1]
    if dtype_name == "bf16":
        ld = (C + 7) // 8 * 8
        d = torch.zeros((v.shape[0], ld), dtype=torch.bfloat16)
        d[:, :C] = v.to(torch.bfloat16)
        ref = d[:, :C].float().numpy()
    else:
        ld = (C + 3) // 4 * 4
        d = torch.zeros((v.shape[0], ld), dtype=torch.float32)
        d[:, :C] = v
        ref = wl["values"]
    return d.cuda(), ld, np.ascontiguousarray(ref)


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("kernels", ["default", "mixed"])
def test_batched_uneven_fields(H, use_graph, kernels):
    """A batch of uneven fields against the oracle; "mixed": the fields' plans
    tuned in turn to the three tensor-core kernels (cell-major, cell-major with
    dense A tiles, channel-major), so one batch (and one graph) holds all of
    them and the dense tiles are built before the capture."""
    wls = _fields()
    plans, args, refs, outs = [], [], [], []
    n_f32 = 0
    try:
        for i, wl in enumerate(wls):
            plans.append(_plan(H, wl))
            if kernels == "mixed":
                H.hegrid_plan_set_tuning(plans[-1], H.HEGRID_MODE_TC_SPLIT, 0, 0, 0, [1, 3, 2][i % 3])
            C = wl["values"].shape[1]
            M = wl["geom"]["nx"] * wl["geom"]["ny"]
            dv, ld, refv = _dev_values(wl, wl["dtype"])
            out = torch.full((M, C), -7.0, device="cuda")
            wout = torch.full((M,), -7.0, device="cuda")
            mode = H.HEGRID_MODE_TC_SPLIT
            if wl["dtype"] == "f32":
                mode = H.HEGRID_MODE_FP32 if n_f32 % 2 == 0 else H.HEGRID_MODE_TC_SPLIT
                n_f32 += 1
            dt = H.HEGRID_BF16 if wl["dtype"] == "bf16" else H.HEGRID_F32
            args.append({"values": dv, "dtype": dt, "n_channels": C, "ld_values": ld,
                         "map_out": out, "ld_map": C, "weight_out": wout, "mode": mode})
            outs.append((out, wout, dv))
            refs.append(refv)
        s = torch.cuda.current_stream().cuda_stream
        if use_graph:
            batch = H.hegrid_batch_create(plans, args, s)
            try:
                for _ in range(2):  # replays are idempotent
                    for o, w, _ in outs:
                        o.fill_(-7.0)
                    H.hegrid_batch_launch(batch, s)
                    torch.cuda.synchronize()
            finally:
                H.hegrid_batch_destroy(batch)
        else:
            H.hegrid_grid_batched(plans, args, s)
            torch.cuda.synchronize()
        for p in plans:
            H.hegrid_status_poll(p)
        for wl, a, (o, w, _), refv in zip(wls, args, outs, refs):
            ref, Wref = oracle.Index(wl["lon"], wl["lat"], wl["geom"], wl["fwhm_deg"]).grid(refv)
            got = o.cpu().numpy()
            err, _, _ = map_error(got, ref, Wref)
            tol = TOL_F32 if a["mode"] == H.HEGRID_MODE_FP32 else TOL_SPLIT
            assert err <= tol, (wl["name"], a["mode"], err)
            assert np.array_equal(np.isnan(got), np.isnan(ref))
    finally:
        for p in plans:
            H.hegrid_plan_destroy(p)


@pytest.mark.parametrize("mode", ["fp32", "tc_split"])
def test_stream_host_chunks(H, mode):
    """Config-5 shape at small scale: channel chunks in pinned host memory."""
    wl = W.config5(size_deg=0.4, target_n=60000)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    n_chunks, cc = 5, 12
    chunks = [W.config5_chunk(wl, k, C_chunk=cc) for k in range(n_chunks)]
    host = [torch.from_numpy(c).pin_memory() for c in chunks]
    hmap = torch.full((M, n_chunks * cc + 3), -7.0).pin_memory()
    hw = torch.zeros(M).pin_memory()
    md = H.HEGRID_MODE_FP32 if mode == "fp32" else H.HEGRID_MODE_TC_SPLIT
    plan = _plan(H, wl)
    try:
        H.hegrid_grid_stream(plan, host, cc, H.HEGRID_F32, md, hmap, n_chunks * cc + 3, hw)
    finally:
        H.hegrid_plan_destroy(plan)
    allv = np.ascontiguousarray(np.concatenate(chunks, axis=1))
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(allv)
    got = hmap.numpy()
    err, _, _ = map_error(got[:, :n_chunks * cc], ref, Wref)
    assert err <= (TOL_F32 if mode == "fp32" else TOL_SPLIT), err
    assert np.all(got[:, n_chunks * cc:] == -7.0)
    assert np.allclose(hw.numpy(), Wref, rtol=2e-5, atol=0)


def test_stream_matches_device_call(H):
    """Streaming the channels in chunks gives the device call's map bit for bit
    (same kernels, same per-chunk tiles)."""
    wl = W.config1(n=8000, C=64, nx=48, ny=48)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    plan = _plan(H, wl)
    try:
        s = torch.cuda.current_stream().cuda_stream
        out = torch.empty((M, 64), device="cuda")
        H.hegrid_grid(plan, torch.from_numpy(wl["values"]).cuda(), H.HEGRID_F32, 64, 64, out, 64,
                      None, H.HEGRID_MODE_FP32, s)
        torch.cuda.synchronize()
        chunks = [torch.from_numpy(np.ascontiguousarray(wl["values"][:, k * 16:(k + 1) * 16]))
                  .pin_memory() for k in range(4)]
        hmap = torch.empty((M, 64)).pin_memory()
        H.hegrid_grid_stream(plan, chunks, 16, H.HEGRID_F32, H.HEGRID_MODE_FP32, hmap, 64)
    finally:
        H.hegrid_plan_destroy(plan)
    a, b = out.cpu().numpy(), hmap.numpy()
    assert np.array_equal(np.isnan(a), np.isnan(b))
    assert np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])


@pytest.mark.parametrize("dtype,cc,n_chunks", [("f32", 50, 1), ("f32", 13, 3), ("bf16", 13, 2)])
def test_stream_unaligned_rows(H, dtype, cc, n_chunks):
    """Host chunks whose rows are not a multiple of 16 bytes (200, 52 and 26
    bytes: each width of the row repack) stream to the map the device call
    makes from the same values in padded rows, bit for bit."""
    wl = W.config1(n=9000, C=cc * n_chunks, nx=40, ny=40)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    N = len(wl["lon"])
    C = cc * n_chunks
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    hdt = H.HEGRID_F32 if dtype == "f32" else H.HEGRID_BF16
    vals = torch.from_numpy(wl["values"]).to(tdt)
    chunks = [vals[:, k * cc:(k + 1) * cc].contiguous().pin_memory() for k in range(n_chunks)]
    eb = 4 if dtype == "f32" else 2
    ld = (cc * eb + 15) // 16 * 16 // eb
    plan = _plan(H, wl)
    try:
        s = torch.cuda.current_stream().cuda_stream
        ref = torch.empty((M, C), device="cuda")
        for k in range(n_chunks):
            dv = torch.zeros((N, ld), dtype=tdt, device="cuda")
            dv[:, :cc] = chunks[k].cuda()
            H.hegrid_grid(plan, dv, hdt, cc, ld, ref[:, k * cc:], C, None,
                          H.HEGRID_MODE_TC_SPLIT, s)
        torch.cuda.synchronize()
        hmap = torch.full((M, C), -7.0).pin_memory()
        H.hegrid_grid_stream(plan, chunks, cc, hdt, H.HEGRID_MODE_TC_SPLIT, hmap, C)
    finally:
        H.hegrid_plan_destroy(plan)
    a, b = ref.cpu().numpy(), hmap.numpy()
    assert np.array_equal(np.isnan(a), np.isnan(b))
    assert np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("kind", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("beside", [False, True])
def test_grid_prescaled_overlapped_with_plan(H, kernel, kind, beside):
    """The channel maxima computed on a second stream while the plan is built
    (hegrid_chan_maxima, the full pass or the one-CTA-per-SM pass of
    HEGRID_MAXIMA_BESIDE), then hegrid_grid_prescaled: the maxima are each
    channel's largest |v| bit for bit, and the map and weight map equal
    hegrid_grid's element for element, for both tensor-core kernels."""
    wl = W.config1(n=15000, C=300, nx=70, ny=50)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    C = 300
    vt = torch.from_numpy(wl["values"])
    dt = {"f32": (torch.float32, H.HEGRID_F32), "bf16": (torch.bfloat16, H.HEGRID_BF16),
          "f16": (torch.float16, H.HEGRID_F16)}[kind]
    ld = 304
    v = torch.zeros((len(wl["lon"]), ld), dtype=dt[0])
    v[:, :C] = vt.to(dt[0])
    v = v.cuda()
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    chmax = torch.empty(C, dtype=torch.int32, device="cuda")
    ready = torch.cuda.Event()
    ready.record(main)
    side.wait_event(ready)
    H.hegrid_chan_maxima(v, dt[1], v.shape[0], C, ld, chmax,
                         H.HEGRID_MAXIMA_BESIDE if beside else 0, side.cuda_stream)
    done = torch.cuda.Event()
    done.record(side)
    plan = H.hegrid_plan_create(len(wl["lon"]), np.ascontiguousarray(wl["lon"]),
                                np.ascontiguousarray(wl["lat"]), 0, g, wl["fwhm_deg"], 3.0, 0,
                                main.cuda_stream)
    try:
        H.hegrid_plan_set_tuning(plan, H.HEGRID_MODE_TC_SPLIT, 0, 0, 0, kernel)
        main.wait_event(done)
        a = torch.full((M, C), -7.0, device="cuda")
        wa = torch.full((M,), -7.0, device="cuda")
        H.hegrid_grid_prescaled(plan, v, dt[1], C, ld, chmax, a, C, wa, H.HEGRID_MODE_TC_SPLIT,
                                main.cuda_stream)
        b = torch.full((M, C), -7.0, device="cuda")
        wb = torch.full((M,), -7.0, device="cuda")
        H.hegrid_grid(plan, v, dt[1], C, ld, b, C, wb, H.HEGRID_MODE_TC_SPLIT, main.cuda_stream)
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
        if kind != "f16":  # scaled values need the maxima
            with pytest.raises(H.HegridError) as e:
                H.hegrid_grid_prescaled(plan, v, dt[1], C, ld, None, a, C, wa,
                                        H.HEGRID_MODE_TC_SPLIT, main.cuda_stream)
            assert e.value.status == H.HEGRID_ERR_INVALID_ARG
    finally:
        H.hegrid_plan_destroy(plan)
    ref = v[:, :C].float().abs().amax(dim=0)
    assert torch.equal(chmax.cpu(), ref.cpu().view(torch.int32))
    assert torch.equal(torch.nan_to_num(a, nan=-1.0), torch.nan_to_num(b, nan=-1.0))
    assert torch.equal(wa, wb)


@pytest.mark.parametrize("kind", ["f32", "bf16", "f16", "bf16x2"])
@pytest.mark.parametrize("C", [1, 7, 300, 1030])
def test_chan_maxima_beside_equals_full(H, kind, C):
    """The one-CTA-per-SM maximum pass (HEGRID_MAXIMA_BESIDE) returns the
    full pass's maxima bit for bit, for every stored type and channel counts
    from one to more than one CTA's columns, over enough rows that several
    CTAs share each column group; for the plain types they are the largest
    |v| of each channel."""
    rng = np.random.default_rng(7 + C)
    n = 70001
    vt = torch.from_numpy((rng.standard_normal((n, C)) *
                           10.0 ** rng.integers(-6, 5, C)).astype(np.float32))
    if kind == "bf16x2":
        hi = vt.to(torch.bfloat16)
        lo = (vt - hi.float()).to(torch.bfloat16)
        packed = torch.stack([hi, lo], dim=-1).contiguous().view(torch.int32).view(n, C)
        ld = (C + 3) // 4 * 4
        v = torch.zeros((n, ld), dtype=torch.int32)
        v[:, :C] = packed
        dt, ref = H.HEGRID_BF16X2, None
    else:
        tdt, dt, mult = {"f32": (torch.float32, H.HEGRID_F32, 4),
                         "bf16": (torch.bfloat16, H.HEGRID_BF16, 8),
                         "f16": (torch.float16, H.HEGRID_F16, 8)}[kind]
        ld = (C + mult - 1) // mult * mult
        v = torch.zeros((n, ld), dtype=tdt)
        v[:, :C] = vt.to(tdt)
        ref = v[:, :C].float().abs().amax(dim=0).view(torch.int32)
    v = v.cuda()
    s = torch.cuda.current_stream().cuda_stream
    full = torch.full((C,), -1, dtype=torch.int32, device="cuda")
    lean = torch.full((C,), -1, dtype=torch.int32, device="cuda")
    H.hegrid_chan_maxima(v, dt, n, C, ld, full, 0, s)
    H.hegrid_chan_maxima(v, dt, n, C, ld, lean, H.HEGRID_MAXIMA_BESIDE, s)
    torch.cuda.synchronize()
    assert torch.equal(full.cpu(), lean.cpu())
    if ref is not None:
        assert torch.equal(full.cpu(), ref)
    with pytest.raises(H.HegridError) as e:
        H.hegrid_chan_maxima(v, dt, n, C, ld, full, 2, s)
    assert e.value.status == H.HEGRID_ERR_INVALID_ARG
