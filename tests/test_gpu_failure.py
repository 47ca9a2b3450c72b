"""Failure detection without a GPU fault.

* A device-side wait that runs out: HEGRID_FAULT=wait:1 runs the next
  tensor-core grid kernel with one producer arrive withheld and a 20 ms wait
  limit.  Every role of the persistent kernel then gives up at its next
  bounded wait, the kernel frees its tensor memory and returns, and
  hegrid_status_poll reports TIMEOUT; the context stays usable (a fresh plan
  grids correctly afterwards).
* Host-side injection: HEGRID_FAULT=alloc:N / launch:N turn the N-th pool
  allocation or kernel launch of a call into an OOM / CUDA status; every
  failed call leaves the library's pool as it found it (no leak).
"""
import numpy as np
import pytest

import oracle
from helpers import map_error
from paper_2207_04584_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_04584_gb300 import build
    build.build()
    from paper_2207_04584_gb300 import hegrid
    hegrid.lib()
    return hegrid


@pytest.fixture
def fault(monkeypatch):
    def set_fault(text):
        if text is None:
            monkeypatch.delenv("HEGRID_FAULT", raising=False)
        else:
            monkeypatch.setenv("HEGRID_FAULT", text)
    yield set_fault
    monkeypatch.delenv("HEGRID_FAULT", raising=False)


def _wl():
    return W.config1(n=6000, C=16, nx=48, ny=40)


def _plan(H, wl, flags=0):
    return H.hegrid_plan_create(len(wl["lon"]), np.ascontiguousarray(wl["lon"]),
                                np.ascontiguousarray(wl["lat"]), 0, wl["geom"], wl["fwhm_deg"],
                                3.0, flags, torch.cuda.current_stream().cuda_stream)


def _used(H):
    torch.cuda.synchronize()
    return H.hegrid_pool_usage()[0]


def test_wait_timeout_sets_status_and_context_survives(H, fault):
    wl = _wl()
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    s = torch.cuda.current_stream().cuda_stream
    v = torch.from_numpy(wl["values"]).cuda()
    out = torch.zeros((M, 16), device="cuda")
    plan = _plan(H, wl)
    try:
        H.hegrid_status_poll(plan)  # a fresh plan reports OK
        fault("wait:1")
        H.hegrid_grid(plan, v, H.HEGRID_F32, 16, 16, out, 16, None, H.HEGRID_MODE_TC_SPLIT, s)
        torch.cuda.synchronize()  # the kernel returns: its waits are bounded
        fault(None)
        with pytest.raises(H.HegridError) as e:
            H.hegrid_status_poll(plan)
        assert e.value.status == H.HEGRID_ERR_TIMEOUT
        assert "timed out" in H.hegrid_last_error()
    finally:
        H.hegrid_plan_destroy(plan)
    # the context is still usable: a new plan grids within tolerance
    plan = _plan(H, wl)
    try:
        H.hegrid_grid(plan, v, H.HEGRID_F32, 16, 16, out, 16, None, H.HEGRID_MODE_TC_SPLIT, s)
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(wl["values"])
    err, _, _ = map_error(out.cpu().numpy(), ref, Wref)
    assert err <= 5e-5, err


@pytest.mark.parametrize("tiles", [False, True])
def test_alloc_faults_in_plan_create_leak_nothing(H, fault, tiles):
    """Every alloc of plan creation made to fail in turn (with the plan's
    dense weight tiles: the second stream's pair kernel and tile builds too)
    returns the error and leaves the pool as it was."""
    wl = _wl()
    flags = H.HEGRID_PLAN_DENSE_TILES if tiles else 0
    base = _used(H)
    failed = 0
    for k in range(1, 64):
        fault(f"alloc:{k}")
        try:
            plan = _plan(H, wl, flags)
        except H.HegridError as e:
            assert e.status == H.HEGRID_ERR_OOM, (k, e.status)
            assert _used(H) == base, k
            failed += 1
            continue
        fault(None)
        H.hegrid_plan_destroy(plan)
        assert _used(H) == base
        break
    else:
        pytest.fail("plan creation never completed")
    assert failed >= 5  # every allocation of plan creation was made to fail once


@pytest.mark.parametrize("tiles", [False, True])
def test_launch_faults_in_plan_create_leak_nothing(H, fault, tiles):
    """Every launch of plan creation made to fail in turn (with the plan's
    dense weight tiles: the second stream's pair kernel and tile builds too)
    returns the error and leaves the pool as it was."""
    wl = _wl()
    flags = H.HEGRID_PLAN_DENSE_TILES if tiles else 0
    base = _used(H)
    failed = 0
    for k in range(1, 96):
        fault(f"launch:{k}")
        try:
            plan = _plan(H, wl, flags)
        except H.HegridError as e:
            assert e.status == H.HEGRID_ERR_CUDA, (k, e.status)
            assert _used(H) == base, k
            failed += 1
            continue
        fault(None)
        H.hegrid_plan_destroy(plan)
        assert _used(H) == base
        break
    else:
        pytest.fail("plan creation never completed")
    assert failed >= 5


@pytest.mark.parametrize("what,status", [("alloc:1", "HEGRID_ERR_OOM"),
                                         ("launch:1", "HEGRID_ERR_CUDA"),
                                         ("launch:2", "HEGRID_ERR_CUDA")])
def test_grid_faults_leak_nothing(H, fault, what, status):
    """The tensor-core grid call: its scratch (the channel maxima) is the first
    allocation, the maxima pass and the grid kernel its launches."""
    wl = _wl()
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    s = torch.cuda.current_stream().cuda_stream
    v = torch.from_numpy(wl["values"]).cuda()
    out = torch.zeros((M, 16), device="cuda")
    plan = _plan(H, wl)
    try:
        base = _used(H)
        fault(what)
        with pytest.raises(H.HegridError) as e:
            H.hegrid_grid(plan, v, H.HEGRID_F32, 16, 16, out, 16, None,
                          H.HEGRID_MODE_TC_SPLIT, s)
        fault(None)
        assert e.value.status == getattr(H, status)
        assert _used(H) == base
        # the next call succeeds
        H.hegrid_grid(plan, v, H.HEGRID_F32, 16, 16, out, 16, None, H.HEGRID_MODE_TC_SPLIT, s)
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)


@pytest.mark.parametrize("kernel", [2, 3])
def test_dense_tile_kernels_wait_timeout(H, fault, kernel):
    """The bounded waits of the kernels that read the dense weight tiles
    (channel-major; cell-major with dense A tiles): one producer warp withholds
    its first arrive, every role gives up, TIMEOUT is reported and the plan
    grids correctly afterwards."""
    wl = W.config1(n=6000, C=200, nx=48, ny=40)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    s = torch.cuda.current_stream().cuda_stream
    v = torch.from_numpy(wl["values"]).cuda()
    out = torch.zeros((M, 200), device="cuda")
    plan = _plan(H, wl)
    try:
        H.hegrid_plan_set_tuning(plan, H.HEGRID_MODE_TC_SPLIT, 0, 0, 0, kernel)
        fault("wait:1")
        H.hegrid_grid(plan, v, H.HEGRID_F32, 200, 200, out, 200, None, H.HEGRID_MODE_TC_SPLIT, s)
        torch.cuda.synchronize()
        fault(None)
        with pytest.raises(H.HegridError) as e:
            H.hegrid_status_poll(plan)
        assert e.value.status == H.HEGRID_ERR_TIMEOUT
    finally:
        H.hegrid_plan_destroy(plan)
    plan = _plan(H, wl)
    try:
        H.hegrid_plan_set_tuning(plan, H.HEGRID_MODE_TC_SPLIT, 0, 0, 0, kernel)
        H.hegrid_grid(plan, v, H.HEGRID_F32, 200, 200, out, 200, None, H.HEGRID_MODE_TC_SPLIT, s)
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(wl["values"])
    err, _, _ = map_error(out.cpu().numpy(), ref, Wref)
    assert err <= 5e-5, err


@pytest.mark.parametrize("kernel", [2, 3])
@pytest.mark.parametrize("what,status", [("alloc:1", "HEGRID_ERR_OOM"),
                                         ("alloc:2", "HEGRID_ERR_OOM"),
                                         ("launch:1", "HEGRID_ERR_CUDA"),
                                         ("launch:2", "HEGRID_ERR_CUDA"),
                                         ("launch:3", "HEGRID_ERR_CUDA")])
def test_dense_tile_first_call_faults_leak_nothing(H, fault, what, status, kernel):
    """The first grid call on a plan with a kernel that reads the dense weight
    tiles (channel-major, or cell-major with dense A tiles) allocates the channel maxima
    (allocation 1) and the plan's dense weight tiles (2), then launches the
    tile build (launch 1), the maxima pass (2) and the grid kernel (3).  A
    failure anywhere returns its status; the tiles stay with the plan only if
    they were built (then the plan owns and later frees them), and the next
    call succeeds."""
    wl = W.config1(n=6000, C=200, nx=48, ny=40)
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    s = torch.cuda.current_stream().cuda_stream
    v = torch.from_numpy(wl["values"]).cuda()
    out = torch.zeros((M, 200), device="cuda")
    base0 = _used(H)
    plan = _plan(H, wl)
    try:
        H.hegrid_plan_set_tuning(plan, H.HEGRID_MODE_TC_SPLIT, 0, 0, 0, kernel)
        base = _used(H)
        b0 = H.hegrid_plan_info(plan)["bytes"]
        fault(what)
        with pytest.raises(H.HegridError) as e:
            H.hegrid_grid(plan, v, H.HEGRID_F32, 200, 200, out, 200, None,
                          H.HEGRID_MODE_TC_SPLIT, s)
        fault(None)
        assert e.value.status == getattr(H, status)
        built = H.hegrid_plan_info(plan)["bytes"] - b0  # the tiles, if they were built
        if what in ("alloc:1", "alloc:2", "launch:1"):
            assert built == 0 and _used(H) == base
        else:
            assert built > 0 and _used(H) > base
        H.hegrid_grid(plan, v, H.HEGRID_F32, 200, 200, out, 200, None, H.HEGRID_MODE_TC_SPLIT, s)
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    assert _used(H) == base0
    ref, Wref = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"]).grid(wl["values"])
    err, _, _ = map_error(out.cpu().numpy(), ref, Wref)
    assert err <= 5e-5, err
