"""The allocation-free bin sort against the plan's own sort.

Some callers cannot allocate device memory (a host framework that owns all
allocations, a real-time loop that must not wait on the allocator); for them
hegrid_bin_sort_noalloc keeps its scratch in a fixed array inside the
library.  Its permutation and bin offsets must equal, bit for bit, what
hegrid_plan_create computes for the same samples (exported by
hegrid_plan_export), on two calls in a row (the second call reuses the scratch
the first one left behind).
"""
import numpy as np
import pytest

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


def _reference(H, wl, flags):
    s = torch.cuda.current_stream().cuda_stream
    plan = H.hegrid_plan_create(len(wl["lon"]), np.ascontiguousarray(wl["lon"]),
                                np.ascontiguousarray(wl["lat"]), 0, wl["geom"], wl["fwhm_deg"],
                                3.0, flags, s)
    try:
        info = H.hegrid_plan_info(plan)
        perm = np.zeros(len(wl["lon"]), np.int32)
        off = np.zeros(info["n_bins"] + 1, np.int32)
        H.hegrid_plan_export(plan, perm, off)
    finally:
        H.hegrid_plan_destroy(plan)
    return perm, off


@pytest.mark.parametrize("flags", [0, 4])
def test_noalloc_matches_plan_twice(H, flags):
    cases = [W.config1(with_values=False),
             W.config1(seed=W.SEED_BASE + 11, n=7777, nx=50, ny=37, with_values=False)]
    for wl in cases:
        ref_perm, ref_off = _reference(H, wl, flags)
        lon = torch.from_numpy(np.ascontiguousarray(wl["lon"])).cuda()
        lat = torch.from_numpy(np.ascontiguousarray(wl["lat"])).cuda()
        n = len(wl["lon"])
        s = torch.cuda.current_stream().cuda_stream
        for _ in range(2):
            perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            off = torch.full((len(ref_off) + 5,), -1, dtype=torch.int32, device="cuda")
            nb = H.hegrid_bin_sort_noalloc(n, lon, lat, wl["geom"], wl["fwhm_deg"], 3.0, perm, off,
                                           off.numel(), flags, s)
            torch.cuda.synchronize()
            assert nb == len(ref_off) - 1
            assert np.array_equal(perm.cpu().numpy(), ref_perm)
            assert np.array_equal(off.cpu().numpy()[:nb + 1], ref_off)


def test_noalloc_limit_and_single_sample(H):
    """The largest accepted input (524,288 samples: the histogram, offset and
    partial-sum regions of the array are full) and the smallest (one sample),
    each bit for bit against the plan's own sort."""
    big = W.config1(seed=W.SEED_BASE + 12, n=524288, nx=160, ny=150, with_values=False)
    one = W.config1(seed=W.SEED_BASE + 13, n=1, with_values=False)
    s = torch.cuda.current_stream().cuda_stream
    for wl in (big, one):
        ref_perm, ref_off = _reference(H, wl, 0)
        n = len(wl["lon"])
        lon = torch.from_numpy(np.ascontiguousarray(wl["lon"])).cuda()
        lat = torch.from_numpy(np.ascontiguousarray(wl["lat"])).cuda()
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        off = torch.full((len(ref_off),), -1, dtype=torch.int32, device="cuda")
        nb = H.hegrid_bin_sort_noalloc(n, lon, lat, wl["geom"], wl["fwhm_deg"], 3.0, perm, off,
                                       off.numel(), 0, s)
        torch.cuda.synchronize()
        assert nb == len(ref_off) - 1
        assert np.array_equal(perm.cpu().numpy(), ref_perm)
        assert np.array_equal(off.cpu().numpy(), ref_off)


def test_noalloc_rejects_oversize_and_small_buffers(H):
    wl = W.config1(with_values=False)
    lon = torch.from_numpy(np.ascontiguousarray(wl["lon"])).cuda()
    lat = torch.from_numpy(np.ascontiguousarray(wl["lat"])).cuda()
    perm = torch.empty(len(wl["lon"]), dtype=torch.int32, device="cuda")
    off = torch.empty(8, dtype=torch.int32, device="cuda")
    with pytest.raises(H.HegridError) as e:
        H.hegrid_bin_sort_noalloc(524289, lon, lat, wl["geom"], wl["fwhm_deg"], 3.0, perm, off, 8)
    assert e.value.status == H.HEGRID_ERR_INVALID_ARG
    with pytest.raises(H.HegridError) as e:
        H.hegrid_bin_sort_noalloc(len(wl["lon"]), lon, lat, wl["geom"], wl["fwhm_deg"], 3.0, perm,
                                  off, 8)
    assert e.value.status == H.HEGRID_ERR_INVALID_ARG
    # HEALPix and Sanson-Flamsteed plans have other keys: refused with a message naming both
    big_off = torch.empty(1 << 20, dtype=torch.int32, device="cuda")
    for flags in (H.HEGRID_PLAN_HEALPIX(10), H.HEGRID_PLAN_SFL):
        with pytest.raises(H.HegridError) as e:
            H.hegrid_bin_sort_noalloc(len(wl["lon"]), lon, lat, wl["geom"], wl["fwhm_deg"], 3.0,
                                      perm, big_off, big_off.numel(), flags)
        assert e.value.status == H.HEGRID_ERR_INVALID_ARG
        assert "HEGRID_PLAN_SFL" in H.hegrid_last_error()
