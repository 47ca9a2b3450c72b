"""Host-side logic that needs no GPU: plan-flag encodings match the header,
flag and argument checks that run before any CUDA call, seeded workload
generators, the bench's traffic table guard, and that the product path has
no fallback and never touches the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2207_04584_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_2207_04584_gb300 import build
    build.build()
    from paper_2207_04584_gb300 import hegrid
    hegrid.lib()
    return hegrid


def test_flag_encodings_match_header(H):
    txt = open(os.path.join(ROOT, "include", "hegrid.h")).read()
    assert "#define HEGRID_PLAN_SFL (1u << 13)" in txt
    assert "#define HEGRID_PLAN_DENSE_TILES (1u << 14)" in txt
    assert H.HEGRID_PLAN_DENSE_TILES == 1 << 14
    assert re.search(r"#define HEGRID_PLAN_HEALPIX\(k\) \(\(\(uint32_t\)\(k\) & 0x1fu\) << 8\)", txt)
    assert H.HEGRID_PLAN_SFL == 1 << 13
    assert H.HEGRID_PLAN_HEALPIX(12) == 12 << 8 and H.HEGRID_PLAN_HEALPIX(33) == 1 << 8
    assert H.HEGRID_PLAN_BIN_CELLS(3) == 3


@pytest.mark.parametrize("flags", [1 << 15, 1 << 31, (14 << 8), (1 << 13) | (12 << 8)])
def test_bad_plan_flags_rejected_before_cuda(H, flags):
    lib = H.lib()
    out = ctypes.c_void_p()
    lon = np.array([10.0, 10.01])
    lat = np.array([20.0, 20.01])
    g = H.hegrid_map_geom(10, 10, 10.0, 20.0, 0.01, 0.01)
    k = H.hegrid_kernel(0.05, 3.0)
    st = lib.hegrid_plan_create(ctypes.byref(out), 2, lon.ctypes.data, lat.ctypes.data, 0,
                                ctypes.byref(g), ctypes.byref(k), flags, None)
    assert st == H.HEGRID_ERR_INVALID_ARG and out.value is None


def test_chan_maxima_flags_checked_before_cuda(H):
    lib = H.lib()
    dummy = ctypes.c_void_p(256)
    assert H.HEGRID_MAXIMA_BESIDE == 1
    txt = open(os.path.join(ROOT, "include", "hegrid.h")).read()
    assert "#define HEGRID_MAXIMA_BESIDE (1u << 0)" in txt
    for flags in (2, 1 << 31):
        st = lib.hegrid_chan_maxima(dummy, H.HEGRID_F32, 1, 4, 4, dummy, flags, None)
        assert st == H.HEGRID_ERR_INVALID_ARG
        assert "flag" in H.hegrid_last_error()


def test_masked_and_stream_argument_checks(H):
    lib = H.lib()
    assert lib.hegrid_grid_masked(None, None, 0, 1, 1, None, 1, None, 0, None) == \
        H.HEGRID_ERR_INVALID_ARG
    assert "plan" in H.hegrid_last_error()


def test_generators_are_seeded():
    a = W.sim_survey(n=3000, C=4)
    b = W.sim_survey(n=3000, C=4)
    assert np.array_equal(a["lon"], b["lon"]) and np.array_equal(a["values"], b["values"])
    g = a["geom"]
    assert (g["nx"], g["ny"], g["lon0"], g["lat0"]) == (3600, 1200, 30.0, 41.0)
    assert np.all((a["lon"] >= 0) & (a["lon"] < 60) & (a["lat"] >= 31) & (a["lat"] < 51))
    c = W.sim_survey(n=3000, C=4, lon_span=10.0)
    assert c["geom"]["nx"] == 600 and c["geom"]["lon0"] == 5.0 and c["lon"].max() < 10.0
    d1 = W.config1(with_values=False)
    d2 = W.config1(with_values=False)
    assert np.array_equal(d1["lat"], d2["lat"])


def test_traffic_guard(monkeypatch):
    import bench
    t = bench.TRAFFIC["k_grid_tc"]
    assert bench.measured_traffic("k_grid_tc") in (None, t["bytes"])
    monkeypatch.setitem(bench.TRAFFIC, "k_grid_tc", dict(t, sha256="0" * 64))
    assert bench.measured_traffic("k_grid_tc") is None
    monkeypatch.setitem(bench.TRAFFIC, "k_grid_tc",
                        dict(t, sha256=bench.sources_sha256(t["sources"])))
    assert bench.measured_traffic("k_grid_tc") == t["bytes"]
    assert bench.job_value(100, 2, 0.5) == 400


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the built CUDA library every call path raises."""
    from paper_2207_04584_gb300 import hegrid
    monkeypatch.setattr(hegrid, "LIB_PATH", str(tmp_path / "libhegrid.so"))
    monkeypatch.setattr(hegrid, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        hegrid.lib()
    with pytest.raises(RuntimeError, match="missing"):
        hegrid.hegrid_launch_count()


def test_product_code_never_uses_the_oracle():
    """The package (Python binding, workloads, CUDA sources) neither imports,
    includes nor loads anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_2207_04584_gb300")
    checked = 0
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if not f.endswith((".py", ".cu", ".cuh", ".h", ".cpp", ".c")):
                continue
            src = open(os.path.join(dirpath, f)).read()
            checked += 1
            assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
            assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", src), f
            code = re.sub(r"//[^\n]*|#[^\n]*", "", src)
            assert "liboracle" not in src and not re.search(r"\bog_\w+\s*\(", code), f
    assert checked >= 6
