"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2207_04584_gb300 import build
    build.build()
    from paper_2207_04584_gb300 import hegrid as H
    return H.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "hegrid.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hegrid_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_boundary():
    syms = declared_symbols()
    for s in ["hegrid_plan_create", "hegrid_grid", "hegrid_plan_destroy"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2207_04584_gb300 import hegrid as H
    nm = subprocess.run(["nm", "-D", "--defined-only", H.LIB_PATH], capture_output=True,
                        text=True, check=True).stdout
    exported = set(re.findall(r"\bT (hegrid_\w+)", nm))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(lib, s)
    assert set(H.EXPORTED) == set(declared_symbols())


def test_argument_errors_without_gpu(lib):
    """Argument checks run before any CUDA call (no GPU needed)."""
    import ctypes
    from paper_2207_04584_gb300 import hegrid as H
    out = ctypes.c_void_p()
    g = H.hegrid_map_geom(0, 10, 0.0, 0.0, 0.01, 0.01)
    k = H.hegrid_kernel(0.05, 3.0)
    st = lib.hegrid_plan_create(ctypes.byref(out), 10, 1, 1, 0, ctypes.byref(g), ctypes.byref(k),
                                0, None)
    assert st == H.HEGRID_ERR_INVALID_ARG and out.value is None
    assert "nx" in H.hegrid_last_error()
    assert lib.hegrid_grid(None, None, 0, 1, 1, None, 1, None, 0, None) == H.HEGRID_ERR_INVALID_ARG


def test_every_status_entry_point_documents_its_errors():
    """Each declaration returning hegrid_status is preceded (after the previous
    declaration) by a comment that states its error behaviour."""
    txt = open(os.path.join(ROOT, "include", "hegrid.h")).read()
    decl = re.compile(r"^hegrid_status\s+(hegrid_\w+)\s*\(", re.M)
    prev_end = 0
    pending = []
    missing = []
    for m in decl.finditer(txt):
        seg = txt[prev_end:m.start()]
        comments = " ".join(re.findall(r"/\*.*?\*/", seg, flags=re.S))
        if comments.strip():
            pending = [comments]
        doc = " ".join(pending)
        if not re.search(r"Errors?\b|INVALID_ARG|Returns OK|no-op", doc):
            missing.append(m.group(1))
        prev_end = txt.index(";", m.end()) + 1
    assert not missing, missing
