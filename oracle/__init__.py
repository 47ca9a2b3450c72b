"""FP64 CPU oracle for convolution-based gridding (Eq. 1, Algorithm 1).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's timed CPU baseline may import this package; the product path
(``paper_2207_04584_gb300``) never does, and this package imports nothing from
it.  The arithmetic lives in ``oracle.cpp``; this file only compiles it with
g++ and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("lon0", ctypes.c_double), ("lat0", ctypes.c_double),
                ("dlon", ctypes.c_double), ("dlat", ctypes.c_double),
                ("proj", ctypes.c_int32)]


class Kernel(ctypes.Structure):
    _fields_ = [("fwhm_deg", ctypes.c_double), ("support", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (plain g++, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off",
               "-shared", "-fPIC", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    G, K = ctypes.POINTER(Geom), ctypes.POINTER(Kernel)
    lib.og_set_mutation.argtypes = [ctypes.c_int]
    lib.og_kernel_constants.argtypes = [K, P]
    lib.og_cell_centres.argtypes = [G, P, P]
    lib.og_bf_count.argtypes = [i64, P, P, G, K, P, ctypes.c_int]
    lib.og_bf_count.restype = i64
    lib.og_bf_fill.argtypes = [i64, P, P, G, K, P, P, P, ctypes.c_int]
    lib.og_grid_csr.argtypes = [i64, P, P, P, i64, P, i64, P, P, ctypes.c_int]
    lib.og_index_create.argtypes = [i64, P, P, G, K]
    lib.og_index_create.restype = P
    lib.og_index_destroy.argtypes = [P]
    lib.og_index_count.argtypes = [P, i64, P, P, ctypes.c_int]
    lib.og_index_count.restype = i64
    lib.og_index_fill.argtypes = [P, i64, P, P, P, P, P, ctypes.c_int]
    lib.og_index_grid.argtypes = [P, i64, P, i64, P, i64, P, P, ctypes.c_int]
    lib.og_index_grid_masked.argtypes = [P, i64, P, i64, P, i64, P, P, ctypes.c_int]
    lib.og_bin_layout.argtypes = [G, K, i32, P]
    lib.og_bin_layout.restype = i64
    lib.og_bin_keys.argtypes = [i64, P, P, G, K, i32, P, P, P]
    lib.og_bin_keys.restype = i64
    lib.og_hpx_ang2pix.argtypes = [i64, i64, P, P, P, P, P]
    lib.og_hpx_centres.argtypes = [i64, P, P]
    lib.og_hpx_layout.argtypes = [G, K, i64, P, P, P]
    lib.og_hpx_layout.restype = i64
    lib.og_hpx_keys.argtypes = [i64, P, P, G, K, i64, P, P, P]
    lib.og_hpx_keys.restype = i64
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _values(values):
    """float32 [N, C] with unit channel stride (rows may be padded)."""
    values = np.asarray(values)
    if values.dtype != np.float32 or values.ndim != 2:
        raise TypeError("oracle takes float32 [N, C] values (upcast exactly inside)")
    if (values.shape[1] > 1 and values.strides[1] != 4) or values.strides[0] % 4 \
            or values.strides[0] < 4 * values.shape[1]:
        values = np.ascontiguousarray(values)
    if values.shape[1] == 1 and values.strides[0] != 4:
        values = np.ascontiguousarray(values)
    return values


def _geom(g) -> Geom:
    proj = {"": 0, "car": 0, "sfl": 1}[str(g.get("proj", "")).lower()]
    return Geom(int(g["nx"]), int(g["ny"]), float(g["lon0"]), float(g["lat0"]),
                float(g["dlon"]), float(g["dlat"]), proj)


def _kern(fwhm_deg, support) -> Kernel:
    return Kernel(float(fwhm_deg), float(support))


def set_mutation(m: int) -> None:
    """Plant mistake ``m`` (0 = none) for the pin-strength tests only."""
    _load().og_set_mutation(int(m))


def kernel_constants(fwhm_deg, support=3.0):
    """(sigma_rad, R_rad, sin^2(R/2))."""
    out = np.zeros(3)
    _load().og_kernel_constants(ctypes.byref(_kern(fwhm_deg, support)), _ptr(out))
    return float(out[0]), float(out[1]), float(out[2])


def cell_centres(geom):
    M = int(geom["nx"]) * int(geom["ny"])
    lon = np.zeros(M)
    lat = np.zeros(M)
    _load().og_cell_centres(ctypes.byref(_geom(geom)), _ptr(lon), _ptr(lat))
    return lon, lat


def neighbours_bruteforce(lon, lat, geom, fwhm_deg, support=3.0, nthreads=0):
    """Canonical CSR by testing every (cell, sample) pair: (nb_off, nb_idx, nb_w)."""
    lib = _load()
    lon, lat = _f64(lon), _f64(lat)
    g, k = _geom(geom), _kern(fwhm_deg, support)
    M = g.nx * g.ny
    off = np.zeros(M + 1, np.int64)
    P = lib.og_bf_count(len(lon), _ptr(lon), _ptr(lat), ctypes.byref(g), ctypes.byref(k),
                        _ptr(off), nthreads)
    idx = np.zeros(P, np.int32)
    w = np.zeros(P, np.float64)
    lib.og_bf_fill(len(lon), _ptr(lon), _ptr(lat), ctypes.byref(g), ctypes.byref(k), _ptr(off),
                   _ptr(idx), _ptr(w), nthreads)
    return off, idx, w


def grid_csr(nb_off, nb_idx, nb_w, values, nthreads=0):
    """Eq. 1 on a given CSR; values float32 [N, C] (ld = row stride)."""
    values = _values(values)
    M = len(nb_off) - 1
    C = values.shape[1]
    ld = values.strides[0] // 4
    out = np.zeros((M, C))
    W = np.zeros(M)
    _load().og_grid_csr(M, _ptr(np.ascontiguousarray(nb_off, np.int64)),
                        _ptr(np.ascontiguousarray(nb_idx, np.int32)),
                        _ptr(np.ascontiguousarray(nb_w, np.float64)), C,
                        values.ctypes.data_as(ctypes.c_void_p), ld, _ptr(out), _ptr(W), nthreads)
    return out, W


class Index:
    """The indexed oracle (declination strips); keeps references to lon/lat."""

    def __init__(self, lon, lat, geom, fwhm_deg, support=3.0):
        self._lib = _load()
        self.lon, self.lat = _f64(lon), _f64(lat)
        self.geom = dict(geom)
        self._g = _geom(geom)
        self._k = _kern(fwhm_deg, support)
        self.M = self._g.nx * self._g.ny
        self._h = self._lib.og_index_create(len(self.lon), _ptr(self.lon), _ptr(self.lat),
                                            ctypes.byref(self._g), ctypes.byref(self._k))

    def close(self):
        if self._h:
            self._lib.og_index_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _cells(self, cells):
        if cells is None:
            return None, self.M
        c = np.ascontiguousarray(cells, np.int64)
        return c, len(c)

    def count(self, cells=None, nthreads=0):
        """Neighbour counts only: (nb_off, P) for ``cells`` (None = all)."""
        c, nc = self._cells(cells)
        off = np.zeros(nc + 1, np.int64)
        P = self._lib.og_index_count(self._h, nc, _ptr(c), _ptr(off), nthreads)
        return off, int(P)

    def neighbours(self, cells=None, nthreads=0, with_h=False):
        """Canonical CSR (ascending n per cell) for ``cells`` (None = all)."""
        c, nc = self._cells(cells)
        off = np.zeros(nc + 1, np.int64)
        P = self._lib.og_index_count(self._h, nc, _ptr(c), _ptr(off), nthreads)
        idx = np.zeros(P, np.int32)
        w = np.zeros(P, np.float64)
        h = np.zeros(P, np.float64) if with_h else None
        self._lib.og_index_fill(self._h, nc, _ptr(c), _ptr(off), _ptr(idx), _ptr(w), _ptr(h),
                                nthreads)
        return (off, idx, w, h) if with_h else (off, idx, w)

    def grid_masked(self, values, cells=None, nthreads=0):
        """Eq. 1 with per-channel masking of non-finite values: (map [ncells, C], W_c
        [ncells, C]) FP64."""
        values = _values(values)
        c, nc = self._cells(cells)
        C = values.shape[1]
        out = np.zeros((nc, C))
        Wc = np.zeros((nc, C))
        self._lib.og_index_grid_masked(self._h, nc, _ptr(c), C,
                                       values.ctypes.data_as(ctypes.c_void_p),
                                       values.strides[0] // 4, _ptr(out), _ptr(Wc), nthreads)
        return out, Wc

    def grid(self, values, cells=None, nthreads=0):
        """Eq. 1 for ``cells``: (map [ncells, C] FP64, W [ncells] FP64)."""
        values = _values(values)
        c, nc = self._cells(cells)
        C = values.shape[1]
        out = np.zeros((nc, C))
        W = np.zeros(nc)
        self._lib.og_index_grid(self._h, nc, _ptr(c), C, values.ctypes.data_as(ctypes.c_void_p),
                                values.strides[0] // 4, _ptr(out), _ptr(W), nthreads)
        return out, W


def bin_layout(geom, fwhm_deg, support=3.0, bin_cells=2):
    lay = np.zeros(4, np.int32)
    n_bins = _load().og_bin_layout(ctypes.byref(_geom(geom)), ctypes.byref(_kern(fwhm_deg, support)),
                                   int(bin_cells), _ptr(lay))
    return int(n_bins), tuple(int(x) for x in lay)


def bin_keys(lon, lat, geom, fwhm_deg, support=3.0, bin_cells=2):
    """(key uint32[N], perm int32[N], bin_off int32[n_bins+1]) of the padded-map bins."""
    lon, lat = _f64(lon), _f64(lat)
    n_bins, _ = bin_layout(geom, fwhm_deg, support, bin_cells)
    if n_bins < 0:
        raise ValueError("geometry reaches a pole or wraps onto itself")
    key = np.zeros(len(lon), np.uint32)
    perm = np.zeros(len(lon), np.int32)
    off = np.zeros(n_bins + 1, np.int32)
    _load().og_bin_keys(len(lon), _ptr(lon), _ptr(lat), ctypes.byref(_geom(geom)),
                        ctypes.byref(_kern(fwhm_deg, support)), int(bin_cells), _ptr(key),
                        _ptr(perm), _ptr(off))
    return key, perm, off


# ---------------------------------------------------------------------------
# HEALPix ring scheme (the paper's pixelisation, Sec. 4.1.1)
# ---------------------------------------------------------------------------
def hpx_ang2pix(nside, z, phi_deg):
    """(ring 1..4N-1, pixel in ring, RING-scheme pixel index) of points given by
    z = sin(lat) and phi in degrees."""
    z, phi = _f64(z), _f64(phi_deg)
    n = len(z)
    ring = np.zeros(n, np.int64)
    pix = np.zeros(n, np.int64)
    ipix = np.zeros(n, np.int64)
    _load().og_hpx_ang2pix(int(nside), n, _ptr(z), _ptr(phi), _ptr(ring), _ptr(pix), _ptr(ipix))
    return ring, pix, ipix


def hpx_centres(nside):
    """(z, phi in degrees) of the 12 nside^2 pixel centres in RING order."""
    n = 12 * int(nside) ** 2
    z = np.zeros(n)
    phi = np.zeros(n)
    _load().og_hpx_centres(int(nside), _ptr(z), _ptr(phi))
    return z, phi


def hpx_layout(geom, fwhm_deg, support=3.0, nside=4096):
    """(n_bins, ring0, table int64[n_rings, 4] = n_i, J0, cnt, half) of the HEALPix
    variant's bins over the padded map."""
    r0 = ctypes.c_int64(0)
    nr = ctypes.c_int64(0)
    G, K = ctypes.byref(_geom(geom)), ctypes.byref(_kern(fwhm_deg, support))
    n_bins = _load().og_hpx_layout(G, K, int(nside), ctypes.byref(r0), ctypes.byref(nr), None)
    if n_bins < 0:
        raise ValueError("geometry reaches a pole or wraps onto itself")
    tab = np.zeros((nr.value, 4), np.int64)
    _load().og_hpx_layout(G, K, int(nside), ctypes.byref(r0), ctypes.byref(nr), _ptr(tab))
    return int(n_bins), int(r0.value), tab


def hpx_keys(lon, lat, geom, fwhm_deg, support=3.0, nside=4096):
    """(key uint32[N], perm int32[N], bin_off int32[n_bins+1]) of the HEALPix variant."""
    lon, lat = _f64(lon), _f64(lat)
    n_bins, _, _ = hpx_layout(geom, fwhm_deg, support, nside)
    key = np.zeros(len(lon), np.uint32)
    perm = np.zeros(len(lon), np.int32)
    off = np.zeros(n_bins + 1, np.int32)
    _load().og_hpx_keys(len(lon), _ptr(lon), _ptr(lat), ctypes.byref(_geom(geom)),
                        ctypes.byref(_kern(fwhm_deg, support)), int(nside), _ptr(key),
                        _ptr(perm), _ptr(off))
    return key, perm, off
