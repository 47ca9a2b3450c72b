"""ctypes binding of libhegrid.so (include/hegrid.h), same names as the C ABI.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Device buffers are passed as raw pointers (e.g. a torch tensor's
``data_ptr()``), streams as ``cudaStream_t`` handles (e.g.
``torch.cuda.current_stream().cuda_stream``).  There is no CPU fallback: if the
library is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhegrid.so")

HEGRID_OK = 0
HEGRID_ERR_INVALID_ARG = -1
HEGRID_ERR_OOM = -2
HEGRID_ERR_CUDA = -3
HEGRID_ERR_TIMEOUT = -4
HEGRID_ERR_UNSUPPORTED = -5
STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "TIMEOUT",
                -5: "UNSUPPORTED"}

HEGRID_F32, HEGRID_BF16, HEGRID_F16, HEGRID_BF16X2 = 0, 1, 2, 3
HEGRID_MODE_FP32, HEGRID_MODE_TC, HEGRID_MODE_TC_SPLIT = 0, 1, 2


def HEGRID_PLAN_BIN_CELLS(b):
    return int(b) & 0xFF


HEGRID_PLAN_SFL = 1 << 13  # plan_create flag: Sanson-Flamsteed map geometry
HEGRID_PLAN_DENSE_TILES = 1 << 14  # plan_create flag: write the dense weight tiles
HEGRID_MAXIMA_BESIDE = 1 << 0  # hegrid_chan_maxima flag: one lean CTA per SM


def HEGRID_PLAN_HEALPIX(k):
    """plan_create flag: bin by HEALPix RING-scheme pixels at nside = 2**k."""
    return (int(k) & 0x1F) << 8

EXPORTED = ["hegrid_plan_create", "hegrid_grid", "hegrid_plan_destroy", "hegrid_grid_batched",
            "hegrid_batch_create", "hegrid_batch_launch", "hegrid_batch_destroy",
            "hegrid_grid_stream", "hegrid_plan_info", "hegrid_plan_export", "hegrid_status_poll",
            "hegrid_launch_count", "hegrid_last_error", "hegrid_bin_sort_noalloc",
            "hegrid_autotune", "hegrid_autotune_bins", "hegrid_plan_set_tuning",
            "hegrid_fp32_peak", "hegrid_grid_masked", "hegrid_pool_usage",
            "hegrid_chan_maxima", "hegrid_grid_prescaled"]


class hegrid_map_geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("lon0_deg", ctypes.c_double),
                ("lat0_deg", ctypes.c_double), ("dlon_deg", ctypes.c_double),
                ("dlat_deg", ctypes.c_double)]


class hegrid_kernel(ctypes.Structure):
    _fields_ = [("fwhm_deg", ctypes.c_double), ("support_sigmas", ctypes.c_double)]


class hegrid_grid_args(ctypes.Structure):
    _fields_ = [("values", ctypes.c_void_p), ("dtype", ctypes.c_int), ("n_channels", ctypes.c_int64),
                ("ld_values", ctypes.c_int64), ("map_out", ctypes.c_void_p),
                ("ld_map", ctypes.c_int64), ("weight_out", ctypes.c_void_p),
                ("mode", ctypes.c_uint32)]


HEGRID_TUNE_MAX = 40


class hegrid_tune_point(ctypes.Structure):
    _fields_ = [("band", ctypes.c_int32), ("seg", ctypes.c_int32), ("group", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("ms", ctypes.c_float)]


class hegrid_tune_report(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("best", ctypes.c_int32),
                ("pt", hegrid_tune_point * HEGRID_TUNE_MAX)]


class HegridError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libhegrid.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P, i64, u32, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    L.hegrid_plan_create.argtypes = [PP, i64, P, P, c_int, ctypes.POINTER(hegrid_map_geom),
                                     ctypes.POINTER(hegrid_kernel), u32, P]
    L.hegrid_grid.argtypes = [P, P, c_int, i64, i64, P, i64, P, u32, P]
    L.hegrid_grid_masked.argtypes = [P, P, c_int, i64, i64, P, i64, P, u32, P]
    L.hegrid_chan_maxima.argtypes = [P, c_int, i64, i64, i64, P, u32, P]
    L.hegrid_grid_prescaled.argtypes = [P, P, c_int, i64, i64, P, P, i64, P, u32, P]
    L.hegrid_plan_destroy.argtypes = [P]
    L.hegrid_grid_batched.argtypes = [c_int, PP, ctypes.POINTER(hegrid_grid_args), P]
    L.hegrid_batch_create.argtypes = [PP, c_int, PP, ctypes.POINTER(hegrid_grid_args), P]
    L.hegrid_batch_launch.argtypes = [P, P]
    L.hegrid_batch_destroy.argtypes = [P]
    L.hegrid_grid_stream.argtypes = [P, PP, c_int, i64, c_int, u32, P, i64, P]
    L.hegrid_plan_info.argtypes = [P, P, P, P, P, P]
    L.hegrid_plan_export.argtypes = [P, P, P, P, P, P, P]
    L.hegrid_status_poll.argtypes = [P]
    L.hegrid_bin_sort_noalloc.argtypes = [i64, P, P, ctypes.POINTER(hegrid_map_geom),
                                          ctypes.POINTER(hegrid_kernel), u32, P, P, i64, P, P]
    L.hegrid_autotune.argtypes = [P, P, c_int, i64, i64, u32, P, ctypes.POINTER(hegrid_tune_report)]
    L.hegrid_autotune_bins.argtypes = [i64, P, P, c_int, ctypes.POINTER(hegrid_map_geom),
                                       ctypes.POINTER(hegrid_kernel), P,
                                       ctypes.POINTER(ctypes.c_int32), P]
    L.hegrid_plan_set_tuning.argtypes = [P, u32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32]
    L.hegrid_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), P]
    L.hegrid_pool_usage.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.hegrid_last_error.restype = ctypes.c_char_p
    L.hegrid_launch_count.restype = ctypes.c_int64
    for name in EXPORTED:
        if name not in ("hegrid_last_error", "hegrid_launch_count"):
            getattr(L, name).restype = c_int
    _lib = L
    return L


def hegrid_last_error() -> str:
    return lib().hegrid_last_error().decode()


def _check(status, where):
    if status != HEGRID_OK:
        raise HegridError(status, where, hegrid_last_error())
    return status


def _ptr(x):
    """Raw address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def geom_struct(geom) -> hegrid_map_geom:
    return hegrid_map_geom(int(geom["nx"]), int(geom["ny"]), float(geom["lon0"]),
                           float(geom["lat0"]), float(geom["dlon"]), float(geom["dlat"]))


def hegrid_plan_create(n_samples, lon_deg, lat_deg, coords_on_device, geom, fwhm_deg,
                       support_sigmas=3.0, flags=0, stream=None):
    """Returns the opaque plan handle (int)."""
    out = ctypes.c_void_p()
    g = geom_struct(geom)
    k = hegrid_kernel(float(fwhm_deg), float(support_sigmas))
    _check(lib().hegrid_plan_create(ctypes.byref(out), int(n_samples), _ptr(lon_deg),
                                    _ptr(lat_deg), int(coords_on_device), ctypes.byref(g),
                                    ctypes.byref(k), int(flags), _ptr(stream)),
           "hegrid_plan_create")
    return out.value


def hegrid_grid(plan, values, dtype, n_channels, ld_values, map_out, ld_map, weight_out, mode,
                stream=None):
    return _check(lib().hegrid_grid(plan, _ptr(values), int(dtype), int(n_channels),
                                    int(ld_values), _ptr(map_out), int(ld_map), _ptr(weight_out),
                                    int(mode), _ptr(stream)), "hegrid_grid")


def hegrid_chan_maxima(values, dtype, n_samples, n_channels, ld_values, chmax_out, flags=0,
                       stream=None):
    """Per-channel largest |v| (FP32 bits) into chmax_out (device uint32 [C])."""
    return _check(lib().hegrid_chan_maxima(_ptr(values), int(dtype), int(n_samples),
                                           int(n_channels), int(ld_values), _ptr(chmax_out),
                                           int(flags), _ptr(stream)), "hegrid_chan_maxima")


def hegrid_grid_prescaled(plan, values, dtype, n_channels, ld_values, chmax, map_out, ld_map,
                          weight_out, mode, stream=None):
    """hegrid_grid with channel maxima from hegrid_chan_maxima."""
    return _check(lib().hegrid_grid_prescaled(plan, _ptr(values), int(dtype), int(n_channels),
                                              int(ld_values), _ptr(chmax), _ptr(map_out),
                                              int(ld_map), _ptr(weight_out), int(mode),
                                              _ptr(stream)), "hegrid_grid_prescaled")


def hegrid_grid_masked(plan, values, dtype, n_channels, ld_values, map_out, ld_map, wc_out,
                       mode, stream=None):
    """Eq. 1 with per-channel masking of non-finite values (see the header)."""
    return _check(lib().hegrid_grid_masked(plan, _ptr(values), int(dtype), int(n_channels),
                                           int(ld_values), _ptr(map_out), int(ld_map),
                                           _ptr(wc_out), int(mode), _ptr(stream)),
                  "hegrid_grid_masked")


def hegrid_plan_destroy(plan):
    return _check(lib().hegrid_plan_destroy(plan), "hegrid_plan_destroy")


def _args_array(args):
    arr = (hegrid_grid_args * len(args))()
    for i, a in enumerate(args):
        arr[i] = hegrid_grid_args(_ptr(a["values"]), int(a["dtype"]), int(a["n_channels"]),
                                  int(a["ld_values"]), _ptr(a["map_out"]), int(a["ld_map"]),
                                  _ptr(a.get("weight_out")), int(a["mode"]))
    return arr


def hegrid_grid_batched(plans, args, stream=None):
    pa = (ctypes.c_void_p * len(plans))(*plans)
    return _check(lib().hegrid_grid_batched(len(plans), pa, _args_array(args), _ptr(stream)),
                  "hegrid_grid_batched")


def hegrid_batch_create(plans, args, stream=None):
    out = ctypes.c_void_p()
    pa = (ctypes.c_void_p * len(plans))(*plans)
    _check(lib().hegrid_batch_create(ctypes.byref(out), len(plans), pa, _args_array(args),
                                     _ptr(stream)), "hegrid_batch_create")
    return out.value


def hegrid_batch_launch(batch, stream=None):
    return _check(lib().hegrid_batch_launch(batch, _ptr(stream)), "hegrid_batch_launch")


def hegrid_batch_destroy(batch):
    return _check(lib().hegrid_batch_destroy(batch), "hegrid_batch_destroy")


def hegrid_grid_stream(plan, host_chunks, chunk_channels, dtype, mode, host_map, ld_host_map,
                       host_weight=None):
    arr = (ctypes.c_void_p * len(host_chunks))(*[_ptr(c) for c in host_chunks])
    return _check(lib().hegrid_grid_stream(plan, arr, len(host_chunks), int(chunk_channels),
                                           int(dtype), int(mode), _ptr(host_map),
                                           int(ld_host_map), _ptr(host_weight)),
                  "hegrid_grid_stream")


def hegrid_plan_info(plan):
    v = [ctypes.c_int64() for _ in range(5)]
    _check(lib().hegrid_plan_info(plan, *[ctypes.byref(x) for x in v]), "hegrid_plan_info")
    return dict(zip(["n_pairs", "n_bins", "n_blocks", "n_cand", "bytes"], [x.value for x in v]))


def hegrid_plan_export(plan, perm=None, bin_off=None, nb_off=None, nb_idx=None, nb_w=None,
                       weight=None):
    return _check(lib().hegrid_plan_export(plan, _ptr(perm), _ptr(bin_off), _ptr(nb_off),
                                           _ptr(nb_idx), _ptr(nb_w), _ptr(weight)),
                  "hegrid_plan_export")


def hegrid_launch_count() -> int:
    return int(lib().hegrid_launch_count())


def hegrid_pool_usage():
    """(used, reserved) bytes of the current device's library pool."""
    used, res = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().hegrid_pool_usage(ctypes.byref(used), ctypes.byref(res)), "hegrid_pool_usage")
    return int(used.value), int(res.value)


def hegrid_status_poll(plan):
    return _check(lib().hegrid_status_poll(plan), "hegrid_status_poll")


def hegrid_bin_sort_noalloc(n_samples, lon_deg, lat_deg, geom, fwhm_deg, support_sigmas,
                            perm_out, bin_off_out, bin_off_capacity, flags=0, stream=None):
    """Bin sort into caller buffers without allocating device memory (see the
    header for the limits).  Returns the number of bins."""
    nb = ctypes.c_int64(0)
    g = geom_struct(geom)
    k = hegrid_kernel(float(fwhm_deg), float(support_sigmas))
    _check(lib().hegrid_bin_sort_noalloc(int(n_samples), _ptr(lon_deg), _ptr(lat_deg),
                                         ctypes.byref(g), ctypes.byref(k), int(flags),
                                         _ptr(perm_out), _ptr(bin_off_out), int(bin_off_capacity),
                                         ctypes.byref(nb), _ptr(stream)),
           "hegrid_bin_sort_noalloc")
    return nb.value


def hegrid_autotune(plan, values, dtype, n_channels, ld_values, mode, stream=None):
    """Time the grid step's launch shapes for `mode`, keep the fastest in the
    plan; returns the report as a dict."""
    r = hegrid_tune_report()
    _check(lib().hegrid_autotune(plan, _ptr(values), int(dtype), int(n_channels), int(ld_values),
                                 int(mode), _ptr(stream), ctypes.byref(r)), "hegrid_autotune")
    pts = [{"band": r.pt[i].band, "seg": r.pt[i].seg, "group": r.pt[i].group,
            "kernel": r.pt[i].kernel, "ms": r.pt[i].ms} for i in range(r.n)]
    return {"points": pts, "best": r.best}


def hegrid_autotune_bins(n_samples, lon_deg, lat_deg, coords_on_device, geom, fwhm_deg,
                         support_sigmas=3.0, stream=None):
    """Fastest plan bin edge (1..4 cells) and the time of each."""
    best = ctypes.c_int32(0)
    ms = (ctypes.c_float * 4)()
    g = geom_struct(geom)
    k = hegrid_kernel(float(fwhm_deg), float(support_sigmas))
    _check(lib().hegrid_autotune_bins(int(n_samples), _ptr(lon_deg), _ptr(lat_deg),
                                      int(coords_on_device), ctypes.byref(g), ctypes.byref(k),
                                      _ptr(stream), ctypes.byref(best), ms),
           "hegrid_autotune_bins")
    return best.value, list(ms)


def hegrid_plan_set_tuning(plan, mode, band, seg=0, group=0, kernel=0):
    return _check(lib().hegrid_plan_set_tuning(plan, int(mode), int(band), int(seg), int(group),
                                               int(kernel)),
                  "hegrid_plan_set_tuning")


def hegrid_fp32_peak(stream=None) -> float:
    """Measured FP32 FMA throughput of the GPU in TFLOP/s."""
    t = ctypes.c_double(0.0)
    _check(lib().hegrid_fp32_peak(ctypes.byref(t), _ptr(stream)), "hegrid_fp32_peak")
    return t.value
