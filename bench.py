"""Throughput of the gridding hot path on the FAST-like drift-scan workload.

One step = one pass of the whole path over one batch of synthetic input:
plan creation (coordinate prep, bin keys, radix sort, bin offsets, neighbour
lists, weights) followed by the grid step (accumulate + normalise) of every
channel, then plan destruction.  Metric: sample x channel contributions per
second, N * C / t_step, whole job over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mode tc_split|tc|fp32]
    python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Under torchrun each rank runs an independent replica (the path shards by
fields or channel slices with no exchange; one GPU per rank): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2207_04584_gb300 import workloads as W  # noqa: E402

METRIC = "sample x channel contributions/s (N*C/t, plan + grid per step)"
# Arithmetic of each grid form: FP32 values in, products on CUDA cores (fp32) or on
# the tensor cores from FP16 parts of per-channel power-of-two-scaled values and
# weights (tc_split: hi*hi + hi*lo + lo*hi; tc: hi*hi), FP32 accumulation.
FORM_DTYPE = {"fp32": "f32",
              "tc_split": "f32 in; f16 hi/lo split (3 MMAs), f32 accumulate",
              "tc": "f32 in; f16 (1 MMA), f32 accumulate"}
UNIT = "contrib/s"
L2_BYTES = 129 * 1024 * 1024


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms",
                 "100", "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, dist, device=None):
    """The largest of x over all ranks (x itself when not distributed)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# DRAM traffic per grid launch on the bench workload, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum; see the capture summary named
# below).  Used only while the kernel's sources hash to the value the capture
# was taken on: a changed kernel reports null.
TRAFFIC = {
    "k_grid_tc": {"sources": ["paper_2207_04584_gb300/csrc/grid_tc.cu",
                              "paper_2207_04584_gb300/csrc/ptx.cuh",
                              "paper_2207_04584_gb300/csrc/hegrid_internal.cuh"],
                  "sha256": "df3138a45841893a091a6afd07b5f9b691fdd520529884f23bc6f6d69ad8c7b3",
                  "bytes": 32.899492224e9 + 1.472701696e9,
                  "capture": "profiles/k_grid_tc_fast_drift_c256.md (the bench's tuned launch, "
                             "C=1024; mean of 4)"},
    "k_grid_tc_dense": {"sources": ["paper_2207_04584_gb300/csrc/grid_tc.cu",
                                    "paper_2207_04584_gb300/csrc/ptx.cuh",
                                    "paper_2207_04584_gb300/csrc/hegrid_internal.cuh"],
                        "sha256": "7a699345de124cb048e4234ceb5094ed1f0841ccd73a9ba59972200f40b8c878",
                        "bytes": 38.2067e9 + 1.473e9,
                        "capture": "profiles/k_grid_tc_fast_drift_c256.md (the bench's tuned "
                                   "launch with dense A tiles, C=1024; mean of 9)"},
    "k_grid_f32": {"sources": ["paper_2207_04584_gb300/csrc/grid_f32.cu",
                               "paper_2207_04584_gb300/csrc/ptx.cuh",
                               "paper_2207_04584_gb300/csrc/hegrid_internal.cuh"],
                   "sha256": "51985c6f0c8a21fafd8c1b2f45a66b77df626f7deee350802c86d269a179f04f",
                   "bytes": 30.3695e9 + 1.470e9,
                   "capture": "profiles/k_grid_f32_fast_drift_c256.md (the bench's FP32-form "
                              "launch, C=1024; mean of 4)"},
}


def sources_sha256(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel):
    t = TRAFFIC.get(kernel)
    if not t or not t["sha256"] or sources_sha256(t["sources"]) != t["sha256"]:
        return None
    return t["bytes"]


def job_value(units_per_rank, world, elapsed_max):
    """Whole-job throughput of independent replicas: all ranks' units over
    the slowest rank's time."""
    return world * units_per_rank / elapsed_max


def cpu_oracle_sample(wl, frac_rows=20, nthreads=0, keep=None):
    """Time the FP64 oracle on a bounded sample: every frac_rows-th map row,
    all channels; extrapolate to the full map as t_index + t_cells * M / cells.
    With ``keep`` (a dict), the oracle's index is left in keep["index"]."""
    import oracle
    g = wl["geom"]
    nx, ny = g["nx"], g["ny"]
    rows = np.arange(0, ny, frac_rows)
    cells = (rows[:, None] * nx + np.arange(nx)[None, :]).ravel()
    t0 = time.perf_counter()
    ix = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"], wl.get("support", 3.0))
    if keep is not None:
        keep["index"] = ix
    t1 = time.perf_counter()
    ix.grid(wl["values"], cells=cells, nthreads=nthreads)
    t2 = time.perf_counter()
    M = nx * ny
    t_full = (t1 - t0) + (t2 - t1) * M / len(cells)
    N, C = wl["values"].shape
    cores = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    return {"value": N * C / t_full, "unit": UNIT, "cores": cores, "kind": "oracle",
            "extrapolated": True,
            "sample": f"FP64 oracle (declination-strip index, OpenMP) on every {frac_rows}th "
                      f"map row ({len(cells)} of {M} cells, all {C} channels); index build "
                      f"{t1 - t0:.2f}s + cells {t2 - t1:.2f}s, extrapolated to the full map "
                      f"({t_full:.1f}s)"}


def cpu_oracle_full(wl, channels=None, nthreads=0):
    """Time one complete run of the FP64 oracle: index build plus Eq. 1 on every
    cell of the map for the given channels (default all).  Returns (record,
    map [M, C] FP64, W [M] FP64)."""
    import oracle
    g = wl["geom"]
    vals = wl["values"] if channels is None else wl["values"][:, channels]
    t0 = time.perf_counter()
    ix = oracle.Index(wl["lon"], wl["lat"], g, wl["fwhm_deg"], wl.get("support", 3.0))
    t1 = time.perf_counter()
    ref, Wref = ix.grid(vals, nthreads=nthreads)
    t2 = time.perf_counter()
    ix.close()
    N, C = vals.shape
    M = g["nx"] * g["ny"]
    cores = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    rec = {"value": N * C / (t2 - t0), "unit": UNIT, "cores": cores, "kind": "oracle",
           "extrapolated": False, "seconds": t2 - t0,
           "sample": f"FP64 oracle (declination-strip index, OpenMP), one complete run: "
                     f"every cell of the {M}-cell map, {C} channels; index build "
                     f"{t1 - t0:.2f}s + cells {t2 - t1:.2f}s"}
    return rec, ref, Wref


def map_errors(got, gw, ref, Wref):
    """Per-channel error of a map against the oracle's (max |got - ref| / RMS(ref)
    over the cells with W >= 1e-3 max W), its max and median over channels, and
    the weight map's max |dW| / max W."""
    mask = Wref >= 1e-3 * Wref.max()
    r = ref[mask]
    rms = np.sqrt(np.mean(r * r, axis=0))
    e = np.zeros(ref.shape[1])
    for c0 in range(0, ref.shape[1], 64):  # channel slices keep the temporaries small
        d = np.abs(got[mask, c0:c0 + 64].astype(np.float64) - r[:, c0:c0 + 64])
        e[c0:c0 + 64] = d.max(axis=0) / rms[c0:c0 + 64]
    nan_ok = bool(np.array_equal(np.isnan(got), np.isnan(ref)))
    return {"max": float(e.max()), "median": float(np.median(e)), "cells": int(mask.sum()),
            "channels": int(ref.shape[1]), "nan_pattern_matches": nan_ok,
            "weight_map": float(np.max(np.abs(gw.astype(np.float64) - Wref)) / Wref.max())}


def workload_desc(N, C):
    return (f"FAST-like 19-beam drift scan, 5x5 deg at (30,41), N={N}, C={C} FP32, 600x600 map "
            "at 0.5', FWHM 2.9', R=3 sigma")


def workload_config(N, C, M, world):
    """The `config` of both arms' bench lines: the workload alone (the form,
    tuning and binning of the GPU arm are reported beside it)."""
    return {"workload": workload_desc(N, C), "N": N, "C": C, "M": M,
            "l2": "inputs larger than L2 (values 8 GB)", "parallelism": f"replicas x{world}"}


REF_SLICE = 256  # channels per reference-arm step


def run_reference(args, rank):
    """The reference arm: the FP64 oracle (the plain definition of Eq. 1, as it
    stands) on the host cores.  Each step is one complete oracle run over the whole
    map for a 256-channel slice of the workload (the slices cycle through all
    1024 channels), timed as run; value = the sample x channel contributions of
    those steps over their time."""
    if rank != 0:
        return
    t_gen = time.perf_counter()
    wl = W.config2()
    t_gen = time.perf_counter() - t_gen
    N, C = wl["values"].shape
    nsl = C // REF_SLICE
    times, rec = [], None
    for i in range(args.warmup + args.steps):
        k = i % nsl
        rec, _, _ = cpu_oracle_full(wl, channels=slice(k * REF_SLICE, (k + 1) * REF_SLICE))
        if i >= args.warmup:
            times.append(rec["seconds"])
    t = statistics.mean(times)
    value = N * REF_SLICE / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(N, C, wl["geom"]["nx"] * wl["geom"]["ny"], 1),
            "seed": W.SEED_BASE + 2,
            "reference_step": f"the whole map for {REF_SLICE} of the {C} channels "
                              "(slices cycled)",
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle",
                             "cores": rec["cores"],
                             "sample": f"each step: {rec['sample']} (channel slice of "
                                       f"{REF_SLICE}; not extrapolated)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gen_s": t_gen}
    print(json.dumps(line), flush=True)


def _link(torch, dev, stream):
    """Pinned host <-> device copy rates (GB/s) of one 1 GiB copy each way, device-timed."""
    out = {}
    lh = torch.empty(1 << 28, dtype=torch.float32, pin_memory=True)
    ld_ = torch.empty_like(lh, device=dev)
    for name, dst, src in (("h2d", ld_, lh), ("d2h", lh, ld_)):
        dst.copy_(src, non_blocking=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dst.copy_(src, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        out[name + "_gbs"] = (1 << 30) / (a.elapsed_time(b) * 1e-3) / 1e9
    del lh, ld_
    return out


def run_config4(args, H, torch, dev, rank):
    """64 uneven fields as the configuration states them: samples log-uniform 1e4-2e6, maps
    64^2-1024^2 at 0.5'-1', 64-4096 channels FP32 or BF16, FWHM 2.9'-6', footprint <= 150 GB
    (--c4-max-gb), gridded by one CUDA-graph-captured batch per step (TC split).  Fields are
    generated one at a time on the host and moved to the device, so host memory holds one
    field's values at most."""
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    t_gen = time.perf_counter()
    fields, est = W.config4_fields(n_fields=64, max_bytes=args.c4_max_gb * 1e9)
    plans, args_b, keep = [], [], []
    units = n_samples = n_bf16 = 0
    t_plans = 0.0
    for f in fields:
        wl = W.field_samples(f)
        g = wl["geom"]
        M = g["nx"] * g["ny"]
        N, C = wl["values"].shape
        t0 = time.perf_counter()
        plans.append(H.hegrid_plan_create(N, np.ascontiguousarray(wl["lon"]),
                                          np.ascontiguousarray(wl["lat"]), 0, g, wl["fwhm_deg"],
                                          3.0, 0, sh))
        torch.cuda.synchronize()
        t_plans += time.perf_counter() - t0
        v = torch.from_numpy(wl["values"])
        if wl["dtype"] == "bf16":
            ld = (C + 7) // 8 * 8
            dv = torch.zeros((N, ld), dtype=torch.bfloat16, device=dev)
            dv[:, :C] = v.to(torch.bfloat16).to(dev)
            dt = H.HEGRID_BF16
            n_bf16 += 1
        else:
            ld = (C + 3) // 4 * 4
            dv = torch.zeros((N, ld), dtype=torch.float32, device=dev)
            dv[:, :C] = v.to(dev)
            dt = H.HEGRID_F32
        del v, wl
        out = torch.empty((M, C), device=dev)
        args_b.append({"values": dv, "dtype": dt, "n_channels": C, "ld_values": ld,
                       "map_out": out, "ld_map": C, "weight_out": None,
                       "mode": H.HEGRID_MODE_TC_SPLIT})
        keep.append((dv, out))
        units += N * C
        n_samples += N
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen - t_plans
    dev_bytes = torch.cuda.memory_allocated(dev) + sum(H.hegrid_plan_info(p)["bytes"]
                                                       for p in plans)
    captured0 = H.hegrid_launch_count()
    batch = H.hegrid_batch_create(plans, args_b, sh)
    graph_kernels = H.hegrid_launch_count() - captured0  # kernels captured in the graph
    try:
        for _ in range(max(3, args.warmup)):
            H.hegrid_batch_launch(batch, sh)
        torch.cuda.synchronize()
        clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            H.hegrid_batch_launch(batch, sh)
        b.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        t = a.elapsed_time(b) / 1e3 / args.steps
        for p in plans:
            H.hegrid_status_poll(p)
        finite = all(bool(torch.isfinite(o).any()) for _, o in keep)
    finally:
        H.hegrid_batch_destroy(batch)
        for p in plans:
            H.hegrid_plan_destroy(p)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC.replace("plan + grid per step", "batched grid per step"),
            "value": units / t, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": t * 1e3, "higher_is_better": True,
            "dtype": "f32 or bf16 in; f16 hi/lo split, f32 accumulate", "data": "synthetic",
            "config": {"workload": "64 uneven fields (drift, raster, uniform), samples "
                                   "log-uniform 1e4-2e6, maps 64^2-1024^2 at 0.5'-1', 64-4096 "
                                   "channels FP32/BF16, FWHM 2.9'-6', one CUDA-graph batch "
                                   "(TC split)",
                       "fields": len(fields), "sample_channels": units, "samples": n_samples,
                       "bf16_fields": n_bf16, "max_channels": max(f["C"] for f in fields),
                       "max_samples": max(f["n"] for f in fields),
                       "footprint_estimate_gb": est / 1e9,
                       "device_bytes_gb": dev_bytes / 1e9,
                       "l2": "inputs larger than L2"},
            "plan_s_all_fields": t_plans, "maps_finite": finite,
            "accuracy": "parity of the batched path: tests/test_gpu_runtime.py",
            "gpu_launches": graph_kernels,
            "graph": f"{graph_kernels} kernels: one channel-maximum pass for all fields, one "
                     "grid launch per tensor-core tile width present",
            "clocks": clk, "gen_s": t_gen}), flush=True)


def run_config5(args, H, torch, dev, rank):
    """65,536 BF16 channels of 1M samples streamed from pinned host memory in 4,096-channel
    chunks (4 distinct chunks cycled, as the 131 GB band does not fit host memory)."""
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    t_gen = time.perf_counter()
    wl = W.config5()
    N = len(wl["lon"])
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    CC, NCH, NDIST = 4096, 16, 4
    chunks = []
    f32 = np.empty((N, CC), np.float32)
    for k in range(NDIST):
        W.config5_chunk(wl, k, C_chunk=CC, out=f32)
        chunks.append(torch.from_numpy(f32).to(torch.bfloat16).pin_memory())
    del f32
    t_gen = time.perf_counter() - t_gen
    host_map = torch.empty((M, NCH * CC), dtype=torch.float32, pin_memory=True)
    host_w = torch.empty(M, dtype=torch.float32, pin_memory=True)
    order = [chunks[k % NDIST] for k in range(NCH)]
    lon_h, lat_h = np.ascontiguousarray(wl["lon"]), np.ascontiguousarray(wl["lat"])
    plan = H.hegrid_plan_create(N, lon_h, lat_h, 0, g, wl["fwhm_deg"], 3.0, 0, sh)
    try:
        link = _link(torch, dev, stream)
        H.hegrid_grid_stream(plan, order, CC, H.HEGRID_BF16, H.HEGRID_MODE_TC_SPLIT, host_map,
                             NCH * CC, host_w)
        ts = time.perf_counter()
        steps = max(1, args.steps // 5)
        for _ in range(steps):
            H.hegrid_grid_stream(plan, order, CC, H.HEGRID_BF16, H.HEGRID_MODE_TC_SPLIT,
                                 host_map, NCH * CC, host_w)
        t = (time.perf_counter() - ts) / steps
        finite = bool(torch.isfinite(host_map[:, :8]).any())
    finally:
        H.hegrid_plan_destroy(plan)
    h2d = N * NCH * CC * 2
    d2h = M * NCH * CC * 4
    bound = max(h2d / link["h2d_gbs"], d2h / link["d2h_gbs"]) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": METRIC.replace("plan + grid per step", "streamed from pinned host memory"),
            "value": N * NCH * CC / t, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "ms_per_step": t * 1e3, "higher_is_better": True,
            "dtype": "bf16 in; f16 values x f16 hi/lo weights (2 MMAs), f32 accumulate",
            "data": "synthetic",
            "config": {"workload": "1M-sample 19-beam drift scan, 3.3x3.3 deg at (30,41), "
                                   f"{M} cells at 0.5', FWHM 2.9', 65,536 BF16 channels in 16 "
                                   "chunks of 4,096 (4 distinct chunks cycled)",
                       "N": N, "C": NCH * CC, "M": M},
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "link": link,
            "link_bound_ms": bound * 1e3, "link_frac": bound / t,
            "maps_finite": finite,
            "accuracy": "parity of the streaming path: tests/test_gpu_runtime.py",
            "gen_s": t_gen}), flush=True)


def run_config3(args, H, torch, dev, rank):
    """The precision variant: config 1's 20,000 uniform samples and 120 x 120 map at
    1', 16,384 channels of smooth per-source spectra, stored as BF16, FP16, BF16 hi/lo
    pairs and FP32, each through the tensor-core forms.  One line per stored type and
    form: grid time (CUDA events, values and map larger than L2, so each call streams
    from HBM), N*C/s, the HBM roofline of the algorithmic bytes (values read once at
    their stored width + FP32 map + weight map) and the error against a complete run
    of the FP64 oracle on the stored values (all cells, all channels)."""
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    t_gen = time.perf_counter()
    wl = W.config3()
    t_gen = time.perf_counter() - t_gen
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    N, C = wl["values"].shape
    hbm, _, peak_kind = _peaks()
    vt = torch.from_numpy(wl["values"])
    hi = vt.to(torch.bfloat16)
    lo = (vt - hi.float()).to(torch.bfloat16)
    h16 = vt.to(torch.float16)
    # stored type -> (values, dtype, bytes per value, the values the oracle sees)
    stored = {
        "bf16": (hi, H.HEGRID_BF16, 2, hi.float().numpy()),
        "f16": (h16, H.HEGRID_F16, 2, h16.float().numpy()),
        "bf16x2": (torch.stack([hi, lo], dim=-1).contiguous().view(torch.int32), H.HEGRID_BF16X2,
                   4, (hi.double() + lo.double()).float().numpy()),
        "f32": (vt, H.HEGRID_F32, 4, wl["values"]),
    }
    forms = [("bf16", "tc_split"), ("bf16", "tc"), ("f16", "tc_split"), ("bf16x2", "tc_split"),
             ("f32", "tc_split"), ("f32", "tc")]
    modes = {"tc_split": H.HEGRID_MODE_TC_SPLIT, "tc": H.HEGRID_MODE_TC}
    lon_d = torch.from_numpy(wl["lon"]).to(dev)
    lat_d = torch.from_numpy(wl["lat"]).to(dev)
    plan = H.hegrid_plan_create(N, lon_d, lat_d, 1, g, wl["fwhm_deg"], 3.0, 0, sh)
    if args.tc_kernel:
        H.hegrid_plan_set_tuning(plan, H.HEGRID_MODE_TC_SPLIT, 0, 0, 0, args.tc_kernel)
    out = torch.empty((M, C), device=dev)
    w_d = torch.empty(M, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, device=dev)
    info = H.hegrid_plan_info(plan)
    results = []
    oracle_cache = {}
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    try:
        for kind, form in forms:
            dv, dt, eb, seen = stored[kind]
            vd = dv.to(dev)
            md = modes[form]
            for _ in range(max(3, args.warmup)):
                H.hegrid_grid(plan, vd, dt, C, C, out, C, w_d, md, sh)
            evs = []
            l0 = H.hegrid_launch_count()
            for _ in range(max(10, args.steps)):
                flush.zero_()  # evict values and map from L2 between calls
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                H.hegrid_grid(plan, vd, dt, C, C, out, C, w_d, md, sh)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize()
            launches = (H.hegrid_launch_count() - l0) / max(10, args.steps)
            ts = sorted(a.elapsed_time(b) for a, b in evs)
            t = statistics.median(ts) / 1e3
            H.hegrid_status_poll(plan)
            bytes_alg = N * C * eb + M * C * 4 + M * 4
            rec = {"stored": kind, "form": form, "grid_ms": t * 1e3, "grid_ms_min": ts[0],
                   "value": N * C / t, "pair_channel_per_s": info["n_pairs"] * C / t,
                   "roofline": {"bound": "hbm", "achieved": bytes_alg / t / 1e9, "peak": hbm,
                                "unit": "GB/s", "frac": bytes_alg / t / 1e9 / hbm,
                                "algorithmic_bytes": bytes_alg, "peak_kind": peak_kind,
                                "limit": "not DRAM (the launch moves ~1.2x the algorithmic "
                                         "bytes, profiles/k_grid_tc_config3_bf16.md): the "
                                         "per-chunk shared-memory work of the B conversion "
                                         "and the MMA operand reads over 7,680 short work "
                                         "items (LSU shared wavefronts ~40% of peak, tensor "
                                         "pipe ~21%)"},
                   "gpu_launches_per_call": launches}
            if not args.no_cpu_baseline and rank == 0:
                if kind not in oracle_cache:  # forms of one stored type are consecutive
                    oracle_cache.clear()
                    oracle_cache[kind] = cpu_oracle_full(
                        dict(wl, values=np.ascontiguousarray(seen)))
                o, ref, Wref = oracle_cache[kind]
                rec["err_vs_oracle"] = map_errors(out.cpu().numpy(), w_d.cpu().numpy(), ref, Wref)
                rec["cpu_baseline"] = {k: o[k] for k in ("value", "unit", "cores", "kind",
                                                           "sample", "seconds")}
            results.append(rec)
            del vd
    finally:
        clk = clocks.stop()
        H.hegrid_plan_destroy(plan)
    if rank == 0:
        for rec in results:
            print(json.dumps({
                "metric": METRIC.replace("plan + grid per step", "grid call"),
                "value": rec["value"], "unit": UNIT, "n_gpus": 1, "steps": max(10, args.steps),
                "warmup": max(3, args.warmup), "ms_per_step": rec["grid_ms"],
                "higher_is_better": True,
                "dtype": (f"{rec['stored']} in; f16 " +
                          ("hi/lo split" if rec["form"] == "tc_split" else "single") +
                          ", f32 accumulate"),
                "data": "synthetic",
                "config": {"workload": "config-1 positions (20,000 uniform samples, 2x2 deg at "
                                       "(180,30)), 120x120 map at 1', FWHM 3', 16,384 channels "
                                       "of smooth spectra",
                           "N": N, "C": C, "M": M, "pairs": info["n_pairs"],
                           "stored": rec["stored"], "form": rec["form"],
                           "tc_kernel": {0: "cell-major (default)", 1: "cell-major",
                                         2: "channel-major",
                                         3: "cell-major, dense A tiles"}[args.tc_kernel],
                           "l2": "L2 flushed (a 258 MB buffer zeroed) before every timed call"},
                **{k: rec[k] for k in rec if k not in ("value", "stored", "form")},
                "clocks": clk, "gen_s": t_gen}), flush=True)


def run_profile_case(args, H, torch, dev, rank):
    """Small cases of the tensor-core grid kernel for profiler captures (a few GB on the
    device): profile-drift is the drift scan over 2.5 x 2.5 deg at (30, 41) (the bench
    workload's density and kernel) with 256 FP32 channels; profile-cfg3 is config 3 with
    its 16,384 channels stored as BF16.  Four split-form grid calls on one plan; prints
    the time of the last."""
    s = torch.cuda.current_stream(dev).cuda_stream
    if args.workload == "profile-drift":
        wl = W.config2(C=256, size_deg=2.5)
        vals = torch.from_numpy(wl["values"]).to(dev)
        dt = H.HEGRID_F32
    else:
        wl = W.config3()
        vals = torch.from_numpy(wl["values"]).to(torch.bfloat16).to(dev)
        dt = H.HEGRID_BF16
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    N, C = wl["values"].shape
    lon = torch.from_numpy(wl["lon"]).to(dev)
    lat = torch.from_numpy(wl["lat"]).to(dev)
    plan = H.hegrid_plan_create(N, lon, lat, 1, g, wl["fwhm_deg"], 3.0, 0, s)
    try:
        if args.tc_kernel:
            H.hegrid_plan_set_tuning(plan, H.HEGRID_MODE_TC_SPLIT, 0, 0, 0, args.tc_kernel)
        out = torch.empty((M, C), device=dev)
        for _ in range(3):
            H.hegrid_grid(plan, vals, dt, C, C, out, C, None, H.HEGRID_MODE_TC_SPLIT, s)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        H.hegrid_grid(plan, vals, dt, C, C, out, C, None, H.HEGRID_MODE_TC_SPLIT, s)
        b.record()
        torch.cuda.synchronize()
        H.hegrid_status_poll(plan)
        info = H.hegrid_plan_info(plan)
    finally:
        H.hegrid_plan_destroy(plan)
    if rank == 0:
        print(json.dumps({"report": args.workload, "N": N, "C": C, "M": M,
                          "pairs": info["n_pairs"], "grid_ms": a.elapsed_time(b)}), flush=True)


# Table 3 (Sec. 5.2): HEGrid's end-to-end times in seconds on a V100 for the simulated
# survey (50 channels) at each sample count; context only (another machine, and the paper's
# times include reading the input files).
SIM_SIZES = (15_000_000, 16_000_000, 17_000_000, 18_000_000, 19_000_000)
PAPER_V100_S = {15_000_000: 30.21, 16_000_000: 32.77, 17_000_000: 35.27, 18_000_000: 38.20,
                19_000_000: 40.94}


def run_sim(args, H, torch, dev, rank):
    """The paper's simulated survey (Table 2): 60 x 20 deg at (30, 41), 1 arcmin cells,
    180 arcsec beam, 50 FP32 channels, 1.5e7 - 1.9e7 uniform samples.  Each step is the whole
    pipeline (plan + grid); every sample count of Table 3 is timed with inputs resident on the
    device and end to end from pinned host buffers to a pinned host map."""
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    C = 50
    sizes = SIM_SIZES if not args.sim_n else (args.sim_n,)
    paper = PAPER_V100_S if args.sim_span == 60.0 else {}
    nmax = max(sizes)
    t_gen = time.perf_counter()
    host_vals = torch.empty((nmax, C), dtype=torch.float32, pin_memory=True)
    wl = W.sim_survey(n=nmax, C=C, out=host_vals.numpy(), lon_span=args.sim_span)
    t_gen = time.perf_counter() - t_gen
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    # coordinates in pinned host memory, like the values
    lon_h = torch.from_numpy(np.ascontiguousarray(wl["lon"])).pin_memory().numpy()
    lat_h = torch.from_numpy(np.ascontiguousarray(wl["lat"])).pin_memory().numpy()
    ldv = (C + 3) // 4 * 4  # device rows padded to 16 bytes
    vals_d = torch.zeros((nmax, ldv), dtype=torch.float32, device=dev)
    vals_d[:, :C].copy_(host_vals.to(dev))
    lon_d = torch.from_numpy(lon_h).to(dev)
    lat_d = torch.from_numpy(lat_h).to(dev)
    map_d = torch.empty((M, C), device=dev)
    w_d = torch.empty(M, device=dev)
    host_map = torch.empty((M, C), dtype=torch.float32, pin_memory=True)
    host_w = torch.empty(M, dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    modes = {"tc_split": H.HEGRID_MODE_TC_SPLIT, "fp32": H.HEGRID_MODE_FP32}
    nmid = sizes[len(sizes) // 2]

    # the form (FP32 or split tensor core, both within the parity bound) and its launch
    # shape, chosen on the middle sample count outside the timed region
    tune = {}
    flags = H.HEGRID_PLAN_HEALPIX(args.healpix) if args.healpix else 0
    if not args.no_tune and not args.healpix:
        flags, bin_ms = H.hegrid_autotune_bins(nmid, lon_d, lat_d, 1, g, wl["fwhm_deg"], 3.0, sh)
        tune["bin_cells"] = flags
        tune["plan_ms_by_bin"] = [round(x, 3) for x in bin_ms]
    p = H.hegrid_plan_create(nmid, lon_d, lat_d, 1, g, wl["fwhm_deg"], 3.0, flags, sh)
    forms = {}
    try:
        for nm, md in modes.items():
            if args.mode not in ("auto", nm):
                continue
            q = {}
            if not args.no_tune:
                rep = H.hegrid_autotune(p, vals_d, H.HEGRID_F32, C, ldv, md, sh)
                best = rep["points"][rep["best"]]
                q = {"band": best["band"], "seg": best["seg"], "group": best["group"],
                     "kernel": best["kernel"], "ms": best["ms"]}
                H.hegrid_plan_set_tuning(p, md, best["band"], best["seg"], best["group"],
                                         best["kernel"])
            H.hegrid_grid(p, vals_d, H.HEGRID_F32, C, ldv, map_d, C, w_d, md, sh)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                H.hegrid_grid(p, vals_d, H.HEGRID_F32, C, ldv, map_d, C, w_d, md, sh)
            b.record(stream)
            torch.cuda.synchronize()
            q["grid_ms"] = a.elapsed_time(b) / 3
            forms[nm] = q
        info = H.hegrid_plan_info(p)
    finally:
        H.hegrid_plan_destroy(p)
    mode_name = min(forms, key=lambda k: forms[k]["grid_ms"])
    mode = modes[mode_name]
    shape = forms[mode_name]

    def new_plan(n, lon, lat, on_device):
        pl = H.hegrid_plan_create(n, lon, lat, on_device, g, wl["fwhm_deg"], 3.0, flags, sh)
        if "band" in shape:
            H.hegrid_plan_set_tuning(pl, mode, shape["band"], shape["seg"], shape.get("group", 0),
                                     shape.get("kernel", 0))
        return pl

    link = _link(torch, dev, stream)
    rows = []
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    launches = 0
    # device-timed steps at every sample count (clocks sampled meanwhile)
    for n in sizes:
        ev = []
        l0 = H.hegrid_launch_count()
        for i in range(args.warmup + args.steps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            pl = new_plan(n, lon_d, lat_d, 1)
            e1.record(stream)
            H.hegrid_grid(pl, vals_d, H.HEGRID_F32, C, ldv, map_d, C, w_d, mode, sh)
            e2.record(stream)
            H.hegrid_plan_destroy(pl)
            if i >= args.warmup:
                ev.append((e0, e1, e2))
        torch.cuda.synchronize()
        if n == nmid:
            launches = (H.hegrid_launch_count() - l0) / (args.warmup + args.steps)
        t_dev = statistics.mean(a.elapsed_time(c) for a, b, c in ev) / 1e3
        t_plan = statistics.mean(a.elapsed_time(b) for a, b, c in ev) / 1e3
        t_grid = statistics.mean(b.elapsed_time(c) for a, b, c in ev) / 1e3
        rows.append({"N": n, "device_ms": t_dev * 1e3, "plan_ms": t_plan * 1e3,
                     "grid_ms": t_grid * 1e3, "device_contrib_per_s": n * C / t_dev})
    clk = clocks.stop()

    # end to end at every sample count, after the sampler has stopped (its
    # nvidia-smi queries contend with the host-side CUDA calls of these steps)
    sample_cells = np.sort(np.random.default_rng(7).choice(M, 256, replace=False))
    sampled = None
    for r in rows:
        n = r["N"]

        def e2e_step():
            pl = new_plan(n, lon_h[:n], lat_h[:n], 0)
            H.hegrid_grid_stream(pl, [host_vals[:n]], C, H.HEGRID_F32, mode, host_map, C, host_w)
            H.hegrid_plan_destroy(pl)

        e2e_step()
        torch.cuda.synchronize()
        te = []
        for _ in range(max(1, args.e2e_steps)):
            ts = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            te.append(time.perf_counter() - ts)
        # median of the steps: a host-side hiccup in one step (seen as single
        # steps of 2-3x the others) does not move it; the mean is reported too
        t_e2e = statistics.median(te)
        if n == nmid:
            sampled = host_map[torch.from_numpy(sample_cells)].numpy().astype(np.float64)
        h2d = n * 16 + n * C * 4
        d2h = M * C * 4 + M * 4
        r.update({"e2e_ms": t_e2e * 1e3, "e2e_mean_ms": statistics.mean(te) * 1e3,
                  "e2e_contrib_per_s": n * C / t_e2e,
                  "h2d_bytes": h2d, "d2h_bytes": d2h,
                  "link_bound_ms": max(h2d / link["h2d_gbs"], d2h / link["d2h_gbs"]) / 1e6,
                  "paper_v100_s": paper.get(n),
                  "paper_v100_contrib_per_s": n * C / paper[n] if n in paper else None})
    head = next(r for r in rows if r["N"] == nmid)
    finite = bool(torch.isfinite(host_map[:: max(1, M // 4096)]).all())

    # CPU baseline: the FP64 oracle on every 100th map row at the headline sample count,
    # and its values on 256 sampled cells of the end-to-end map of that count
    cpu, err = None, None
    if rank == 0 and not args.no_cpu_baseline:
        keep = {}
        cpu = cpu_oracle_sample({"lon": lon_h[:nmid], "lat": lat_h[:nmid], "geom": g,
                                 "fwhm_deg": wl["fwhm_deg"], "support": 3.0,
                                 "values": host_vals.numpy()[:nmid]}, frac_rows=100, keep=keep)
        ref, Wref = keep["index"].grid(host_vals.numpy()[:nmid], cells=sample_cells)
        mask = Wref >= 1e-3 * Wref.max()
        rms = np.sqrt(np.mean(ref[mask] ** 2, axis=0))
        e = np.max(np.abs(sampled[mask] - ref[mask]), axis=0) / rms
        err = {mode_name: {"max": float(e.max()), "median": float(np.median(e)),
                           "cells": int(mask.sum()), "map": "end-to-end host map"}}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": head["device_contrib_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["device_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": FORM_DTYPE[mode_name], "data": "synthetic",
            "config": {"workload": f"simulated survey (Table 2): {g['nx'] / 60:g}x20 deg at "
                                   f"({g['lon0']:g},41), {g['nx']}x1200 map at 1', FWHM 180'', "
                                   "R=3 sigma, 50 FP32 channels, uniform samples, "
                                   f"headline N={nmid}",
                       "N": nmid, "C": C, "M": M, "pairs": info["n_pairs"], "mode": mode_name,
                       "l2": "inputs larger than L2 (values 3.4 GB)",
                       "tuning": tune, "forms": forms,
                       "binning": (f"HEALPix RING nside {1 << args.healpix}" if args.healpix
                                   else "map bins")},
            "e2e": {"value": head["e2e_contrib_per_s"], "unit": UNIT,
                    "h2d_bytes_per_step": head["h2d_bytes"],
                    "d2h_bytes_per_step": head["d2h_bytes"], "ms_per_step": head["e2e_ms"],
                    "path": "hegrid_plan_create(host coords) + hegrid_grid_stream(one pinned "
                            "50-channel chunk -> pinned host map)"},
            "table3": rows, "link": link, "maps_finite": finite,
            "cpu_baseline": cpu, "err_vs_oracle": err,
            "accuracy": "parity on this workload's shape: tests/test_gpu_sim.py",
            "gpu_launches": launches, "clocks": clk, "gen_s": t_gen}), flush=True)


def run_sweep(args, H, torch, dev, rank):
    """The paper's concurrency and reuse studies (Sec. 5.3: thread-block size with L1/L2 hit
    rates, stream count, thread-level reuse), as reports of this design's knobs on the
    FAST-like drift scan: the plan's bin edge and HEALPix nside (the index resolution), the
    grid step's launch shapes (band width: which cell blocks run together and share sample
    rows in L2; segment length), the streaming path's chunk count (copy/compute overlap),
    and the reuse a 16x8 cell block gets from one staged candidate list."""
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    pos = W.config2(with_values=False, C=args.channels)
    N = len(pos["lon"])
    C = args.channels
    host_vals = torch.empty((N, C), dtype=torch.float32, pin_memory=True)
    wl = W.config2(C=C, out=host_vals.numpy())
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    fw = wl["fwhm_deg"]
    lon_d = torch.from_numpy(wl["lon"]).to(dev)
    lat_d = torch.from_numpy(wl["lat"]).to(dev)
    vals_d = host_vals.to(dev)
    torch.cuda.synchronize()

    def plan_ms(flags, reps=3):
        p = H.hegrid_plan_create(N, lon_d, lat_d, 1, g, fw, 3.0, flags, sh)
        H.hegrid_plan_destroy(p)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            p = H.hegrid_plan_create(N, lon_d, lat_d, 1, g, fw, 3.0, flags, sh)
            H.hegrid_plan_destroy(p)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    # index resolution: map-bin edge 1..4 cells, HEALPix nside 2^10..2^13
    index = [{"binning": f"map bins {B}", "plan_ms": plan_ms(B)} for B in (1, 2, 3, 4)]
    index += [{"binning": f"HEALPix nside {1 << k}", "plan_ms": plan_ms(H.HEGRID_PLAN_HEALPIX(k))}
              for k in (10, 11, 12, 13)]
    # the same map as a Sanson-Flamsteed grid (cells dlon apart along each parallel)
    index.append({"binning": "map bins 2, Sanson-Flamsteed map",
                  "plan_ms": plan_ms(H.HEGRID_PLAN_SFL)})

    # launch shapes of the grid step (both tensor-core forms and the FP32 form)
    p = H.hegrid_plan_create(N, lon_d, lat_d, 1, g, fw, 3.0, 0, sh)
    info = H.hegrid_plan_info(p)
    shapes = {}
    try:
        for nm, md in (("tc_split", H.HEGRID_MODE_TC_SPLIT), ("fp32", H.HEGRID_MODE_FP32)):
            rep = H.hegrid_autotune(p, vals_d, H.HEGRID_F32, C, C, md, sh)
            shapes[nm] = [{"band": q["band"], "seg": q["seg"], "group": q["group"],
                           "kernel": q["kernel"], "grid_ms": q["ms"]}
                          for q in rep["points"]]
        # streaming: the same plan, C channels from pinned host memory in k chunks
        host_map = torch.empty((M, C), dtype=torch.float32, pin_memory=True)
        streams = []
        for k in (1, 2, 4, 8, 16):
            if C % k:
                continue
            cc = C // k
            chunks = [host_vals[:, i * cc:(i + 1) * cc].contiguous().pin_memory() for i in range(k)]
            H.hegrid_grid_stream(p, chunks, cc, H.HEGRID_F32, H.HEGRID_MODE_TC_SPLIT, host_map, C,
                                 None)
            ts = time.perf_counter()
            for _ in range(3):
                H.hegrid_grid_stream(p, chunks, cc, H.HEGRID_F32, H.HEGRID_MODE_TC_SPLIT,
                                     host_map, C, None)
            streams.append({"chunks": k, "chunk_channels": cc,
                            "ms": (time.perf_counter() - ts) / 3 * 1e3})
            del chunks
        # per-channel masking: two passes of the plan (values with non-finite entries
        # zeroed, then the 0/1 mask) against one plain pass, 1% of the values NaN
        vm = vals_d.clone()
        vm.view(-1)[::97] = float("nan")
        out = torch.empty((M, C), device=dev)
        masked = {}
        for nm, fn in (("grid_ms", lambda: H.hegrid_grid(p, vm, H.HEGRID_F32, C, C, out, C, None,
                                                         H.HEGRID_MODE_TC_SPLIT, sh)),
                       ("masked_grid_ms", lambda: H.hegrid_grid_masked(
                           p, vm, H.HEGRID_F32, C, C, out, C, None, H.HEGRID_MODE_TC_SPLIT, sh))):
            fn()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            masked[nm] = a.elapsed_time(b) / 3
        del vm, out
    finally:
        H.hegrid_plan_destroy(p)
    for r in streams:
        r["speedup_vs_one_chunk"] = streams[0]["ms"] / r["ms"]
    # reuse (the paper's gamma: cells sharing one contribution region): each candidate row
    # staged for a 16x8 cell block serves all 128 of its cells
    P, K = info["n_pairs"], info["n_cand"]
    reuse = {"pairs": P, "candidate_slots": K, "blocks": info["n_blocks"],
             "samples_needed_per_cell": P / M, "rows_staged_per_cell": K / M,
             "reuse_factor": P / K, "dense_macs_per_useful": K * 128 / P}
    if rank == 0:
        print(json.dumps({
            "report": "concurrency and reuse sweeps (Sec. 5.3 analogues)",
            "config": {"workload": workload_desc(N, C), "N": N, "C": C, "M": M},
            "index_resolution": index, "launch_shapes": shapes, "streaming": streams,
            "masking": masked,
            "reuse": reuse}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="auto", choices=["auto", "tc_split", "tc", "fp32"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--channels", type=int, default=1024)
    ap.add_argument("--shape", default="",
                    help="band,seg,group,kernel (as --shape=-8,16,0,3): apply this launch shape (bin edge 2) "
                         "instead of running the autotuner (profiler captures of the shape "
                         "the autotuner keeps)")
    ap.add_argument("--plan-tiles", default="on", choices=["on", "off"],
                    help="with a tuned kernel that reads dense weight tiles: have plan creation "
                         "write them (on) or the first grid call build them (off)")
    ap.add_argument("--step-priority", default="normal", choices=["normal", "high"],
                    help="priority of the step's stream against the side stream of the "
                         "channel-maximum pass")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (default launch shapes, bin edge 2)")
    ap.add_argument("--workload", default="config2",
                    choices=["config2", "config3", "config4", "config5", "sim", "sweep",
                             "profile-drift", "profile-cfg3"],
                    help="config2 (default): the bench line; config3: 16,384 channels stored "
                         "as BF16, FP16, BF16 hi/lo and FP32, one line per stored type and "
                         "tensor-core form; profile-drift / profile-cfg3: small cases of the "
                         "grid kernel for profiler captures; config4: 64 uneven fields in one "
                         "graph-captured batch; config5: 65,536 BF16 channels streamed from "
                         "pinned host memory; sim: the paper's 60x20 deg simulated survey "
                         "at every sample count of Table 3, plan + grid, device and end to "
                         "end")
    ap.add_argument("--c4-max-gb", type=float, default=150.0,
                    help="config4: device footprint cap of the 64 fields (GB)")
    ap.add_argument("--healpix", type=int, default=0,
                    help="bin the samples by HEALPix RING-scheme pixels at nside 2^K (the "
                         "paper's own index) instead of map bins; 0: map bins")
    ap.add_argument("--sim-n", type=int, default=0,
                    help="sim workload: time this one sample count only")
    ap.add_argument("--sim-span", type=float, default=60.0,
                    help="sim workload: RA span of the field in degrees (60: the paper's; "
                         "smaller: a cut of it, for profiler captures)")
    ap.add_argument("--tc-kernel", type=int, default=0, choices=[0, 1, 2, 3],
                    help="config3 / profile-drift / profile-cfg3: tensor-core kernel (1 "
                         "cell-major, 2 channel-major, 3 cell-major with dense A tiles; 0 the "
                         "library's default)")
    ap.add_argument("--lean", action="store_true",
                    help="timed steps only (no per-form timings, accuracy check, e2e or CPU "
                         "baseline): the command used for profiler captures")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    from paper_2207_04584_gb300 import hegrid as H
    H.lib()
    if args.workload == "config3":
        return run_config3(args, H, torch, dev, rank)
    if args.workload.startswith("profile-"):
        return run_profile_case(args, H, torch, dev, rank)
    if args.workload == "config4":
        return run_config4(args, H, torch, dev, rank)
    if args.workload == "config5":
        return run_config5(args, H, torch, dev, rank)
    if args.workload == "sim":
        return run_sim(args, H, torch, dev, rank)
    if args.workload == "sweep":
        return run_sweep(args, H, torch, dev, rank)

    # ---- workload (config 2: FAST-like drift scan, FP32 values) ----------
    t_gen = time.perf_counter()
    pos = W.config2(with_values=False, C=args.channels)
    N = len(pos["lon"])
    C = args.channels
    host_vals = torch.empty((N, C), dtype=torch.float32, pin_memory=True)
    wl = W.config2(C=C, out=host_vals.numpy())
    t_gen = time.perf_counter() - t_gen
    g = wl["geom"]
    M = g["nx"] * g["ny"]
    lon_d = torch.from_numpy(wl["lon"]).to(dev)
    lat_d = torch.from_numpy(wl["lat"]).to(dev)
    vals_d = host_vals.to(dev)
    map_d = torch.empty((M, C), device=dev)
    w_d = torch.empty(M, device=dev)
    if args.step_priority == "high":
        # the step's own stream above the side stream of the channel-maximum
        # pass, so that the plan's kernels are scheduled first
        stream = torch.cuda.Stream(dev, priority=-1)
        torch.cuda.set_stream(stream)
    else:
        stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    modes = {"tc_split": H.HEGRID_MODE_TC_SPLIT, "tc": H.HEGRID_MODE_TC,
             "fp32": H.HEGRID_MODE_FP32}
    mode_name = args.mode
    if mode_name == "auto":
        mode_name = "tc_split"
        try:
            p = H.hegrid_plan_create(64, wl["lon"][:64].copy(), wl["lat"][:64].copy(), 0, g,
                                     wl["fwhm_deg"], 3.0, 0, sh)
            try:
                H.hegrid_grid(p, vals_d, H.HEGRID_F32, C, C, map_d, C, w_d,
                              H.HEGRID_MODE_TC_SPLIT, sh)
            finally:
                H.hegrid_plan_destroy(p)
        except H.HegridError:
            mode_name = "fp32"
    mode = modes[mode_name]

    # ---- autotuning, outside the timed region: the plan's bin edge and the
    # grid step's launch shape, applied to every plan the steps create -----
    tune = {}
    hpx_flag = H.HEGRID_PLAN_HEALPIX(args.healpix) if args.healpix else 0
    if args.shape:
        b_, s_, g_, k_ = (int(x) for x in args.shape.split(","))
        tune = {"bin_cells": hpx_flag or 2, "band": b_, "seg": s_, "group": g_, "kernel": k_,
                "given": True}
    elif not args.no_tune:
        t_tune = time.perf_counter()
        if args.healpix:
            bin_cells, bin_ms = hpx_flag, []
        else:
            bin_cells, bin_ms = H.hegrid_autotune_bins(N, lon_d, lat_d, 1, g, wl["fwhm_deg"],
                                                       3.0, sh)
        p = H.hegrid_plan_create(N, lon_d, lat_d, 1, g, wl["fwhm_deg"], 3.0, bin_cells, sh)
        try:
            rep = H.hegrid_autotune(p, vals_d, H.HEGRID_F32, C, C, mode, sh)
        finally:
            H.hegrid_plan_destroy(p)
        best = rep["points"][rep["best"]]
        tune = {"bin_cells": bin_cells, "band": best["band"], "seg": best["seg"], "group": best["group"],
                "kernel": best["kernel"],
                "plan_ms_by_bin": [round(x, 3) for x in bin_ms],
                "grid_ms_by_shape": [[q["band"], q["seg"], q["group"], q["kernel"], round(q["ms"], 3)]
                                     for q in rep["points"]],
                "seconds": round(time.perf_counter() - t_tune, 2)}
    flags = tune.get("bin_cells", hpx_flag)
    # Kernels 2 and 3 read dense weight tiles: plan creation writes them
    # (HEGRID_PLAN_DENSE_TILES) unless --plan-tiles off, when the first grid
    # call builds them.
    if tune.get("kernel", 0) in (2, 3):
        tune["plan_tiles"] = args.plan_tiles == "on"
        if tune["plan_tiles"]:
            flags |= H.HEGRID_PLAN_DENSE_TILES

    def new_plan(lon, lat, on_device):
        p = H.hegrid_plan_create(N, lon, lat, on_device, g, wl["fwhm_deg"], 3.0, flags, sh)
        if tune:
            H.hegrid_plan_set_tuning(p, mode, tune["band"], tune["seg"], tune["group"],
                                     tune["kernel"])
        return p

    ev = []
    # Tensor-core modes: each channel's largest |v| (which sets its FP16 scale)
    # depends on the values only, so the step computes it on a side stream
    # while the plan is created (HBM-bound beside instruction-bound work) and
    # grids with the precomputed maxima.
    overlap = mode != H.HEGRID_MODE_FP32
    side = torch.cuda.Stream(dev)
    chmax_d = torch.empty(C, dtype=torch.int32, device=dev)

    def step(record):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if overlap:
            side.wait_event(e0)
            H.hegrid_chan_maxima(vals_d, H.HEGRID_F32, N, C, C, chmax_d, H.HEGRID_MAXIMA_BESIDE,
                                 side.cuda_stream)
            es = torch.cuda.Event()
            es.record(side)
        plan = new_plan(lon_d, lat_d, 1)
        e1.record(stream)
        if overlap:
            stream.wait_event(es)
            H.hegrid_grid_prescaled(plan, vals_d, H.HEGRID_F32, C, C, chmax_d, map_d, C, w_d,
                                    mode, sh)
        else:
            H.hegrid_grid(plan, vals_d, H.HEGRID_F32, C, C, map_d, C, w_d, mode, sh)
        e2.record(stream)
        H.hegrid_plan_destroy(plan)
        if record:
            ev.append((e0, e1, e2))
        return plan

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = H.hegrid_launch_count()
    clocks = ClockSampler(local_rank)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(True)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    launches = (H.hegrid_launch_count() - launches0) // max(1, args.steps)
    elapsed = max_over_ranks(t0.elapsed_time(t1) / 1e3, dist, dev)
    t_plan = statistics.mean(a.elapsed_time(b) for a, b, c in ev) / 1e3
    t_grid = statistics.mean(b.elapsed_time(c) for a, b, c in ev) / 1e3
    value = job_value(N * C * args.steps, world, elapsed)

    # plan facts, per-form timings, and each form's whole map (compared with
    # the FP64 oracle's complete run in the CPU-baseline leg below)
    maps = {}
    plan = new_plan(lon_d, lat_d, 1)
    info = H.hegrid_plan_info(plan)
    P = info["n_pairs"]
    forms = {}
    err = {}
    for nm, md in ([] if args.lean else modes.items()):
        try:
            H.hegrid_grid(plan, vals_d, H.HEGRID_F32, C, C, map_d, C, w_d, md, sh)
        except H.HegridError as e:
            forms[nm] = {"unavailable": str(e)}
            continue
        torch.cuda.synchronize()
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        es.record(stream)
        for _ in range(reps):
            H.hegrid_grid(plan, vals_d, H.HEGRID_F32, C, C, map_d, C, w_d, md, sh)
        ee.record(stream)
        torch.cuda.synchronize()
        tg = es.elapsed_time(ee) / 1e3 / reps
        forms[nm] = {"grid_ms": tg * 1e3, "grid_contrib_per_s": N * C / tg,
                     "pair_channel_per_s": P * C / tg, "dtype": FORM_DTYPE[nm]}
        if not args.no_cpu_baseline and rank == 0:
            maps[nm] = (map_d.cpu().numpy(), w_d.cpu().numpy())
    H.hegrid_plan_destroy(plan)

    # ---- roofline of the dominant kernel (the grid step) ------------------
    hbm, tc_peak, peak_kind = _peaks()
    alg_bytes = N * C * 4 + M * C * 4 + M * 4
    # FP32 FMA peak of this GPU, measured (the plain form's ALU roofline)
    fp32_peak = H.hegrid_fp32_peak(sh)
    if "fp32" in forms and "grid_ms" in forms["fp32"]:
        f = 2.0 * P * C / (forms["fp32"]["grid_ms"] * 1e-3) / 1e12
        forms["fp32"]["useful_tflops"] = f
        forms["fp32"]["alu_frac"] = f / fp32_peak
    if mode == H.HEGRID_MODE_FP32:
        peak = fp32_peak
        achieved = 2.0 * P * C / t_grid / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": measured_traffic("k_grid_f32"),
                "note": "FP32 FMA peak measured by hegrid_fp32_peak (independent FMA chains "
                        "on every SM); achieved = 2 P C / grid-kernel time"}
    else:
        achieved = alg_bytes / t_grid / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm,
                "traffic": measured_traffic({1: "k_grid_tc", 3: "k_grid_tc_dense"}.get(
                    tune.get("kernel", 1), "")),
                "kernel": {1: "k_grid_tc (cell-major)", 2: "k_grid_tcm (channel-major)",
                           3: "k_grid_tc (cell-major, dense A tiles)"}.get(tune.get("kernel", 1),
                                                                          "k_grid_tc"),
                "note": f"algorithmic bytes N*C*4 + M*C*4 + M*4 per grid call / the device "
                        f"time of hegrid_grid_prescaled in the timed steps ("
                        + ("the grid kernel alone: plan creation wrote the dense weight tiles"
                           if tune.get("plan_tiles") else
                           "the grid kernel, plus the dense weight-tile build for the kernels "
                           "that read them" if tune.get("kernel", 1) in (2, 3) else
                           "the grid kernel alone")
                        + f"; the per-channel maximum pass runs beside plan creation); "
                        f"peak {peak_kind}"}

    # ---- end to end through the C ABI with host buffers -------------------
    e2e = None
    if args.e2e_steps > 0 and not args.lean:
        host_map = torch.empty((M, C), dtype=torch.float32, pin_memory=True)
        host_w = torch.empty(M, dtype=torch.float32, pin_memory=True)
        # coordinates in pinned host memory, like the values
        lon_h = torch.from_numpy(np.ascontiguousarray(wl["lon"])).pin_memory().numpy()
        lat_h = torch.from_numpy(np.ascontiguousarray(wl["lat"])).pin_memory().numpy()
        # 8 chunks: the copy/compute overlap leaves the shortest tail (sweep report)
        n_chunks = 8 if C % 8 == 0 else 1
        cc = C // n_chunks
        chunks = [torch.empty((N, cc), dtype=torch.float32, pin_memory=True)
                  for _ in range(n_chunks)]
        for k in range(n_chunks):
            chunks[k].copy_(host_vals[:, k * cc:(k + 1) * cc])

        def e2e_step():
            p = new_plan(lon_h, lat_h, 0)
            H.hegrid_grid_stream(p, chunks, cc, H.HEGRID_F32, mode, host_map, C, host_w)
            H.hegrid_plan_destroy(p)

        # the host link: one pinned 1 GiB copy each way, timed on the device
        link = _link(torch, dev, stream)
        e2e_step()
        torch.cuda.synchronize()
        ts = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        te = (time.perf_counter() - ts) / args.e2e_steps
        e2e = {"value": world * N * C / te, "unit": UNIT,
               "h2d_bytes_per_step": N * 16 + N * C * 4,
               "d2h_bytes_per_step": M * C * 4 + M * 4, "ms_per_step": te * 1e3,
               "link": link,
               "link_bound_ms": max((N * 16 + N * C * 4) / link["h2d_gbs"],
                                    (M * C * 4 + M * 4) / link["d2h_gbs"]) / 1e6,
               "path": f"hegrid_plan_create(host coords) + hegrid_grid_stream({n_chunks} pinned "
                       "channel chunks -> pinned host map)"}

    # ---- CPU baseline: one complete run of the FP64 oracle on the host cores
    # (every cell, every channel), and each form's map against it -------------
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and not args.lean:
        cpu, ref, Wref = cpu_oracle_full(wl)
        for nm, (got, gw) in maps.items():
            err[nm] = map_errors(got, gw, ref, Wref)
        del ref, Wref, maps
        # the same oracle on one host core, on every 100th map row (extrapolated)
        one = cpu_oracle_sample(wl, frac_rows=100, nthreads=1)
        cpu["single_thread"] = {"value": one["value"], "cores": 1, "sample": one["sample"],
                                "extrapolated": True}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": FORM_DTYPE[mode_name], "data": "synthetic",
                "config": workload_config(N, C, M, world),
                "form": mode_name, "pairs": P, "tuning": tune,
                "binning": (f"HEALPix RING nside {1 << args.healpix}" if args.healpix
                            else "map bins"),
                "plan_ms": t_plan * 1e3, "grid_ms": t_grid * 1e3,
                "step_structure": ("plan creation, with the per-channel maxima of the values "
                                   "on a side stream beside it (hegrid_chan_maxima), then "
                                   "hegrid_grid_prescaled" if overlap else
                                   "plan creation, then hegrid_grid"),
                "forms": forms, "fp32_peak_tflops": fp32_peak, "err_vs_oracle": err,
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "gen_s": t_gen}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
