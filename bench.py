"""Benchmark of the APPGA hot path on GB300.

One step = one APPGA iteration (steps a0-a6: extrapolation, forward projection
with the Poisson-ratio epilogue, transposed-CSR back-projection, SHOITV
stencil, EM-preconditioned projected update, FP64 objective) of a 256x256
slice with 180 angles x 367 bins.  The timed steps run as back-to-back
reconstructions of 500 iterations each (the workload's iteration count),
each from the TMC initial image.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun) every rank reconstructs its own slice (independent
replicas, weak scaling); rank 0 prints one JSON line.
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
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "APPGA iters/s per 256² slice & projector HBM GB/s; p50/p99 recon latency"
UNIT = "iters/s"
GEOM = "256"
COUNTS = 1e6
OMEGA = 0.5
LAM1, LAM2, EPS = 0.1, 0.05, 1e-3
ITERS_PER_RECON = 500
WORKLOAD = ("single 256x256 slice, parallel beam 180 angles x 367 bins, Siddon CSR A "
            "(15.02M nnz, FP32 values, int32 columns) + transposed CSR, lesion phantom, "
            "1e6 counts, gamma 10%, lambda1/lambda2 0.1/0.05, eps 1e-3, omega 0.5, beta 1, "
            "FP64 objective every iteration; 500-iteration reconstructions back to back")


BATCH_K = 64
BATCH_ITERS = 200
SERVE_GEOMS = ("128", "256", "400")
SERVE_RATE = 100.0
SERVE_SLOTS = 0  # adaptive pool widths (32 / 64 / 128 slots by demand)
SERVE_STEPS = 8
SAT_RATE = 400.0      # requests/s of the saturated serving leg
SAT_REQUESTS = 1500


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=1000)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fold", choices=("auto", "on", "off"), default="auto",
                    help="quarter-turn folded loop for the main single-slice leg: auto folds "
                         "only when the folded streams still exceed L2 (the timed inputs stay "
                         "larger than L2); the other layout is reported beside it")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="wall-time bound of the reference arm's timed oracle steps")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-slice batched leg")
    ap.add_argument("--no-other-layout", action="store_true",
                    help="skip the single-slice loop in the other matrix layout")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-large", action="store_true", help="skip the 120 x 512^2 batched leg")
    ap.add_argument("--no-volume", action="store_true",
                    help="skip the 64-slice 3-D SHOITV volume leg")
    ap.add_argument("--no-afppa", action="store_true",
                    help="skip the AFPPA (non-smooth HOITV) and figures-of-merit legs")
    ap.add_argument("--volume-only", action="store_true",
                    help="run only the volume leg and print its JSON (for profiling)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-slots", type=int, default=SERVE_SLOTS, choices=(0, 32, 64, 128),
                    help="slots per server pool (0: adaptive widths)")
    ap.add_argument("--serve-steps", type=int, default=SERVE_STEPS,
                    help="APPGA maps per graph replay of a server pool")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving leg and print its JSON (for tuning)")
    ap.add_argument("--serve-rate", type=float, default=SERVE_RATE,
                    help="Poisson arrival rate of the serving stream (requests/s)")
    ap.add_argument("--serve-max-pools", type=int, default=0,
                    help="cap on the server's live pools (0: none)")
    ap.add_argument("--serve-geom-pools", type=int, default=2,
                    help="cap on the server's live pools per geometry (0: none)")
    return ap.parse_args()


# ----------------------------------------------------------------- inputs

def make_inputs(rank: int):
    from paper_2409_13344_gb300 import workload as W
    geom = W.GEOMETRIES[GEOM]
    A = W.system_matrix(GEOM)
    sl = W.make_slice(A, geom, COUNTS, W.seed_for(2, rank), phantom="lesions")
    return geom, A, sl


# ------------------------------------------------------------- clock sampling

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, period_ms: int = 100):
        self.period = period_ms
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 f"-lms", str(self.period)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        idxs = sorted({r[0] for r in rows})
        want = vis.split(",")[0] if vis and vis.split(",")[0].isdigit() and vis.split(",")[0] in idxs \
            else idxs[0]
        rows = [r for r in rows if r[0] == want]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- roofline data

def kernel_bytes(m: int, d: int, nnz: int, per_nnz: int = 8, sliced: bool = False,
                 folded: bool = False):
    """Algorithmic bytes per launch of the two iteration kernels: the stored
    matrix stream at `per_nnz` bytes per nonzero (8: FP32 values and 4-byte
    column indices; 6: FP32 values and 2-byte packed columns, or BF16 values
    and 4-byte columns), its row (or slice) offsets, and every vector once.
    Folded (the quarter-turn symmetry): the loop stores and streams the first
    half of A's rows and their transpose, nnz/2 entries each."""
    rows_per_offset = 8 if sliced else 1   # the sliced layout keeps one offset per 8 rows
    stored = nnz // 2 if folded else nnz
    m_rows = m // 2 if folded else m
    fwd = (per_nnz * stored + 4 * (m_rows // rows_per_offset + 1)
           + 4 * d + 28 * m               # f gathered once; g, gamma, y_prev (8 B), y (8 B), w
           + 12 * d)                      # stencil: f^k, f^{k-1} in, B^T grad phi~ out
    pix = (per_nnz * stored + 4 * (d // rows_per_offset + 1)
           + 4 * m                        # w gathered once
           + 20 * d)                      # f^k, f^{k-1}, B^T grad phi~, 1/Lambda in; f^{k+1} out
    return fwd, pix


# the sources that decide the single-slice loop's kernels and matrix layout
KERNEL_SOURCES = ("kernels.cu", "appga_internal.h", "device_common.cuh")


def kernel_sources_sha256(root: str) -> str:
    """SHA-256 of the loop kernels' sources, concatenated in KERNEL_SOURCES order."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(root, "paper_2409_13344_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def main_leg_folds(choice: str, fold_stream_bytes: int, l2_bytes: int) -> bool:
    """Whether the main single-slice leg runs the quarter-turn folded loop:
    `choice` "on" / "off" decides; "auto" folds only when the folded streams
    of an iteration still exceed L2, so the timed iterations never reuse the
    matrix from L2."""
    if choice == "on":
        return True
    if choice == "off":
        return False
    return fold_stream_bytes > l2_bytes


def committed_traffic(kernel: str, layout: str = "unfolded"):
    """DRAM bytes per launch of `kernel` in the loop's `layout` ("unfolded" or
    "folded") from the committed ncu summary, if it was taken on the current
    kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        sha = kernel_sources_sha256(ROOT)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_sources_sha256") != sha:
        return None
    ent = rec.get("layouts", {}).get(layout, {}).get("kernels", {}).get(kernel)
    return None if ent is None else ent.get("dram_bytes_per_launch")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# --------------------------------------------------------- batched and served

def batched_bytes(m: int, d: int, nnz: int, K: int):
    """Algorithmic bytes of one batched iteration (both kernels) for K slices:
    the two matrix streams once, plus every per-slice vector once."""
    mats = 8 * nnz + 4 * (m + 1) + 8 * nnz + 4 * (d + 1) + 4 * d  # A, A^T, 1/Lambda
    fwd = K * (4 * d + 4 * m * 5)          # f^k gather; y_prev, g, gamma in; y, w out
    stencil = K * (4 * d * 2 + 4 * d)      # f^k, f^{k-1} in; gR out
    pix = K * (4 * m + 4 * d * 4)          # w gather; f^k, f^{k-1}, gR in; f^{k+1} out
    return mats + fwd + stencil + pix


def bench_batched(AP, ctx, geom, A, dev, single_rate, K=BATCH_K, lo=1e5, hi=1e7,
                  omega=OMEGA, iters=BATCH_ITERS, distinct=None, config=3, label=None):
    """K independent slices sharing A (per-slice counts log-uniform lo..hi),
    FP32 and BF16 values of A, default and autotuned launch schedules:
    slices x iterations per second.  `distinct` slices are generated and
    repeated to K (sinogram generation is host-bound at large sizes)."""
    import numpy as np
    import torch
    from paper_2409_13344_gb300 import workload as W
    rng = np.random.default_rng(config)
    counts = W.log_uniform_counts(rng, lo, hi, K)
    nd = K if distinct is None else distinct
    sls = [W.make_slice(A, geom, float(counts[i]), W.seed_for(config, i), phantom="lesions")
           for i in range(nd)]
    mat = AP.Matrix(ctx, A, geom.n, geom.n_angles, bf16=True)
    g = torch.from_numpy(np.stack([sls[i % nd].g for i in range(K)])).to(dev)
    gam = torch.from_numpy(np.stack([sls[i % nd].gamma for i in range(K)])).to(dev)
    f = torch.empty((K, geom.d), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {"workload": label or (
               f"{K} independent {geom.n}x{geom.n} slices ({geom.n_angles} x {geom.n_bins} "
               f"sinograms) sharing one A, counts log-uniform {lo:g}..{hi:g}, omega {omega:g}, "
               f"beta 1, {iters} iterations per call, one call = one SpMM solver run under "
               "captured CUDA graphs"),
           "K": K, "nnz": int(mat.info().nnz)}
    nb = batched_bytes(geom.m, geom.d, int(mat.info().nnz), K)

    def measure(prec):
        def call(n_maps):
            p = AP.default_params(lambda1=LAM1, lambda2=LAM2, eps=EPS, omega=omega,
                                  max_iters=n_maps, a_precision=prec)
            AP.appga_reconstruct_batched(ctx.handle, mat.handle, K, g, gam, None, p, f)
        for _ in range(3):
            call(8)
        # per-iteration time = (t(8 + iters) - t(8)) / iters, median of three
        # repetitions (setup and the final read-back cancel in the difference)
        reps = []
        for _ in range(3):
            ms = {}
            for n_maps in (8, 8 + iters):
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call(n_maps)
                e1.record(stream)
                torch.cuda.synchronize()
                ms[n_maps] = e0.elapsed_time(e1)
            reps.append(((ms[8 + iters] - ms[8]) / iters, ms[8 + iters]))
        per_iter, ms_call = sorted(reps)[1]
        ms = {8 + iters: ms_call}
        rate = K / (per_iter * 1e-3)
        return {"slices_iters_per_s": rate, "us_per_batched_iter": 1e3 * per_iter,
                "us_per_slice_iter": 1e3 * per_iter / K,
                "call_slices_iters_per_s": K * (8 + iters) / (ms[8 + iters] * 1e-3),
                "algorithmic_gbs": nb / (per_iter * 1e-3) / 1e9,
                "vs_single_slice": rate / single_rate}

    for name, prec in (("fp32", 0), ("bf16", 1)):
        out[name] = measure(prec)
        # the library's autotuner picks the launch schedule for this width and
        # precision on these slices; the tuned schedule is then measured the same way
        t = AP.appga_autotune_batched(ctx.handle, mat.handle, K, g, gam,
                                      AP.default_params(lambda1=LAM1, lambda2=LAM2, eps=EPS,
                                                        omega=omega, a_precision=prec))
        tuned = measure(prec)
        tuned["schedule"] = {"spmv_per_sm": t.spmv_per_sm, "pixel_per_sm": t.pixel_per_sm,
                             "stencil_per_sm": t.stencil_per_sm, "chunk": t.chunk,
                             "gather_rows_fw": t.gather_rows_fw,
                             "gather_rows_px": t.gather_rows_px,
                             "trial_us_per_slice_iter": t.us_per_slice_iter,
                             "trial_us_default": t.us_per_slice_iter_default}
        out[name + "_autotuned"] = tuned
    # the second ceiling of the batched kernels: their gather loop alone
    # (L1/L2-bound), timed by the library's probe on this matrix
    sch = out["fp32_autotuned"]["schedule"]
    k_eff = sch["chunk"] if 0 < sch["chunk"] < K else K
    width = 32 if k_eff <= 32 else (64 if k_eff <= 64 else 128)
    p_fwd, p_bwd = AP.appga_gather_probe(ctx.handle, mat.handle, width, 20)
    info = mat.info()
    b_fwd = int(info.nnz_padded_a) * 4 * width  # gathered bytes per (sub-)batch projection
    b_bwd = int(info.nnz_padded_t) * 4 * width
    # the iteration's gather ceiling: both projections at their probed rates
    t_ceil = b_fwd / (p_fwd * 1e9) + b_bwd / (p_bwd * 1e9)
    t_iter = k_eff / out["fp32_autotuned"]["slices_iters_per_s"]  # per (sub-)batch iteration
    out["fp32_autotuned"]["gather_roofline"] = {
        "bound": "l1/l2 gathers", "unit": "GB/s", "width": width,
        "probe_fwd_gbs": p_fwd, "probe_bwd_gbs": p_bwd,
        "achieved_gbs": (b_fwd + b_bwd) / t_iter / 1e9,
        "peak": (b_fwd + b_bwd) / t_ceil / 1e9, "frac": t_ceil / t_iter,
        "note": "bytes = Kp-wide rows gathered by both projections per (sub-)batch iteration; "
                "peak = those bytes at the rates appga_gather_probe measures for the projectors' "
                "inner loop alone (column/value stream + gathers, no epilogue, stencil or pixel "
                "update; fastest grid size) on this matrix, so frac is the share of the "
                "iteration's time that is projector gathers"}
    out["algorithmic_bytes_per_iter"] = nb
    mat.close()
    return out


def bench_volume(AP, ctx, geom, A, dev, batched_rate, nz=64, counts=6.4e7, iters=100):
    """APPGA with the 3-D SHOITV regulariser on one volume of nz slices of
    the main geometry sharing A (ellipsoid phantom, Poisson counts per
    slice): slices x iterations per second, and the 3-D stencil kernel alone
    against the HBM roofline."""
    import numpy as np
    import torch
    from paper_2409_13344_gb300 import workload as W
    vol = W.make_volume(A, geom, nz, counts, W.seed_for(6, 4))
    mat = AP.Matrix(ctx, A, geom.n, geom.n_angles, bf16=True)
    g = torch.from_numpy(vol.g).to(dev)
    gam = torch.from_numpy(vol.gamma).to(dev)
    f = torch.empty((nz, geom.d), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {"workload": f"one volume of {nz} slices of {geom.n}x{geom.n} ({geom.n_angles} x "
                       f"{geom.n_bins} sinograms per slice) sharing one A, ellipsoid phantom, "
                       f"{counts:g} expected counts over the volume, 3-D SHOITV (3 + 9 "
                       "components per voxel), omega 0.5, beta 1, objective every iteration; "
                       "batched SpMM kernels + 3-D stencil under captured CUDA graphs",
           "nz": nz}

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for name, prec in (("fp32", 0), ("bf16", 1)):
        def call(n_maps):
            p = AP.default_params(lambda1=LAM1, lambda2=LAM2, eps=EPS, omega=OMEGA,
                                  max_iters=n_maps, a_precision=prec, track_objective=1)
            AP.appga_reconstruct_volume(ctx.handle, mat.handle, nz, g, gam, None, p, f)
        for _ in range(2):
            call(8)
        reps = sorted((timed(lambda: call(8 + iters)) - timed(lambda: call(8))) / iters
                      for _ in range(3))
        per_iter = reps[1]
        out[name] = {"slices_iters_per_s": nz / (per_iter * 1e-3),
                     "us_per_volume_iter": 1e3 * per_iter, "us_per_slice_iter": 1e3 * per_iter / nz}
        if batched_rate and name in batched_rate:
            out[name]["vs_batched_2d"] = out[name]["slices_iters_per_s"] / batched_rate[name]
    # the 3-D stencil alone: slice-major volume in, gradient out (8 bytes per voxel)
    vox = nz * geom.d
    fin = f.clone()
    gout = torch.empty_like(fin)
    run = lambda: AP.appga_shoitv3d_grad(ctx.handle, geom.n, nz, fin, LAM1, LAM2, EPS, gout)
    for _ in range(5):
        run()
    ms = timed(lambda: [run() for _ in range(50)]) / 50
    peaks, src = measured_peaks()
    hbm = peaks["hbm_gbs"]
    out["stencil3d"] = {"kernel": "k_stencil3d", "us_per_launch": 1e3 * ms,
                        "algorithmic_bytes_per_launch": 8 * vox,
                        "achieved_gbs": 8 * vox / (ms * 1e-3) / 1e9, "peak_gbs": hbm,
                        "peak_source": src, "frac": 8 * vox / (ms * 1e-3) / 1e9 / hbm}
    mat.close()
    return out


def bench_other_layout(AP, ctx, geom, A, g, gamma, params, fold, l2_bytes, fold_stream,
                       plain_stream, iters=4000):
    """The single-slice loop in the other matrix layout of the main leg
    (quarter-turn folded or not), timed as the main leg: 500-iteration
    reconstructions back to back, CUDA events on the launching stream, and
    each loop kernel timed alone.  When its streams fit in L2 the iterations
    reuse part of the matrix from L2, which the entry states."""
    import torch
    mat = AP.Matrix(ctx, A, geom.n, geom.n_angles, fold=fold)
    try:
        info = mat.info()
        if fold and not info.quarter_turn_folded:
            return {"unavailable": "the matrix has no exact quarter-turn symmetry"}
        f = torch.empty(geom.d, dtype=torch.float32, device=g.device)
        stream = torch.cuda.current_stream()
        for _ in range(2):
            AP.appga_reconstruct(ctx.handle, mat.handle, g, gamma, None, params(ITERS_PER_RECON), f)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done = 0
        while done < iters:
            it = min(ITERS_PER_RECON, iters - done)
            AP.appga_reconstruct(ctx.handle, mat.handle, g, gamma, None, params(it), f)
            done += it
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        AP.appga_kernel_times(ctx.handle, mat.handle, g, gamma, params(50), 50)
        tp, tf = AP.appga_kernel_times(ctx.handle, mat.handle, g, gamma, params(300), 300)
        stream_bytes = fold_stream if fold else plain_stream
        return {
            "layout": ("quarter-turn folded (half of A and A^T stored), " if fold else "")
                      + "sliced, packed 2-byte columns + FP32 values",
            "iters_per_s": iters / (ms * 1e-3), "us_per_iter": ms * 1e3 / iters,
            "k_pixel_us": tp * 1e3, "k_forward_us": tf * 1e3,
            "stream_bytes_per_iter": stream_bytes,
            "l2": (f"the loop streams {stream_bytes / 1e6:.0f} MB per iteration, "
                   + ("below" if stream_bytes < l2_bytes else "above")
                   + f" L2 ({l2_bytes / 1e6:.0f} MB)"
                   + ("; iterations reuse part of the matrix from L2 (measured at 256x256 "
                      "without cache flushes: 38-40 MB of DRAM reads per launch of the "
                      "47-48 MB stored), so this rate is not the main leg's"
                      if stream_bytes < l2_bytes else "")),
        }
    finally:
        mat.close()


def bench_afppa(AP, ctx, geom, A, sl, dev, appga_ms, cpu: bool, iters=200, fold=True):
    """AFPPA with GN momentum for the non-smooth HOITV model (Sec. 4.4) on the
    main slice: time per step on the GPU (projectors + dual-update kernel)
    against one APPGA iteration, the FP64 oracle's step on the host, and the
    figures of merit of the result (MSE, PSNR, RC / NRC on a lesion mask,
    central line profile) with their own call time."""
    import numpy as np
    import torch
    mat = AP.Matrix(ctx, A, geom.n, geom.n_angles, fold=fold)
    g = torch.from_numpy(sl.g).to(dev)
    gam = torch.from_numpy(sl.gamma).to(dev)
    f = torch.empty(geom.d, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def call(n):
        p = AP.default_params(lambda1=LAM1, lambda2=LAM2, omega=OMEGA, max_iters=n)
        AP.appga_afppa_reconstruct(ctx.handle, mat.handle, g, gam, None, p, f)
    for _ in range(2):
        call(8)
    per = sorted((timed(lambda: call(8 + iters)) - timed(lambda: call(8))) / iters
                 for _ in range(3))[1]
    out = {"workload": f"AFPPA (GN momentum, omega {OMEGA:g}) for the non-smooth HOITV model on "
                       f"the main {geom.n}x{geom.n} slice, lambda1/lambda2 {LAM1:g}/{LAM2:g}, "
                       f"rates over {iters} timed steps",
           "us_per_step": 1e3 * per, "steps_per_s": 1.0 / (per * 1e-3),
           "vs_appga_iteration": per / appga_ms}
    if cpu:
        from oracle import afppa_oracle as F
        from oracle import appga_oracle as O
        prob = O.Problem(A, sl.g, sl.gamma, geom.n)
        par = O.Params(lambda1=LAM1, lambda2=LAM2, omega=OMEGA, max_iters=3)
        t0 = time.perf_counter()
        F.afppa(prob, par, n_angles=geom.n_angles)
        el = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": 3 / el, "unit": "steps/s", "cores": 1,
                               "host_cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"3 FP64 oracle AFPPA steps of the same slice, {el:.1f} s"}
    # figures of merit of the AFPPA result against the phantom (Sec. 4.1)
    call(iters)
    n = geom.n
    truth = torch.from_numpy(sl.f_true.astype(np.float32)).to(dev)
    hot = sl.f_true > 1.5 * np.median(sl.f_true[sl.f_true > 0])
    body = (sl.f_true > 0) & ~hot
    roi_h = torch.from_numpy(hot.astype(np.uint8)).to(dev)
    roi_b = torch.from_numpy(body.astype(np.uint8)).to(dev)
    vmax = float(sl.f_true.max())
    for _ in range(3):
        fm = AP.appga_figures_of_merit(ctx.handle, geom.d, f, truth, roi_h, roi_b, vmax)
    t0 = time.perf_counter()
    for _ in range(20):
        fm = AP.appga_figures_of_merit(ctx.handle, geom.d, f, truth, roi_h, roi_b, vmax)
    us_fom = (time.perf_counter() - t0) / 20 * 1e6
    prof = torch.empty(n, dtype=torch.float32, device=dev)
    AP.appga_central_line_profile(ctx.handle, n, f, prof)
    torch.cuda.synchronize()
    out["figures_of_merit"] = {"mse": fm.mse, "psnr_db": fm.psnr, "nrc": fm.nrc,
                               "roi_hot_pixels": int(fm.n_roi_h),
                               "us_per_call": us_fom,
                               "note": "one call = MSE, PSNR, RC and NRC reductions in double-float "
                                       "plus the host read-back (latency-bound at this size)"}
    mat.close()
    return out


def bench_serving(AP, ctx, n_requests: int, rate: float, main_geom, main_A,
                  slots: int = SERVE_SLOTS, steps: int = SERVE_STEPS, max_pools: int = 0,
                  geom_pools: int = 2):
    """Poisson stream of reconstruction requests mixing 128^2, 256^2 and 400^2
    slices (200..800 iterations each, or the relative objective change
    < 1e-7) through the continuous-batching server."""
    import numpy as np
    from paper_2409_13344_gb300 import workload as W
    rng = np.random.default_rng(4)
    mats, slices = {}, {}
    for idx, nm in enumerate(SERVE_GEOMS):
        geom = W.GEOMETRIES[nm]
        A = main_A if nm == GEOM else W.system_matrix(nm)
        mats[nm] = AP.Matrix(ctx, A, geom.n, geom.n_angles)
        counts = W.log_uniform_counts(rng, 1e5, 1e7, 6)
        slices[nm] = [W.make_slice(A, geom, float(c), W.seed_for(4, 100 * idx + i),
                                   phantom="lesions") for i, c in enumerate(counts)]
    srv = AP.Server(ctx, slots_per_pool=slots, steps_per_launch=steps, max_pools=max_pools,
                    max_pools_per_geometry=geom_pools)
    gids = {nm: srv.add_geometry(mats[nm]) for nm in SERVE_GEOMS}
    # warm-up: one short request per geometry (pools and graphs are created here)
    for nm in SERVE_GEOMS:
        x = slices[nm][0]
        srv.submit(gids[nm], x.g, x.gamma, AP.default_params(max_iters=16))
    while srv.step():
        pass
    for rid in list(srv._geom_of):
        srv.collect(rid)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    kinds = rng.integers(0, len(SERVE_GEOMS), n_requests)
    iters = rng.integers(200, 801, n_requests)
    omegas = rng.choice([0.5, 1.0], n_requests)
    info, lat, per_geom = {}, [], {nm: [] for nm in SERVE_GEOMS}
    finished = []  # (completion time, iterations) of every request
    done_iters, stopped = 0, 0
    nxt, rounds = 0, 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while nxt < n_requests and arrivals[nxt] <= now:
            nm = SERVE_GEOMS[kinds[nxt]]
            x = slices[nm][nxt % len(slices[nm])]
            p = AP.default_params(lambda1=LAM1, lambda2=LAM2, eps=EPS, omega=float(omegas[nxt]),
                                  max_iters=int(iters[nxt]), rel_obj_tol=1e-7)
            info[srv.submit(gids[nm], x.g, x.gamma, p)] = (arrivals[nxt], nm)
            nxt += 1
        pending = srv.step()
        rounds += 1
        t_seen = time.perf_counter() - t0
        for rid in list(info):
            if srv.poll(rid).state == AP.APPGA_REQ_DONE:
                a, nm = info.pop(rid)
                _, st = srv.collect(rid)
                lat.append(t_seen - a)  # from the request's arrival
                per_geom[nm].append(t_seen - a)
                finished.append((t_seen, st.iters))
                done_iters += st.iters
                stopped += st.stopped_early
        if nxt >= n_requests and pending == 0:
            break
        if pending == 0:
            time.sleep(max(0.0, min(arrivals[nxt] - (time.perf_counter() - t0), 0.01)))
    elapsed = time.perf_counter() - t0
    summ = srv.summary()
    srv.close()
    for m in mats.values():
        m.close()
    lat = np.asarray(lat)
    # steady state: iterations of the requests completed between the arrival
    # of the first fifth of the stream and the last arrival (the queue is
    # still being fed there; the drain after the last arrival is left out)
    w0, w1 = float(arrivals[n_requests // 5]), float(arrivals[-1])
    in_win = sum(n for t, n in finished if w0 <= t <= w1)
    steady = in_win / (w1 - w0) if w1 > w0 else float("nan")
    return {
        "workload": f"Poisson stream of {n_requests} requests at {rate:g}/s mixing 128^2 (90x185), "
                    "256^2 (180x367) and 400^2 (288x575) slices, 200..800 iterations each or "
                    "relative objective change < 1e-7, omega 0.5/1.0, counts log-uniform 1e5..1e7",
        "requests": n_requests, "rate_per_s": rate, "elapsed_s": elapsed,
        "scheduling_rounds": rounds,
        "slices_iters_per_s": done_iters / elapsed, "slice_iters": done_iters,
        "steady_slices_iters_per_s": steady,
        "steady_window_s": [w0, w1],
        "stopped_early": stopped,
        "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
        "mean_latency_s": float(lat.mean()),
        "per_geometry": {nm: {"n": len(v), "p50_s": float(np.percentile(v, 50)),
                              "p99_s": float(np.percentile(v, 99))} for nm, v in per_geom.items() if v},
        "server_p50_latency_s": summ.p50_latency_s, "server_p99_latency_s": summ.p99_latency_s,
        "latency_from": "arrival time of the request in the stream (the server's own figures "
                        "count from submission)",
        "pools": summ.pools, "device_bytes": summ.device_bytes, "slots_per_pool": slots,
        "max_pools_per_geometry": geom_pools,
        "slot_occupancy": summ.live_slot_steps / max(summ.pool_slot_steps, 1),
        "replay_seconds_over_elapsed": summ.replay_seconds / elapsed,
        "steps_per_launch": steps,
    }


# ----------------------------------------------------------------- oracle

def oracle_rate(geom, A, sl, seconds: float, min_iters: int = 3):
    """Plain FP64 oracle on the same slice, timed on the host (one core)."""
    from oracle import appga_oracle as O
    prob = O.Problem(A, sl.g, sl.gamma, geom.n)
    par = O.Params(lambda1=LAM1, lambda2=LAM2, eps=EPS, omega=OMEGA)
    lam = prob.em_lambda()
    f = O.initial_image(sl.g, sl.gamma, geom.n, geom.n_angles)
    fm = f.copy()
    t0 = time.perf_counter()
    k = 0
    while True:
        k += 1
        th = O.gn_theta(k, par.a, par.b, par.omega)
        fn, _ = O.appga_step(prob, f, fm, th, par, lam)
        prob.objective(fn, LAM1, LAM2, EPS)  # the objective is part of every step
        fm, f = f, fn
        el = time.perf_counter() - t0
        if k >= min_iters and el >= seconds:
            break
    return k, el


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    geom, A, sl = make_inputs(0)
    from oracle import appga_oracle as O
    prob = O.Problem(A, sl.g, sl.gamma, geom.n)
    par = O.Params(lambda1=LAM1, lambda2=LAM2, eps=EPS, omega=OMEGA)
    lam = prob.em_lambda()
    f = O.initial_image(sl.g, sl.gamma, geom.n, geom.n_angles)
    fm = f.copy()

    def step(k):
        nonlocal f, fm
        th = O.gn_theta(k, par.a, par.b, par.omega)
        fn, _ = O.appga_step(prob, f, fm, th, par, lam)
        prob.objective(fn, LAM1, LAM2, EPS)
        fm, f = f, fn

    # One oracle iteration takes tens of milliseconds on one host core, so the
    # run is bounded in wall time: at most 3 warm-up steps, then steps until
    # --steps are done or --ref-seconds have passed (at least one).
    k = 0
    warm = min(args.warmup, 3)
    for _ in range(warm):
        k += 1
        step(k)
    t0 = time.perf_counter()
    done, el = 0, 0.0
    while done < max(args.steps, 1):
        k += 1
        step(k)
        done += 1
        el = time.perf_counter() - t0
        if el >= args.ref_seconds:
            break
    val = done / el
    sample = (f"{done} FP64 oracle APPGA iterations of the 256x256 slice (of {args.steps} "
              f"requested; bounded to {args.ref_seconds:g} s) after {warm} warm-up")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": done, "requested_steps": args.steps, "warmup": warm,
        "ms_per_step": 1e3 * el / done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference": "FP64 NumPy/SciPy oracle on the host"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


# ------------------------------------------------------------------- ours

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2409_13344_gb300 import build, replicas
    from paper_2409_13344_gb300 import appga as AP

    rank, world, local = replicas.dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    geom, A, sl = make_inputs(rank)
    ctx = AP.Context(dev.index)
    if args.volume_only:
        print(json.dumps({"volume": bench_volume(AP, ctx, geom, A, dev, None)}), flush=True)
        ctx.close()
        return 0
    if args.serve_only:
        print(json.dumps({"serving": bench_serving(AP, ctx, args.serve_requests, args.serve_rate,
                                                   geom, A, args.serve_slots,
                                                   args.serve_steps,
                                                   args.serve_max_pools,
                                                   args.serve_geom_pools)}), flush=True)
        ctx.close()
        return 0
    # the main leg's layout: its per-iteration streams must exceed L2, so the
    # timed iterations do not reuse the matrix from L2
    l2_bytes = int(torch.cuda.get_device_properties(dev).L2_cache_size)
    nnz = int(A.nnz)
    fold_stream = sum(kernel_bytes(geom.m, geom.d, nnz, 6, True, True))
    plain_stream = sum(kernel_bytes(geom.m, geom.d, nnz, 6, True, False))
    fold = main_leg_folds(args.fold, fold_stream, l2_bytes)
    mat = AP.Matrix(ctx, A, geom.n, geom.n_angles, fold=fold)
    g = torch.from_numpy(sl.g).to(dev)
    gamma = torch.from_numpy(sl.gamma).to(dev)
    f_out = torch.empty(geom.d, dtype=torch.float32, device=dev)

    param_cache = {}

    def params(iters):
        # one parameter block per length, built once (as a caller would)
        if iters not in param_cache:
            param_cache[iters] = AP.default_params(lambda1=LAM1, lambda2=LAM2, eps=EPS,
                                                   omega=OMEGA, max_iters=iters,
                                                   track_objective=1)
        return param_cache[iters]

    def chunks(total):
        out = []
        while total > 0:
            out.append(min(ITERS_PER_RECON, total))
            total -= out[-1]
        return out

    def run_device(total):
        for it in chunks(total):
            AP.appga_reconstruct(ctx.handle, mat.handle, g, gamma, None, params(it), f_out)

    def launches(total):
        # per run: the start-state/momentum kernel, the initial image (two
        # kernels, with the input check), the first forward phase, then per
        # iteration the pixel kernel (which also finalises the previous step)
        # and the forward kernel (exactly `it` maps), the last finalisation
        # (objective of the result) and the result copy
        n = 0
        for it in chunks(total):
            n += 6 + 2 * it
        return n

    def barrier():
        if world > 1:
            dist.barrier()

    # the graphs and buffers of these calls exist after a first call
    run_device(3)
    torch.cuda.synchronize()
    clocks = ClockSampler()
    stream = torch.cuda.current_stream()
    clocks.start()
    time.sleep(0.3)
    # warm-up right before the timed steps (the clock sampler is already on)
    run_device(max(args.warmup, 3))
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run_device(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max = replicas.max_over_ranks(ms, device=dev)
    total_steps = replicas.sum_over_ranks(args.steps, device=dev)
    value = total_steps / (ms_max / 1e3)

    # end to end through the host-buffer entry point (pinned host memory)
    g_h = torch.from_numpy(sl.g).pin_memory()
    gam_h = torch.from_numpy(sl.gamma).pin_memory()
    f_h = torch.empty(geom.d, dtype=torch.float32).pin_memory()
    e_steps = min(args.steps, 20 * ITERS_PER_RECON)
    for it in chunks(min(e_steps, ITERS_PER_RECON)):
        AP.appga_reconstruct_host(ctx.handle, mat.handle, g_h, gam_h, None, params(it), f_h)
    barrier()
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    n_calls = 0
    for it in chunks(e_steps):
        AP.appga_reconstruct_host(ctx.handle, mat.handle, g_h, gam_h, None, params(it), f_h)
        n_calls += 1
    e3.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = replicas.max_over_ranks(e2.elapsed_time(e3), device=dev)
    e2e_value = replicas.sum_over_ranks(e_steps, device=dev) / (ms_e2e / 1e3)

    # per-kernel device times for the roofline (CUDA events on the launch stream)
    AP.appga_kernel_times(ctx.handle, mat.handle, g, gamma, params(50), 50)  # warm-up
    tp, tf = AP.appga_kernel_times(ctx.handle, mat.handle, g, gamma, params(300), 300)
    info = mat.info()
    per_nnz = 6 if info.packed_columns else 8
    folded = bool(info.quarter_turn_folded)
    # algorithmic bytes: the method's work with A and A^T each read once as
    # FP32 values + int32 columns, and every vector once
    c_fwd, c_pix = kernel_bytes(geom.m, geom.d, int(info.nnz))
    # what the loop's layout streams: the folded half (when folded) at
    # per_nnz bytes per stored nonzero
    b_fwd, b_pix = kernel_bytes(geom.m, geom.d, int(info.nnz), per_nnz, bool(info.sliced_layout),
                                folded)
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    dom = ("k_pixel", tp, c_pix, b_pix) if tp >= tf else ("k_forward", tf, c_fwd, b_fwd)
    other = (("k_forward", tf, c_fwd, b_fwd) if dom[0] == "k_pixel"
             else ("k_pixel", tp, c_pix, b_pix))
    achieved = dom[2] / (dom[1] * 1e-3) / 1e9
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
        "traffic": committed_traffic(dom[0], "folded" if folded else "unfolded"),
        "kernel": dom[0], "peak_source": peak_src,
        # each launch timed alone (the step finalisation runs inside k_pixel)
        "timed_as": dom[0],
        "ms_per_launch": dom[1], "algorithmic_bytes_per_launch": dom[2],
        "algorithmic_bytes": "A (or A^T) once as FP32 values + int32 columns (8 B per nonzero), "
                             "its row offsets, and every vector once",
        # the bytes the loop's layout actually streams, and the rate at which
        # it streams them
        "stored_stream": {
            "layout": ("quarter-turn folded (half of A and A^T stored), " if folded else "")
                      + ("sliced, packed 2-byte columns + FP32 values" if info.packed_columns
                         else ("sliced, 4-byte columns" if info.sliced_layout else "CSR")),
            "bytes_per_nnz": per_nnz, "bytes_per_launch": dom[3],
            "achieved_gbs": dom[3] / (dom[1] * 1e-3) / 1e9,
            "frac": dom[3] / (dom[1] * 1e-3) / 1e9 / hbm},
        "other_kernel": {"kernel": other[0], "ms_per_launch": other[1],
                         "algorithmic_bytes_per_launch": other[2],
                         "achieved_gbs": other[2] / (other[1] * 1e-3) / 1e9,
                         "frac": other[2] / (other[1] * 1e-3) / 1e9 / hbm},
        # a whole loop iteration (both launches back to back, as timed by the
        # step rate above)
        "iteration": {"algorithmic_bytes": c_fwd + c_pix,
                      "achieved_gbs": (c_fwd + c_pix) * args.steps / (ms * 1e-3) / 1e9,
                      "frac": (c_fwd + c_pix) * args.steps / (ms * 1e-3) / 1e9 / hbm},
    }

    # the loop in the other layout (folded when the main leg is not, and the
    # reverse), timed the same way
    other_layout = None
    if world == 1 and not args.no_other_layout:
        other_layout = bench_other_layout(AP, ctx, geom, A, g, gamma, params, not fold,
                                          l2_bytes, fold_stream, plain_stream)
    batched = serving = None
    large = None
    if world == 1 and not args.no_batched:
        batched = bench_batched(AP, ctx, geom, A, dev, value)
    if world == 1 and not args.no_large:
        # 120 slices of 512x512 (360 x 731), dynamic-frame counts 1e4..1e7, omega 1, 300 iterations
        from paper_2409_13344_gb300 import workload as W
        g5 = W.GEOMETRIES["512"]
        large = bench_batched(AP, ctx, g5, W.system_matrix("512"), dev, value, K=120, lo=1e4,
                              hi=1e7, omega=1.0, iters=60, distinct=8, config=5,
                              label="120 independent 512x512 slices (360 x 731 sinograms, "
                                    "Siddon A 120.2M nnz) sharing one A, dynamic-frame counts "
                                    "log-uniform 1e4..1e7 (8 distinct sinograms repeated), "
                                    "omega 1, beta 1; rates over 60 timed iterations of a "
                                    "300-iteration schedule")
    afppa = None
    if world == 1 and not args.no_afppa:
        afppa = bench_afppa(AP, ctx, geom, A, sl, dev, ms_max / args.steps,
                            cpu=rank == 0 and not args.no_cpu_baseline, fold=fold)
    volume = None
    if world == 1 and not args.no_volume:
        brate = None
        if batched:  # the volume runs the batched kernels' default schedule
            brate = {k: batched[k]["slices_iters_per_s"] for k in ("fp32", "bf16")}
        volume = bench_volume(AP, ctx, geom, A, dev, brate)
    serving_sat = None
    if world == 1 and not args.no_serve:
        serving = bench_serving(AP, ctx, args.serve_requests, args.serve_rate, geom, A,
                                args.serve_slots, args.serve_steps)
        # an arrival rate above what the server completes: its saturated throughput
        serving_sat = bench_serving(AP, ctx, SAT_REQUESTS, SAT_RATE, geom, A, args.serve_slots,
                                    args.serve_steps)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        k, el = oracle_rate(geom, A, sl, args.cpu_seconds)
        cpu = {"value": k / el, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"{k} FP64 oracle APPGA iterations (with the objective) of the same "
                         f"256x256 slice from the initial image, {el:.1f} s on one host core"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "geometry": "256x256, 180 x 367",
                       "nnz": int(info.nnz),
                       "l2": "inputs larger than L2: the loop streams "
                             + ("the folded halves of A and A^T, " if folded
                                else "A and A^T, ")
                             + f"{(fold_stream if folded else plain_stream) / 1e6:.0f} MB per "
                             f"iteration (L2 {l2_bytes / 1e6:.0f} MB)",
                       "layout": roofline["stored_stream"]["layout"],
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * geom.m * n_calls / e_steps,
                    "d2h_bytes_per_step": 4 * geom.d * n_calls / e_steps},
            "gpu_launches": launches(args.steps),
            "clocks": clk,
            "batched": batched,
            "large_batch": large,
            "volume": volume,
            "afppa": afppa,
            "other_layout": other_layout,
            "serving": serving,
            "serving_saturated": serving_sat,
        }
        print(json.dumps(line), flush=True)
    mat.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
