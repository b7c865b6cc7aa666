#!/usr/bin/env python3
"""Benchmark of the fused Gaussian-polynomial bilateral filter on one GB300.

Headline workload (one step): 96 distinct 2048 x 2048 float32 images of
64-pixel blocks with uniform levels in [0,255] plus N(0, 10^2) noise (seeded,
synthetic: 8 seeded images in 12 row rotations each, 7.7 GB of images,
cotangents and outputs, far larger than L2), Gaussian spatial kernel
sigma_s = 3 (W = 9), sigma_r = 30, N = 40 (the order from the accuracy bound
for delta = 1, eq. eps + eq. LambW, chosen once on the host before the timed
region).  Each image of a step goes through the fused forward (out and Q') and
the fused backward (image gradient and sigma_r gradient).  The headline value
is forward+backward Mpixel/s over the whole step; forward-only Mpixel/s, the
direct eq. BF filter (forward and forward+backward) on the same image, the
end-to-end rate through the Python API with host buffers, the achieved HBM
GB/s and the FP32-pipe roofline of the dominant kernel are reported beside it.

The other workloads are timed after the headline region, each on its own:
the fast path at equal stated max error against the direct filter, the
8192^2 Gaussian W = 60 forward, 32 x 512^2 forward + backward (power images
recomputed or stored), the uneven 256-image batch as one CUDA graph (built-in
and autotuned variants), and the small-N box forward at 4096^2 against the
HBM roofline.  The CPU-baseline leg times the FP64 checker on the host cores
and measures every kept GPU output against it at sampled pixels.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank filters its own images (weak scaling, no
data-path collective); the barrier and the max over ranks of the timed
region are the only collectives.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpixel/s fwd & fwd+bwd vs direct GPU BF at stated max error; HBM GB/s"
UNIT = "Mpixel/s"
WORKLOAD = ("96 x 2048x2048 blocks(64)+N(0,10^2) images per step; Gaussian spatial sigma_s=3 "
            "(W=9), sigma_r=30, N=40 (bound for delta=1); per image fused forward + fused "
            "backward (image and sigma_r gradients)")


def workload(S, kind, R, ss, sr, N, only, B=96):
    """The workload text of a run (the default run's is WORKLOAD)."""
    spatial = ("Gaussian spatial sigma_s=%g (W=%d)" % (ss, R) if kind == 1
               else "box spatial W=%d" % R)
    step = {"all": "fused forward + fused backward (image and sigma_r gradients)",
            "fwd": "fused forward", "bwd": "fused backward (image and sigma_r gradients)"}[only]
    return "%d x %dx%d blocks(64)+N(0,10^2) images per step; %s, sigma_r=%g, N=%d; per image %s" % (
        B, S, S, spatial, sr, N, step)


L2_NOTE = ("inputs larger than L2 (each step filters 96 distinct 2048^2 images); L2 also "
           "flushed between steps (512 MB write, outside the step's events)")
FIXED_RADII = (3, 5, 9, 15)  # radii with compile-time-specialised kernels


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=96, help="distinct images per step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=2048, help="image side (profiling runs only)")
    ap.add_argument("--kind", default="gauss", choices=["gauss", "box"])
    ap.add_argument("--radius", type=int, default=9)
    ap.add_argument("--sigma-s", type=float, default=3.0)
    ap.add_argument("--sigma-r", type=float, default=30.0)
    ap.add_argument("--order", type=int, default=0, help="N (0 = from delta = 1)")
    ap.add_argument("--only", default="all", choices=["all", "fwd", "bwd"],
                    help="restrict the timed step (profiling runs only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-direct", action="store_true")
    ap.add_argument("--no-hbm-study", action="store_true",
                    help="skip the small-N 4096^2 HBM measurements of the JSON line")
    ap.add_argument("--no-studies", action="store_true",
                    help="skip the other workloads (equal error, 8192^2, 32 x 512^2, batch)")
    ap.add_argument("--sweep", default="",
                    help="comma list of extra studies, one JSON line per point: "
                         "grid2048, roofline4096, large8192, recursive, batch256, grad512, "
                         "joint2048, tightness, volume (or 'all')")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_ops(sm_count: int, mhz: float) -> float:
    """FP32 pipe peak in lane-ops/s: SMs x 128 FP32 lanes x clock (one FMA = one op)."""
    return sm_count * 128.0 * mhz * 1e6


def fwd_ops_per_pixel(kind: int, R: int, N: int) -> float:
    """Algorithmic FP32 lane-ops per output pixel of the fused forward:
    per channel (N+1 of them) 2 (advance a_n) + filter + 3 (recombine), the
    filter being 2(2R+1) FMAs for the separable Gaussian and 4 adds for the
    box running sums; plus ~12 per pixel (centre, exp, ratio)."""
    filt = 2 * (2 * R + 1) if kind == 1 else 4
    return (N + 1) * (2 + filt + 3) + 12


def rec_ops_per_pixel(N: int) -> float:
    """The recursive-Gaussian forward: per channel, rows carry 10 (the
    zero-state tile finals of both directions as dot products, advance a_n),
    rows apply 35 (both recursions with their outputs, the column tiles'
    finals, advance a_n), columns apply 32 (both recursions, recombination,
    advance a_n), the two tile scans ~2; plus ~20 per pixel."""
    return (N + 1) * 79 + 20


def rec_bytes_per_pixel(N: int) -> float:
    """DRAM bytes per pixel the recursive forward's decomposition moves: per
    channel the row pass's plane (4 written, 4 read by the column pass) and the
    32-pixel tile carries (1 B/px per channel, written, scanned in place, read:
    4 per direction); per pixel f read by three kernels (12) and out written (4)."""
    return (N + 1) * 16 + 16


def bwd_ops_per_pixel(kind: int, R: int, N: int) -> float:
    """Backward: per channel 2 (advance) + 3 (adjoint seed) + two filters +
    8 (gather); plus ~20 per pixel."""
    filt = 2 * (2 * R + 1) if kind == 1 else 4
    return (N + 1) * (2 + 3 + 2 * filt + 8) + 20


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


# ----------------------------------------------------------------- CPU leg
def cpu_baseline(img, kind, R, ss, sr, N, target_s=12.0, gpu_out=None):
    """Time the FP64 checker (Algorithm 2 at sampled pixels + exact gradient
    on a crop) on the host cores; report Mpixel/s of fwd+bwd work.  When
    gpu_out is given, also return the GPU output's max error at the samples."""
    import numpy as np

    import oracle
    w = oracle.spatial_kernel(kind, R, ss)
    H, W = img.shape
    rng = np.random.default_rng(11)
    # forward: Algorithm 2 at sampled pixels; size the sample to ~target/2 seconds
    n = 64
    while True:
        ys = rng.integers(0, H, n)
        xs = rng.integers(0, W, n)
        t0 = time.perf_counter()
        ref = oracle.gpa_alg2_at(img, w, sr, N, (ys, xs))
        dt_f = time.perf_counter() - t0
        if dt_f > 0.25 * target_s or n >= 1 << 20:
            break
        n = int(n * min(8.0, max(2.0, 0.3 * target_s / max(dt_f, 1e-3))))
    fwd_px_s = n / dt_f
    err = None
    if gpu_out is not None:
        err = float(np.abs(gpu_out[ys, xs].astype(np.float64) - ref).max())
    # backward: the exact gradient on a square crop sized to ~target/2 seconds
    side = 32
    while True:
        crop = img[:side, :side]
        g = np.ones_like(crop, dtype=np.float64)
        t0 = time.perf_counter()
        oracle.gpa_grad(crop, w, sr, N, g)
        dt_b = time.perf_counter() - t0
        if dt_b > 0.25 * target_s or side >= min(H, W):
            break
        side = min(min(H, W), int(side * min(3.0, max(1.4, math.sqrt(0.3 * target_s / max(dt_b, 1e-3))))))
    bwd_px_s = side * side / dt_b
    fb = 1.0 / (1.0 / fwd_px_s + 1.0 / bwd_px_s) / 1e6
    sample = ("Algorithm 2 at %d sampled pixels (%.1f s) + exact gradient on a %dx%d crop "
              "(%.1f s), FP64, OpenMP" % (n, dt_f, side, side, dt_b))
    # the same two samples, scaled down to about half the time, on one core
    cores = cpu_cores()
    n1 = max(64, n // max(2 * cores, 1))
    side1 = max(16, int(side / math.sqrt(max(2 * cores, 1))))
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.gpa_alg2_at(img, w, sr, N, (ys[:n1], xs[:n1]))
        dt_f1 = time.perf_counter() - t0
        crop = img[:side1, :side1]
        t0 = time.perf_counter()
        oracle.gpa_grad(crop, w, sr, N, np.ones_like(crop, dtype=np.float64))
        dt_b1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    one = 1.0 / (dt_f1 / n1 + dt_b1 / (side1 * side1)) / 1e6
    return {"value": fb, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "fwd_mpx_s": fwd_px_s / 1e6, "bwd_mpx_s": bwd_px_s / 1e6,
            "one_core": {"value": one, "unit": UNIT,
                         "sample": "Algorithm 2 at %d sampled pixels + exact gradient on a %dx%d "
                                   "crop, FP64, 1 thread" % (n1, side1, side1)}}, err


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_1603_08109_gb300 import synth
    kind = 1 if args.kind == "gauss" else 0
    R, ss, sr = args.radius, args.sigma_s, args.sigma_r
    from oracle import order
    N = args.order or order.order_from_delta(kind, R, ss, sr, 1.0)
    img = synth.blocks_image(args.size, args.size, 64, 10.0, seed=1000)
    w = oracle.spatial_kernel(kind, R, ss)
    # bounded sample per step: Algorithm 2 at 2048 pixels + exact gradient on a 48x48 crop
    rng = np.random.default_rng(0)
    crop = img[:48, :48]
    g = np.ones_like(crop, dtype=np.float64)

    def step():
        ys = rng.integers(0, args.size, 2048)
        xs = rng.integers(0, args.size, 2048)
        t0 = time.perf_counter()
        oracle.gpa_alg2_at(img, w, sr, N, (ys, xs))
        t1 = time.perf_counter()
        oracle.gpa_grad(crop, w, sr, N, g)
        t2 = time.perf_counter()
        return t1 - t0, t2 - t1

    for _ in range(args.warmup):
        step()
    tf = tb = 0.0
    for _ in range(args.steps):
        a, b = step()
        tf += a
        tb += b
    fwd = 2048 * args.steps / tf
    bwd = 48 * 48 * args.steps / tb
    value = 1.0 / (1.0 / fwd + 1.0 / bwd) / 1e6
    sample = ("per step: Algorithm 2 at 2048 sampled pixels + exact gradient on a 48x48 crop "
              "of the workload image, FP64 checker, OpenMP")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * (tf + tb) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- workload studies
# Each study times one workload on the GPU (CUDA events on the launching
# stream, L2 flushed between repetitions) and returns its JSON fields; the
# host copies of sampled outputs go to `keep`, from which the CPU-baseline leg
# computes the errors against the checker.
def _samples(rng, H, W, n):
    ys = rng.integers(0, H, n)
    xs = rng.integers(0, W, n)
    return ys, xs


def study_equal_error(bf, x_np, x, g, kind, R, ss, sr, N, dev, stream, flush, keep):
    """Fast forward + backward at equal stated max error against the direct
    filter: the order N_eq from the accuracy bound for delta = 1e-3 (Prop.
    accuracy: |f_GPA - f_BF| <= delta), the parity tolerance of the float32
    outputs, so both filters are stated accurate to 1e-3 of eq. BF; the
    CPU-baseline leg measures both errors against FP64 eq. BF at the same
    sampled pixels."""
    import numpy as np
    import torch
    N_eq = bf.order_from_delta(kind, R, ss, sr, 1e-3)
    o, q = bf.gpa_forward(x, kind, sr, N_eq, radius=R, sigma_s=ss, return_q=True)

    def fb():
        oo, qq = bf.gpa_forward(x, kind, sr, N_eq, radius=R, sigma_s=ss, return_q=True, out=o)
        bf.gpa_backward(x, oo, qq, g, kind, sr, N_eq, radius=R, sigma_s=ss)
    fbms = _time_ms(fb, 5, stream, flush)
    fms = _time_ms(lambda: bf.gpa_forward(x, kind, sr, N_eq, radius=R, sigma_s=ss, out=o), 5,
                   stream, flush)
    S = x.shape[0]
    ys, xs = _samples(np.random.default_rng(21), S, x.shape[1], 3000)
    keep["equal_error"] = {"img": x_np, "ys": ys, "xs": xs, "kind": kind, "R": R, "ss": ss,
                           "sr": sr, "N_eq": N_eq, "fast_eq": _at(o, ys, xs)}
    px = float(x.numel())
    return {"workload": "the headline image and filter; fast path at N_eq from the bound for "
                        "delta = 1e-3 (the float32 parity tolerance) against the direct filter",
            "delta": 1e-3, "N_eq": N_eq, "fast_fwd_ms": fms, "fast_fwd_bwd_ms": fbms,
            "fast_fwd_bwd_mpx_s": px / fbms / 1e3}


def study_large8192(bf, synth, dev, stream, flush, fp32, keep, with_direct=True):
    """8192^2 gradient + 64 polygons + N(0, 15^2); Gaussian sigma_s = 20
    (W = 60), sigma_r = 40, N from the bound for delta = 0.5: the two-pass
    banded forward, its FP32-pipe fraction, and the direct filter."""
    import numpy as np
    import torch
    S, R, ss, sr = 8192, 60, 20.0, 40.0
    img = synth.gradient_polygons_image(S, S, 64, 15.0, seed=2001)
    x = torch.from_numpy(img).to(dev)
    o = torch.empty_like(x)
    N = bf.order_from_delta(bf.GAUSS, R, ss, sr, 0.5)
    fms = _time_ms(lambda: bf.gpa_forward(x, bf.GAUSS, sr, N, radius=R, sigma_s=ss, out=o), 3,
                   stream, flush)
    px = float(S * S)
    ops = fwd_ops_per_pixel(1, R, N) * px
    ys, xs = _samples(np.random.default_rng(22), S, S, 200)
    res = {"workload": "8192x8192 gradient+64 polygons+N(0,15^2); Gaussian sigma_s=20 (W=60), "
                       "sigma_r=40, N=%d (bound for delta=0.5); two-pass banded forward" % N,
           "N": N, "fwd_ms": fms, "fwd_mpx_s": px / fms / 1e3,
           "fwd_alu": {"bound": "alu", "kernel": "band_vpass+band_hpass",
                       "achieved": ops / (fms * 1e-3) / 1e12, "peak": fp32 / 1e12,
                       "unit": "TFLOP/s", "frac": ops / (fms * 1e-3) / fp32}}
    keep["large_8192"] = {"img": img, "ys": ys, "xs": xs, "N": N, "R": R, "ss": ss, "sr": sr,
                          "fast": _at(o, ys, xs)}
    if with_direct:
        d = torch.empty_like(x)
        dms = _time_ms(lambda: bf.direct(x, bf.GAUSS, sr, radius=R, sigma_s=ss, out=d), 1, stream,
                       flush)
        res.update({"direct_fwd_ms": dms, "direct_fwd_mpx_s": px / dms / 1e3,
                    "speedup_vs_direct": dms / fms,
                    "max_abs_fast_vs_direct": float((o.double() - d.double()).abs().max())})
        keep["large_8192"]["direct"] = _at(d, ys, xs)
        del d
    del x, o
    torch.cuda.empty_cache()
    return res


def _at(t, ys, xs):
    """Values of a device image at sampled pixels, on the host."""
    import torch
    iy = torch.as_tensor(ys, device=t.device, dtype=torch.long)
    ix = torch.as_tensor(xs, device=t.device, dtype=torch.long)
    return t[iy, ix].double().cpu().numpy()


def _tune_buckets(bf, specs, dev, reps=3):
    """Autotune every (kind, radius bucket, order bucket) the specs occupy:
    each bucket is timed on a synthetic image of the size and parameters of
    its costliest member (the image that dominates the bucket's time); returns
    the number of buckets and the seconds spent."""
    import torch

    from paper_1603_08109_gb300 import synth
    rep = {}
    for sp in specs:
        key = (sp["kind"], bf.radius_bucket(sp["radius"]), bf.order_bucket(sp["N"]))
        cost = (sp["N"] + 1) * (2 * sp["radius"] + 1) * sp["height"] * sp["width"]
        if key not in rep or cost > rep[key][0]:
            rep[key] = (cost, sp)
    t0 = time.perf_counter()
    for _, sp in rep.values():
        img = torch.from_numpy(synth.blocks_image(sp["height"], sp["width"], 16, 20.0,
                                                  seed=sp["seed"] + 7919)).to(dev)
        bf.autotune(img, sp["kind"], sp["sigma_r"], sp["N"], radius=sp["radius"],
                    sigma_s=sp["sigma_s"], reps=reps)
    torch.cuda.synchronize(dev)
    return len(rep), time.perf_counter() - t0


def study_batch256(bf, synth, dev, stream, flush, keep, tune=True):
    """256 images, sizes U{64..768} x U{64..1024}, blocks(16)+N(0,20^2), per
    image kind, sigma_s in [2, 15] (W = ceil(3 sigma_s)), sigma_r in [10, 80],
    N from the bound for delta = 1: one captured graph of the batch plan, with
    the built-in variant choice and after autotuning the buckets present."""
    import collections

    import numpy as np
    import torch

    from paper_1603_08109_gb300 import tuning
    specs = synth.batch_specs(256, seed=3000)
    for sp in specs:
        sp["N"] = bf.order_from_delta(sp["kind"], sp["radius"], sp["sigma_s"], sp["sigma_r"], 1.0)
    host = [synth.blocks_image(sp["height"], sp["width"], 16, 20.0, seed=sp["seed"]) for sp in specs]
    imgs = [torch.from_numpy(a).to(dev) for a in host]
    outs = [torch.empty_like(t) for t in imgs]
    px = float(sum(sp["height"] * sp["width"] for sp in specs))
    saved = {(k, rb, ob): bf.tuning_get(k, rb, ob)
             for k in (bf.BOX, bf.GAUSS) for rb in range(8) for ob in range(6)}

    def measure():
        plan = bf.BatchPlan(imgs, outs, specs)
        items, ctas = plan.info()
        var = plan.variants()
        ms = _time_ms(plan.replay, 5, stream, flush)
        plan.close()
        return ms, items, var

    try:
        for key in saved:
            bf.tuning_set(*key, -1)
        ums, items, uvar = measure()
        res = {"workload": "256 images 64..768 x 64..1024 blocks(16)+N(0,20^2); per image box or "
                           "Gaussian, sigma_s in [2,15], sigma_r in [10,80], N from delta=1; one "
                           "CUDA graph of the batch plan",
               "images": 256, "megapixels": px / 1e6,
               "N_range": [min(s["N"] for s in specs), max(s["N"] for s in specs)],
               "untuned": {"graph_ms": ums, "mpx_s": px / ums / 1e3, "work_items": items,
                           "variants": dict(collections.Counter(str(v) for v in uvar))}}
        if tune:
            # (1) each bucket tuned on one image in isolation (bf_autotune)
            nb, tsec = _tune_buckets(bf, specs, dev)
            tms, titems, tvar = measure()
            res["tuned_single_image"] = {
                "graph_ms": tms, "mpx_s": px / tms / 1e3, "work_items": titems,
                "buckets_tuned": nb, "tuning_s": tsec,
                "variants": dict(collections.Counter(str(v) for v in tvar)),
                "images_changed": int(sum(a != b for a, b in zip(uvar, tvar)))}
            # (2) each bucket tuned on the whole batch's graph time, from the built-in table
            for key in saved:
                bf.tuning_set(*key, -1)
            t0 = time.perf_counter()
            entries, _, _ = tuning.autotune_batch(imgs, outs, specs, reps=2, coverage=0.9)
            bsec = time.perf_counter() - t0
            bms, bitems, bvar = measure()
            res["tuned"] = {"graph_ms": bms, "mpx_s": px / bms / 1e3, "work_items": bitems,
                            "tuner": "per bucket on the batch graph time (greedy, 1% margin, "
                                     "buckets covering 90% of the work)",
                            "buckets_tuned": len(entries), "tuning_s": bsec,
                            "entries_changed": int(sum(e["variant"] != -1 for e in entries)),
                            "variants": dict(collections.Counter(str(v) for v in bvar)),
                            "images_changed": int(sum(a != b for a, b in zip(uvar, bvar)))}
        k = int(np.argmax([sp["N"] for sp in specs]))
        sp = specs[k]
        ys, xs = _samples(np.random.default_rng(23), sp["height"], sp["width"], 200)
        keep["batch_256"] = {"img": host[k], "ys": ys, "xs": xs, "spec": sp,
                             "fast": _at(outs[k], ys, xs)}
    finally:
        for key, v in saved.items():
            bf.tuning_set(*key, v)
    del imgs, outs
    torch.cuda.empty_cache()
    return res


def study_grad512(bf, synth, dev, stream, flush, keep):
    """32 images of 512^2 blocks(16)+N(0,20^2); Gaussian sigma_s = 5 (W = 15),
    sigma_r = 25, N from the bound for delta = 1: forward + backward (image and
    sigma_r gradients), power images recomputed or stored, against the direct
    filter's forward + backward; the 32 images on 8 streams in one captured
    graph (a 512^2 image alone fills only part of the GPU)."""
    import numpy as np
    import torch
    R, ss, sr = 15, 5.0, 25.0
    N = bf.order_from_delta(bf.GAUSS, R, ss, sr, 1.0)
    host = [synth.blocks_image(512, 512, 16, 20.0, seed=4000 + k) for k in range(32)]
    ghost = [synth.random_like((512, 512), seed=5000 + k) for k in range(32)]
    xs_ = [torch.from_numpy(a).to(dev) for a in host]
    gs_ = [torch.from_numpy(a).to(dev) for a in ghost]
    side = [torch.cuda.Stream(dev) for _ in range(8)]

    def fanout(body):
        def run():
            cur = torch.cuda.current_stream(dev)
            for k, (x, g) in enumerate(zip(xs_, gs_)):
                s = side[k % len(side)]
                s.wait_stream(cur)
                with torch.cuda.stream(s):
                    body(x, g)
            for s in side:
                cur.wait_stream(s)
        return run

    def fb(store):
        def body(x, g):
            if store:
                o, q, ab = bf.gpa_forward_stored(x, bf.GAUSS, sr, N, radius=R, sigma_s=ss)
            else:
                o, q = bf.gpa_forward(x, bf.GAUSS, sr, N, radius=R, sigma_s=ss, return_q=True)
                ab = None
            bf.gpa_backward(x, o, q, g, bf.GAUSS, sr, N, radius=R, sigma_s=ss, abar=ab)
        return fanout(body)

    def dbody(x, g):
        bf.direct(x, bf.GAUSS, sr, radius=R, sigma_s=ss)
        bf.direct_backward(x, g, bf.GAUSS, sr, radius=R, sigma_s=ss)

    def graphed(fn):
        s = torch.cuda.Stream(dev)
        s.wait_stream(stream)
        with torch.cuda.stream(s):
            fn()
            fn()
        torch.cuda.synchronize(dev)
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            fn()
        torch.cuda.synchronize(dev)
        return gr

    px = 32 * 512.0 * 512.0
    g_r, g_s, g_d = graphed(fb(False)), graphed(fb(True)), graphed(fanout(dbody))
    rms = _time_ms(g_r.replay, 3, stream, flush)
    sms = _time_ms(g_s.replay, 3, stream, flush)
    dms = _time_ms(g_d.replay, 2, stream, flush)
    del g_r, g_s, g_d
    # image 0's outputs and gradients (both routes) for the checker
    x0, g0 = xs_[0], gs_[0]
    o, q = bf.gpa_forward(x0, bf.GAUSS, sr, N, radius=R, sigma_s=ss, return_q=True)
    gin, gsig = bf.gpa_backward(x0, o, q, g0, bf.GAUSS, sr, N, radius=R, sigma_s=ss)
    so, sq, ab = bf.gpa_forward_stored(x0, bf.GAUSS, sr, N, radius=R, sigma_s=ss)
    sgin, sgsig = bf.gpa_backward(x0, so, sq, g0, bf.GAUSS, sr, N, radius=R, sigma_s=ss, abar=ab)
    ys, xs = _samples(np.random.default_rng(24), 512, 512, 48)
    keep["grad_512x32"] = {"img": host[0], "g": ghost[0], "ys": ys, "xs": xs, "N": N, "R": R,
                           "ss": ss, "sr": sr, "fast": _at(o, ys, xs), "gin": _at(gin, ys, xs),
                           "gin_scale": float(gin.abs().max()), "gsig": float(gsig.item()),
                           "stored_gin": _at(sgin, ys, xs), "stored_gsig": float(sgsig.item())}
    del xs_, gs_
    torch.cuda.empty_cache()
    return {"workload": "32 x 512x512 blocks(16)+N(0,20^2); Gaussian sigma_s=5 (W=15), "
                        "sigma_r=25, N=%d (bound for delta=1); forward + backward (image and "
                        "sigma_r gradients); 8 streams in one CUDA graph" % N,
            "N": N, "recompute_fwd_bwd_ms": rms, "recompute_mpx_s": px / rms / 1e3,
            "stored_fwd_bwd_ms": sms, "stored_mpx_s": px / sms / 1e3,
            "stored_plane_bytes_per_image": 4 * (N + 1) * 512 * 512,
            "direct_fwd_bwd_ms": dms, "direct_mpx_s": px / dms / 1e3,
            "speedup_vs_direct": dms / rms,
            "max_abs_stored_vs_recompute_gin": float((sgin - gin).abs().max()) /
            max(float(gin.abs().max()), 1e-30)}


# ----------------------------------------------------------------- CPU leg: parity
def cpu_parity(keep):
    """Errors of the GPU outputs that the studies kept at sampled pixels,
    against the FP64 checker: Algorithm 2 at the same N (the parity bar), and
    eq. BF itself (the filter being approximated), for the fast path and for
    the direct filter, so that "equal max error" is measured, not assumed."""
    import numpy as np

    import oracle

    def mx(a, b):
        return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max())

    out = {}
    t0 = time.perf_counter()
    h = keep.get("headline")
    if h:
        w = oracle.spatial_kernel(h["kind"], h["R"], h["ss"])
        pix = (h["ys"], h["xs"])
        alg2 = oracle.gpa_alg2_at(h["img"], w, h["sr"], h["N"], pix)
        exact = oracle.bf_direct(h["img"], w, h["sr"], samples=pix)
        d = {"samples": int(len(h["ys"])), "N": h["N"],
             "fast_vs_alg2_max_abs": mx(h["fast"], alg2),
             "fast_vs_eq_bf_max_abs": mx(h["fast"], exact)}
        if "direct" in h:
            d["direct_vs_eq_bf_max_abs"] = mx(h["direct"], exact)
        e = keep.get("equal_error")
        if e:
            d["N_eq"] = e["N_eq"]
            d["fast_N_eq_vs_alg2_max_abs"] = mx(e["fast_eq"], oracle.gpa_alg2_at(
                e["img"], w, e["sr"], e["N_eq"], (e["ys"], e["xs"])))
            d["fast_N_eq_vs_eq_bf_max_abs"] = mx(e["fast_eq"], oracle.bf_direct(
                e["img"], w, e["sr"], samples=(e["ys"], e["xs"])))
        out["headline"] = d
    big = keep.get("large_8192")
    if big:
        w = oracle.spatial_kernel(1, big["R"], big["ss"])
        pix = (big["ys"], big["xs"])
        exact = oracle.bf_direct(big["img"], w, big["sr"], samples=pix)
        d = {"samples": int(len(big["ys"])),
             "fast_vs_alg2_max_abs": mx(big["fast"], oracle.gpa_alg2_at(big["img"], w, big["sr"],
                                                                       big["N"], pix)),
             "fast_vs_eq_bf_max_abs": mx(big["fast"], exact)}
        if "direct" in big:
            d["direct_vs_eq_bf_max_abs"] = mx(big["direct"], exact)
        out["large_8192"] = d
    b = keep.get("batch_256")
    if b:
        sp = b["spec"]
        w = oracle.spatial_kernel(sp["kind"], sp["radius"], sp["sigma_s"])
        out["batch_256"] = {"image": "the largest-N image (N=%d)" % sp["N"],
                            "samples": int(len(b["ys"])),
                            "fast_vs_alg2_max_abs": mx(b["fast"], oracle.gpa_alg2_at(
                                b["img"], w, sp["sigma_r"], sp["N"], (b["ys"], b["xs"])))}
    gr = keep.get("grad_512x32")
    if gr:
        w = oracle.spatial_kernel(1, gr["R"], gr["ss"])
        pix = (gr["ys"], gr["xs"])
        gref, gsref = oracle.gpa_grad(gr["img"], w, gr["sr"], gr["N"],
                                      gr["g"].astype(np.float64), samples=pix)
        scale = max(float(np.abs(gref).max()), gr["gin_scale"], 1e-30)
        out["grad_512x32"] = {
            "image": "the first of the 32", "samples": int(len(gr["ys"])),
            "fast_vs_alg2_max_abs": mx(gr["fast"], oracle.gpa_alg2_at(gr["img"], w, gr["sr"],
                                                                      gr["N"], pix)),
            "gin_rel_err": mx(gr["gin"], gref) / scale,
            "stored_gin_rel_err": mx(gr["stored_gin"], gref) / scale,
            "gsigma_rel_err": abs(gr["gsig"] - gsref) / max(abs(gsref), 1e-30),
            "stored_gsigma_rel_err": abs(gr["stored_gsig"] - gsref) / max(abs(gsref), 1e-30)}
    out["checker_s"] = time.perf_counter() - t0
    return out


# ----------------------------------------------------------------- sweeps
def _time_ms(fn, reps, stream, flush=None):
    """Mean CUDA-event time of fn() over reps calls (L2 flushed between)."""
    import torch
    fn()
    torch.cuda.synchronize()
    total = 0.0
    for k in range(reps):
        if flush is not None:
            flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total / reps


def run_sweeps(args):
    """Extra studies behind the headline: one JSON line per measured point."""
    import numpy as np
    import torch

    import paper_1603_08109_gb300 as bf
    from paper_1603_08109_gb300 import synth
    names = set(args.sweep.split(",")) if args.sweep != "all" else {
        "grid2048", "roofline4096", "large8192", "recursive", "batch256", "grad512", "joint2048",
        "tightness", "volume"}
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    pk, pk_src = peaks()
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))

    def emit(d):
        print(json.dumps(d), flush=True)

    if "grid2048" in names:
        # 2048^2 blocks(64)+N(0,10^2); box W in {5,20,50}, Gaussian sigma_s in {3,10};
        # sigma_r in {10,30,60}; N in {2, bound/2, bound}; fast vs direct, forward only
        x = torch.from_numpy(synth.blocks_image(2048, 2048, 64, 10.0, seed=1000)).to(dev)
        o = torch.empty_like(x)
        d = torch.empty_like(x)
        for kind, R, ss in ((bf.BOX, 5, 0.0), (bf.BOX, 20, 0.0), (bf.BOX, 50, 0.0),
                            (bf.GAUSS, 9, 3.0), (bf.GAUSS, 30, 10.0)):
            for sr in (10.0, 30.0, 60.0):
                nb = bf.order_from_delta(kind, R, ss, sr, 1.0)
                dms = _time_ms(lambda: bf.direct(x, kind, sr, radius=R, sigma_s=ss, out=d),
                               3, stream, flush)
                for N in sorted({2, max(2, nb // 2), nb}):
                    try:
                        fms = _time_ms(lambda: bf.gpa_forward(x, kind, sr, N, radius=R,
                                                              sigma_s=ss, out=o), 5, stream, flush)
                    except bf._lib.BFError as e:
                        emit({"sweep": "grid2048", "kind": kind, "radius": R, "sigma_r": sr,
                              "N": N, "error": str(e)})
                        continue
                    err = float((o.double() - d.double()).abs().max()) if N == nb else None
                    emit({"sweep": "grid2048", "kind": "box" if kind == 0 else "gaussian",
                          "radius": R, "sigma_s": ss, "sigma_r": sr, "N": N, "N_bound": nb,
                          "fast_fwd_ms": fms, "fast_fwd_mpx_s": 4.194304 / fms * 1e3,
                          "direct_fwd_ms": dms, "direct_fwd_mpx_s": 4.194304 / dms * 1e3,
                          "speedup_vs_direct": dms / fms, "max_abs_fast_vs_direct": err})
    if "roofline4096" in names:
        # 4096^2 gradient + polygons; HBM fraction of the fused forward (8 B/px: f in, out)
        x = torch.from_numpy(synth.gradient_polygons_image(4096, 4096, 64, 15.0, seed=2000)).to(dev)
        o = torch.empty_like(x)
        px = 4096.0 * 4096.0
        cms = _time_ms(lambda: o.copy_(x), 10, stream, flush)
        emit({"sweep": "roofline4096", "kernel": "torch copy (reference)", "ms": cms,
              "gbs": 8 * px / cms / 1e6, "frac_of_measured_hbm": 8 * px / cms / 1e6 / hbm_peak})
        for kind, R, ss in ((bf.BOX, 3, 0.0), (bf.BOX, 5, 0.0), (bf.GAUSS, 9, 3.0)):
            nb = bf.order_from_delta(kind, R, ss, 40.0, 1.0)
            for N in (1, 2, 3, 5, 8, nb):
                fms = _time_ms(lambda: bf.gpa_forward(x, kind, 40.0, N, radius=R, sigma_s=ss,
                                                      out=o), 10, stream, flush)
                gbs = 8 * px / fms / 1e6
                emit({"sweep": "roofline4096", "kind": "box" if kind == 0 else "gaussian",
                      "radius": R, "sigma_r": 40.0, "N": N, "fwd_ms": fms,
                      "fwd_mpx_s": px / fms / 1e3, "algorithmic_gbs": gbs,
                      "frac_of_measured_hbm": gbs / hbm_peak, "hbm_peak_src": pk_src,
                      "alu_ops_frac": fwd_ops_per_pixel(kind, R, N) * px / (fms * 1e-3) /
                      fp32_peak_ops(152, float(pk.get("sm_max_mhz", 2070.0)))})
        # back-to-back launches over 8 rotating image/output pairs (1 GB in all, so every
        # launch reads inputs and writes outputs that are not in L2): the per-launch time
        # without an isolated launch's latency and ramp, for the copy and the small-N box
        K = 8
        xs = [torch.from_numpy(synth.gradient_polygons_image(4096, 4096, 64, 15.0,
                                                             seed=2000 + k)).to(dev) for k in range(K)]
        os_ = [torch.empty_like(xs[0]) for _ in range(K)]

        def stream_ms(body, rounds=5):
            for k in range(K):
                body(xs[k], os_[k])
            torch.cuda.synchronize()
            best = []
            for _ in range(rounds):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for k in range(K):
                    body(xs[k], os_[k])
                e1.record(stream)
                e1.synchronize()
                best.append(e0.elapsed_time(e1) / K)
            return statistics.median(best)

        cms = stream_ms(lambda a, b: b.copy_(a))
        emit({"sweep": "roofline4096", "timing": "back-to-back, 8 rotating pairs",
              "kernel": "torch copy (reference)", "ms": cms, "gbs": 8 * px / cms / 1e6,
              "frac_of_measured_hbm": 8 * px / cms / 1e6 / hbm_peak})
        for R in (3, 5):
            for N in (1, 2, 3):
                fms = stream_ms(lambda a, b: bf.gpa_forward(a, bf.BOX, 40.0, N, radius=R, out=b))
                gbs = 8 * px / fms / 1e6
                emit({"sweep": "roofline4096", "timing": "back-to-back, 8 rotating pairs",
                      "kind": "box", "radius": R, "sigma_r": 40.0, "N": N, "fwd_ms": fms,
                      "fwd_mpx_s": px / fms / 1e3, "algorithmic_gbs": gbs,
                      "frac_of_measured_hbm": gbs / hbm_peak, "hbm_peak_src": pk_src})
        # the same 8 images as one batch (bf_fast_forward_many): one launch of the
        # warp-strip kernel for all of them; per-image time = batch time / 8
        xb = torch.stack(xs)
        ob = torch.empty_like(xb)
        del xs, os_
        cms = _time_ms(lambda: ob.copy_(xb), 5, stream, flush) / K
        emit({"sweep": "roofline4096", "timing": "one call for a batch of 8", "kernel":
              "torch copy (reference)", "ms": cms, "gbs": 8 * px / cms / 1e6,
              "frac_of_measured_hbm": 8 * px / cms / 1e6 / hbm_peak})
        for R in (3, 5):
            for N in (1, 2, 3):
                fms = _time_ms(lambda: bf.gpa_forward_many(xb, bf.BOX, 40.0, N, radius=R, out=ob),
                               5, stream, flush) / K
                gbs = 8 * px / fms / 1e6
                emit({"sweep": "roofline4096", "timing": "one call for a batch of 8",
                      "kind": "box", "radius": R, "sigma_r": 40.0, "N": N, "fwd_ms": fms,
                      "fwd_mpx_s": px / fms / 1e3, "algorithmic_gbs": gbs,
                      "frac_of_measured_hbm": gbs / hbm_peak, "hbm_peak_src": pk_src})
        del xb, ob
        torch.cuda.empty_cache()
        # the same generator at 8192^2: the small-N box forward past the launch ramp and tail
        x = torch.from_numpy(synth.gradient_polygons_image(8192, 8192, 64, 15.0, seed=2001)).to(dev)
        o = torch.empty_like(x)
        px = 8192.0 * 8192.0
        cms = _time_ms(lambda: o.copy_(x), 10, stream, flush)
        emit({"sweep": "roofline4096", "size": 8192, "kernel": "torch copy (reference)", "ms": cms,
              "gbs": 8 * px / cms / 1e6, "frac_of_measured_hbm": 8 * px / cms / 1e6 / hbm_peak})
        for R in (3, 5):
            fms = _time_ms(lambda: bf.gpa_forward(x, bf.BOX, 40.0, 1, radius=R, out=o), 10, stream,
                           flush)
            gbs = 8 * px / fms / 1e6
            emit({"sweep": "roofline4096", "size": 8192, "kind": "box", "radius": R, "sigma_r": 40.0,
                  "N": 1, "fwd_ms": fms, "fwd_mpx_s": px / fms / 1e3, "algorithmic_gbs": gbs,
                  "frac_of_measured_hbm": gbs / hbm_peak, "hbm_peak_src": pk_src})
        del x, o
    if "large8192" in names:
        keep = {}
        emit(dict(sweep="large8192", **study_large8192(bf, synth, dev, stream, flush, fp32_peak_ops(
            152, float(pk.get("sm_max_mhz", 2070.0))), keep)))
    if "recursive" in names:
        # Algorithm 2 with the recursive (Deriche) Gaussian: cost independent of
        # sigma_s, against the truncated-Gaussian FIR forward (fused tile or banded
        # two-pass) at the same sigma_s; gradient + polygons, sigma_r=40, delta=0.5
        fp32 = fp32_peak_ops(152, float(pk.get("sm_max_mhz", 2070.0)))
        for size in (2048, 8192):
            x = torch.from_numpy(synth.gradient_polygons_image(size, size, 64, 15.0,
                                                               seed=2001)).to(dev)
            o = torch.empty_like(x)
            o2 = torch.empty_like(x)
            px = float(size * size)
            for ss in (3.0, 10.0, 20.0, 40.0):
                N = bf.order_from_delta(bf.GAUSS_RECURSIVE, 0, ss, 40.0, 0.5)
                ws = torch.empty(bf.recursive_workspace_bytes(size, size, N) // 4, device=dev)
                rms = _time_ms(lambda: bf.recursive_forward(x, 40.0, N, ss, out=o, ws=ws), 5,
                               stream, flush)
                row = {"sweep": "recursive", "size": size, "sigma_s": ss, "sigma_r": 40.0, "N": N,
                       "rec_fwd_ms": rms, "rec_fwd_mpx_s": px / rms / 1e3,
                       "rec_algorithmic_gbs": rec_bytes_per_pixel(N) * px / rms / 1e6,
                       "rec_frac_of_measured_hbm": rec_bytes_per_pixel(N) * px / rms / 1e6 / hbm_peak,
                       "rec_alu_ops_frac": rec_ops_per_pixel(N) * px / (rms * 1e-3) / fp32}
                del ws
                R = int(math.ceil(3.0 * ss - 1e-9))
                if R <= 96:
                    Nf = bf.order_from_delta(bf.GAUSS, R, ss, 40.0, 0.5)
                    fms = _time_ms(lambda: bf.gpa_forward(x, bf.GAUSS, 40.0, Nf, radius=R,
                                                          sigma_s=ss, out=o2), 3, stream, flush)
                    row.update({"fir_radius": R, "fir_N": Nf, "fir_fwd_ms": fms,
                                "speedup_vs_fir": fms / rms,
                                "max_abs_rec_vs_fir": float((o - o2).abs().max())})
                    if size == 2048 and ss in (3.0, 20.0):
                        d = torch.empty_like(x)
                        dms = _time_ms(lambda: bf.direct(x, bf.GAUSS, 40.0, radius=R, sigma_s=ss,
                                                         out=d), 1, stream, flush)
                        row.update({"direct_ms": dms, "speedup_vs_direct": dms / rms,
                                    "max_abs_rec_vs_direct": float((o - d).abs().max()),
                                    "max_abs_fir_vs_direct": float((o2 - d).abs().max())})
                        del d
                emit(row)
            # forward + backward (image and sigma_r gradients) at sigma_s = 20
            ss = 20.0
            N = bf.order_from_delta(bf.GAUSS_RECURSIVE, 0, ss, 40.0, 0.5)
            q = torch.empty_like(x)
            g = torch.from_numpy(synth.random_like((size, size), seed=2002)).to(dev)
            ws = torch.empty(bf.recursive_workspace_bytes(size, size, N) // 4, device=dev)
            o, q = bf.recursive_forward(x, 40.0, N, ss, return_q=True, ws=ws)
            del ws
            bms = _time_ms(lambda: bf.recursive_backward(x, o, q, g, 40.0, N, ss), 3, stream, flush)
            fms = _time_ms(lambda: bf.recursive_forward(x, 40.0, N, ss, out=o2), 3, stream, flush)
            # the stored pair: the forward keeps the power images' row-pass planes
            wsb = torch.empty(bf.recursive_backward_workspace_bytes(size, size, N) // 4, device=dev)
            so, sq, _ = bf.recursive_forward_stored(x, 40.0, N, ss, ws=wsb)
            sbms = _time_ms(lambda: bf.recursive_backward_stored(x, so, sq, g, 40.0, N, ss, wsb), 3,
                            stream, flush)
            sfms = _time_ms(lambda: bf.recursive_forward_stored(x, 40.0, N, ss, out=so, ws=wsb), 3,
                            stream, flush)
            del wsb, sq
            row = {"sweep": "recursive", "size": size, "sigma_s": ss, "sigma_r": 40.0, "N": N,
                   "rec_fwd_ms": fms, "rec_bwd_ms": bms,
                   "rec_fwd_bwd_mpx_s": px / (fms + bms) / 1e3,
                   "stored_fwd_ms": sfms, "stored_bwd_ms": sbms,
                   "stored_fwd_bwd_mpx_s": px / (sfms + sbms) / 1e3}
            if size == 2048:
                R = 60
                Nf = bf.order_from_delta(bf.GAUSS, R, ss, 40.0, 0.5)
                of, qf = bf.gpa_forward(x, bf.GAUSS, 40.0, Nf, radius=R, sigma_s=ss, return_q=True)
                ffms = _time_ms(lambda: bf.gpa_forward(x, bf.GAUSS, 40.0, Nf, radius=R, sigma_s=ss,
                                                       out=o2), 3, stream, flush)
                fbms = _time_ms(lambda: bf.gpa_backward(x, of, qf, g, bf.GAUSS, 40.0, Nf, radius=R,
                                                        sigma_s=ss), 3, stream, flush)
                row.update({"fir_fwd_ms": ffms, "fir_bwd_ms": fbms,
                            "fir_fwd_bwd_mpx_s": px / (ffms + fbms) / 1e3,
                            "speedup_vs_fir_fwd_bwd": (ffms + fbms) / (fms + bms)})
                del of, qf
            emit(row)
            del g, q
            torch.cuda.empty_cache()
            # the spatial operator alone, and its kernel against the sampled Gaussian
            ws = torch.empty(bf.recursive_workspace_bytes(size, size, 0) // 4, device=dev)
            for ss in (3.0, 40.0):
                ms = _time_ms(lambda: bf.recursive_gauss(x, ss, out=o, ws=ws), 10, stream, flush)
                emit({"sweep": "recursive", "size": size, "filter_only_sigma_s": ss, "ms": ms,
                      "mpx_s": px / ms / 1e3})
            del ws, x, o, o2
            torch.cuda.empty_cache()
        for ss in (3.0, 20.0):
            n = int(math.ceil(12 * ss)) * 2 + 1
            imp = torch.zeros((n, n), device=dev)
            imp[n // 2, n // 2] = 1.0
            hh = bf.recursive_gauss(imp, ss).double().cpu().numpy()
            k = np.arange(n) - n // 2
            g = np.exp(-k * k / (2.0 * ss * ss))
            g2 = np.outer(g, g) / g.sum() ** 2
            emit({"sweep": "recursive", "kernel_vs_sampled_gaussian_sigma_s": ss,
                  "max_abs_dev_rel_to_peak": float(np.abs(hh - g2).max() / g2.max()),
                  "centre_weight_recursive": bf.centre_weight(bf.GAUSS_RECURSIVE, 0, ss),
                  "centre_weight_truncated": bf.centre_weight(bf.GAUSS, int(math.ceil(3 * ss)), ss)})
    if "batch256" in names:
        emit(dict(sweep="batch256", **study_batch256(bf, synth, dev, stream, flush, {})))
    if "tightness" in names:
        # Fig. tightness: orders from Chebyshev / Chernoff / exact Poisson / exhaustive grid
        # search, and the grid sup-norm error each order achieves (1025^2 grid of [-T, T]^2)
        for eps in (0.1, 1e-3):
            for sr in (10.0, 20.0, 30.0, 40.0, 50.0, 60.0):
                ch, cn, po = bf.order_estimates(sr, eps, 128.0)
                ex = bf.exhaustive_order(sr, eps, 128.0, grid=1025)
                t0 = time.perf_counter()
                errs = {k: bf.kernel_error_max(n, sr, 128.0, 1025)
                        for k, n in (("chebyshev", ch), ("chernoff", cn), ("poisson", po),
                                     ("exhaustive", ex))}
                gpu_s = (time.perf_counter() - t0) / 4
                emit({"sweep": "tightness", "eps": eps, "sigma_r": sr, "N_chebyshev": ch,
                      "N_chernoff": cn, "N_poisson": po, "N_exhaustive": ex,
                      "grid_error": errs, "s_per_grid_eval_gpu": gpu_s})
    if "volume" in names:
        # a 128 x 256 x 256 volume (video: 128 frames of blocks(16)+N(0,10^2));
        # separable 3-D kernel, sigma_r=30, N from delta=1 with w(0) = w1(0)^3
        D3, H3, W3 = 128, 256, 256
        v = torch.from_numpy(np.stack([synth.blocks_image(H3, W3, 16, 10.0, seed=6000 + k)
                                       for k in range(D3)])).to(dev)
        o = torch.empty_like(v)
        vox = float(D3 * H3 * W3)
        for kind, R, ss in ((bf.GAUSS, 6, 2.0), (bf.BOX, 3, 0.0)):
            N = bf.volume_order_from_delta(kind, R, ss, 30.0, 1.0)
            ws = torch.empty(bf.volume_workspace_bytes(D3, H3, W3, kind, 30.0, N, R, ss) // 4,
                             device=dev)
            vms = _time_ms(lambda: bf.gpa_volume(v, kind, 30.0, N, radius=R, sigma_s=ss, out=o,
                                                 ws=ws), 5, stream, flush)
            # algorithmic FMAs per voxel and channel: the three 1-D filterings
            ops = (N + 1) * (3 * (2 * R + 1) + 3) * vox
            emit({"sweep": "volume", "shape": [D3, H3, W3], "kind": "box" if kind == 0 else "gaussian",
                  "radius": R, "sigma_r": 30.0, "N": N, "ms": vms, "mvoxel_s": vox / vms / 1e3,
                  "fp32_frac": ops / (vms * 1e-3) / fp32_peak_ops(152, 2070.0),
                  "workspace_bytes": ws.numel() * 4})
            del ws
        del v, o
        torch.cuda.empty_cache()
    if "joint2048" in names:
        # cross (joint) filter: 2048^2 blocks(64) image, gradient+polygons guide
        x = torch.from_numpy(synth.blocks_image(2048, 2048, 64, 10.0, seed=1000)).to(dev)
        e = torch.from_numpy(synth.gradient_polygons_image(2048, 2048, 64, 15.0, seed=1001)).to(dev)
        o = torch.empty_like(x)
        d = torch.empty_like(x)
        for kind, R, ss, sr in ((bf.GAUSS, 9, 3.0, 30.0), (bf.GAUSS, 30, 10.0, 30.0),
                                (bf.BOX, 20, 0.0, 30.0)):
            N = bf.order_from_delta(kind, R, ss, sr, 1.0)
            fms = _time_ms(lambda: bf.joint_forward(x, e, kind, sr, N, radius=R, sigma_s=ss, out=o),
                           5, stream, flush)
            dms = _time_ms(lambda: bf.joint_direct(x, e, kind, sr, radius=R, sigma_s=ss, out=d),
                           3, stream, flush)
            emit({"sweep": "joint2048", "kind": "box" if kind == 0 else "gaussian", "radius": R,
                  "sigma_r": sr, "N": N, "fast_fwd_ms": fms, "fast_fwd_mpx_s": 4.194304 / fms * 1e3,
                  "direct_fwd_ms": dms, "direct_fwd_mpx_s": 4.194304 / dms * 1e3,
                  "speedup_vs_direct": dms / fms,
                  "max_abs_fast_vs_direct": float((o.double() - d.double()).abs().max())})
        # the recursive Gaussian (the same cost for any sigma_s) against the banded
        # truncated-Gaussian joint filter at sigma_s = 10 and 20
        for ss in (10.0, 20.0):
            N = bf.order_from_delta(bf.GAUSS_RECURSIVE, 0, ss, 30.0, 1.0)
            ws = torch.empty(bf.recursive_backward_workspace_bytes(2048, 2048, N) // 4, device=dev)
            rms = _time_ms(lambda: bf.recursive_joint_forward(x, e, 30.0, N, ss, out=o, ws=ws), 5,
                           stream, flush)
            R = int(math.ceil(3.0 * ss - 1e-9))
            Nf = bf.order_from_delta(bf.GAUSS, R, ss, 30.0, 1.0)
            fms = _time_ms(lambda: bf.joint_forward(x, e, bf.GAUSS, 30.0, Nf, radius=R, sigma_s=ss,
                                                    out=d), 3, stream, flush)
            emit({"sweep": "joint2048", "kind": "gaussian_recursive", "sigma_s": ss,
                  "sigma_r": 30.0, "N": N, "rec_fwd_ms": rms, "rec_fwd_mpx_s": 4.194304 / rms * 1e3,
                  "fir_radius": R, "fir_N": Nf, "fir_fwd_ms": fms, "speedup_vs_fir": fms / rms,
                  "max_abs_rec_vs_fir": float((o.double() - d.double()).abs().max())})
            del ws
    if "grad512" in names:
        emit(dict(sweep="grad512", **study_grad512(bf, synth, dev, stream, flush, {})))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweeps(args)

    import ctypes

    import numpy as np
    import torch

    import paper_1603_08109_gb300 as bf
    from paper_1603_08109_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    kind = bf.GAUSS if args.kind == "gauss" else bf.BOX
    R, ss, sr = args.radius, args.sigma_s, args.sigma_r
    S, B = args.size, args.batch
    t0 = time.perf_counter()
    N = args.order or bf.order_from_delta(kind, R, ss, sr, 1.0)  # A0, host, once per workload
    order_ms = 1e3 * (time.perf_counter() - t0)
    # B distinct device images per step: NB seeded host images, each in B / NB
    # row rotations (a rotated blocks image is a blocks image of the same recipe)
    NB = min(B, 8)
    base_np = [synth.blocks_image(S, S, 64, 10.0, seed=1000 + rank * NB + k) for k in range(NB)]
    gbase_np = [synth.random_like((S, S), seed=77 + rank * NB + k) for k in range(NB)]
    base = [torch.from_numpy(a).to(dev) for a in base_np]
    gbase = [torch.from_numpy(a).to(dev) for a in gbase_np]
    xs = [torch.roll(base[k % NB], shifts=37 * (k // NB), dims=0).contiguous() for k in range(B)]
    gs_ = [torch.roll(gbase[k % NB], shifts=37 * (k // NB), dims=0).contiguous() for k in range(B)]
    del base, gbase
    outs = [torch.empty_like(xs[0]) for _ in range(B)]
    qs = [torch.empty_like(xs[0]) for _ in range(B)]
    gins = [torch.empty_like(xs[0]) for _ in range(B)]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    p = bf._lib.make_params(kind, R, ss, sr, N)
    lib = bf._lib.lib()
    sp = ctypes.c_void_p(stream.cuda_stream)
    nws = ctypes.c_size_t(0)
    if args.only != "fwd":
        bf._lib.check(lib.bf_fast_backward_workspace(S, S, ctypes.byref(p), ctypes.byref(nws)),
                      "ws")
    ws = torch.empty(max(nws.value, 1), dtype=torch.uint8, device=dev)
    gsig = torch.zeros(B, dtype=torch.float64, device=dev)
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    # the banded two-pass forward (radii above 15 by default) needs a workspace
    nfws = ctypes.c_size_t(0)
    bf._lib.check(lib.bf_fast_forward_workspace(S, S, ctypes.byref(p), ctypes.byref(nfws)), "fws")
    fws = torch.empty(max(nfws.value, 16), dtype=torch.uint8, device=dev)

    def fwd(k):
        bf._lib.check(lib.bf_fast_forward_ws(P(xs[k]), P(outs[k]), P(qs[k]), S, S, S,
                                             ctypes.byref(p), P(fws), nfws, sp), "fwd")

    def bwd(k):
        bf._lib.check(lib.bf_fast_backward(P(xs[k]), P(outs[k]), P(qs[k]), P(gs_[k]), P(gins[k]),
                                           ctypes.c_void_p(gsig.data_ptr() + 8 * k), S, S, S,
                                           ctypes.byref(p), P(ws), nws, sp), "bwd")

    fwd_launches = 1
    if nfws.value > 0:  # banded forward: a column pass and a row pass per band
        band_rows = nfws.value // ((N + 1) * ((S + 3) // 4 * 4) * 4)
        fwd_launches = 2 * ((S + band_rows - 1) // band_rows)
    launches_per = B * {"all": fwd_launches + 2, "fwd": fwd_launches, "bwd": 2}[args.only]
    if args.only == "bwd":
        for k in range(B):
            fwd(k)

    def step(ev):
        for k in range(B):
            if args.only in ("all", "fwd"):
                ev[k][0].record(stream)
                fwd(k)
                ev[k][1].record(stream)
            if args.only in ("all", "bwd"):
                ev[k][2].record(stream)
                bwd(k)
                ev[k][3].record(stream)

    def new_events():
        return [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(B)]

    for _ in range(args.warmup):
        step(new_events())
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    if rank == 0:
        sampler.start()
    evs = [new_events() for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))  # evict L2 between steps (outside the step's events)
        step(evs[k])
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clocks = sampler.stop() if rank == 0 else None

    first = 0 if args.only in ("all", "fwd") else 2
    last = 3 if args.only in ("all", "bwd") else 1
    step_spans = [e[0][first].elapsed_time(e[B - 1][last]) for e in evs]
    fwd_ms = ([e[k][0].elapsed_time(e[k][1]) for e in evs for k in range(B)]
              if args.only in ("all", "fwd") else [0.0])
    bwd_ms = ([e[k][2].elapsed_time(e[k][3]) for e in evs for k in range(B)]
              if args.only in ("all", "bwd") else [0.0])
    t_total = sum(step_spans)
    if dist:
        tt = torch.tensor([t_total], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_total = float(tt.item())
    px = float(S) * S
    value = px * B * world * args.steps / (t_total * 1e-3) / 1e6
    mf = statistics.mean(fwd_ms) if args.only != "bwd" else None
    mb = statistics.mean(bwd_ms) if args.only != "fwd" else None
    fwd_mpx = px / (mf * 1e-3) / 1e6 if mf else None

    # ---- e2e through the public API with host buffers (pinned), copies inside the region.
    # Every image copies its own input and cotangent host->device and its gradients
    # device->host; the copies run on their own streams, double-buffered, so image
    # k+1's upload and image k's download overlap image k's filter.
    e2e = None
    if args.only == "all":
        hx = torch.from_numpy(base_np[0]).pin_memory()
        hg = torch.from_numpy(gbase_np[0]).pin_memory()
        hgin = torch.empty((S, S), dtype=torch.float32).pin_memory()
        hgs = torch.empty(1, dtype=torch.float64).pin_memory()
        sig = torch.tensor(sr, device=dev, requires_grad=True)
        up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        dx = [torch.empty((S, S), dtype=torch.float32, device=dev) for _ in range(2)]
        dg = [torch.empty((S, S), dtype=torch.float32, device=dev) for _ in range(2)]
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_free = [torch.cuda.Event() for _ in range(2)]
        for e in ev_free:
            e.record(stream)

        def upload(k):
            b = k % 2
            up.wait_event(ev_free[b])  # the image that last used buffer b is done with it
            with torch.cuda.stream(up):
                dx[b].copy_(hx, non_blocking=True)
                dg[b].copy_(hg, non_blocking=True)
            ev_in[b].record(up)

        def compute(k):
            b = k % 2
            stream.wait_event(ev_in[b])
            xd = dx[b].detach().requires_grad_(True)
            o = bf.gpa_bilateral(xd, sig, kind=kind, N=N, radius=R, sigma_s=ss)
            o.backward(dg[b])
            ev_free[b].record(stream)
            grad, sgrad = xd.grad, sig.grad.double().reshape(1)
            sig.grad = None
            down.wait_stream(stream)
            grad.record_stream(down)
            sgrad.record_stream(down)
            with torch.cuda.stream(down):
                hgin.copy_(grad, non_blocking=True)
                hgs.copy_(sgrad, non_blocking=True)

        def run(n):
            upload(0)
            for k in range(n):
                if k + 1 < n:
                    upload(k + 1)
                compute(k)
            stream.wait_stream(down)

        run(2)
        torch.cuda.synchronize(dev)
        ne = max(10, min(args.steps * B, 200))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        up.wait_stream(stream)
        run(ne)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ems = e0.elapsed_time(e1) / ne
        e2e = {"value": px / (ems * 1e-3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(hx.numel() * 4 + hg.numel() * 4) * B,
               "d2h_bytes_per_step": int(hgin.numel() * 4 + 8) * B,
               "ms_per_image": ems, "images_timed": ne,
               "api": "paper_1603_08109_gb300.gpa_bilateral + backward",
               "copies": "per image: input and cotangent up, image and sigma_r gradients down; "
                         "separate upload/download streams, double-buffered inputs",
               "sigma_r": "a CUDA tensor with requires_grad, unchanged between images: the "
                          "binding reads its host value once per tensor version"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    keep = {}
    x0, out0, g0 = xs[0], outs[0], gs_[0]
    rng = np.random.default_rng(20)
    hys, hxs = _samples(rng, S, S, 3000)
    if args.only != "bwd":
        fwd(0)
        keep["headline"] = {"img": base_np[0], "ys": hys, "xs": hxs, "kind": kind, "R": R,
                            "ss": ss, "sr": sr, "N": N, "fast": _at(out0, hys, hxs)}

    # ---- direct filter on the same image (same-GPU comparison)
    direct = None
    if not args.no_direct and args.only == "all":
        pd = bf._lib.make_params(kind, R, ss, sr, 1)
        dws_n = ctypes.c_size_t()
        bf._lib.check(lib.bf_direct_backward_workspace(S, S, ctypes.byref(pd), ctypes.byref(dws_n)),
                      "dws")
        dws = torch.empty(dws_n.value, dtype=torch.uint8, device=dev)
        dout = torch.empty_like(x0)
        dgin = torch.empty_like(x0)
        dgs = torch.zeros(1, dtype=torch.float64, device=dev)

        def dfwd():
            bf._lib.check(lib.bf_direct(P(x0), P(dout), S, S, S, ctypes.byref(pd), sp), "direct")

        dbwd_ok = [True]

        def dbwd():
            if not dbwd_ok[0]:
                return
            st = lib.bf_direct_backward(P(x0), P(gs_[0]), P(dgin), P(dgs), S, S, S,
                                        ctypes.byref(pd), P(dws), dws_n, sp)
            if st == 3:  # the direct gradient's tile does not fit shared memory at this radius
                dbwd_ok[0] = False
                return
            bf._lib.check(st, "dbwd")
        for _ in range(2):
            dfwd()
            dbwd()
        nd = 10
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(nd)]
        for k in range(nd):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            dfwd()
            ev[k][1].record(stream)
            dbwd()
            ev[k][2].record(stream)
        torch.cuda.synchronize(dev)
        dfm = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
        dbm = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
        diff = (out0.double() - dout.double())
        direct = {"fwd_mpx_s": px / (dfm * 1e-3) / 1e6,
                  "fwd_bwd_mpx_s": px / ((dfm + dbm) * 1e-3) / 1e6 if dbwd_ok[0] else None,
                  "fwd_ms": dfm, "bwd_ms": dbm if dbwd_ok[0] else None,
                  "fast_vs_direct_max_abs": float(diff.abs().max()),
                  "fast_vs_direct_mse_db": float(10 * math.log10(max(float((diff ** 2).mean()),
                                                                     1e-300)))}
        keep["headline"]["direct"] = _at(dout, hys, hxs)
        del dws, dout, dgin

    # ---- roofline of the dominant kernel (FP32 pipe), live CUDA-event timing
    pk, pk_src = peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    fpeak = fp32_peak_ops(props.multi_processor_count, sm_max)
    fo = fwd_ops_per_pixel(kind, R, N) * px
    bo = bwd_ops_per_pixel(kind, R, N) * px
    cand = []
    if mf:
        cand.append(("gpa_fwd_fixed_db_kernel" if R in FIXED_RADII else
                     ("band_vpass+band_hpass" if nfws.value > 0 else "gpa_fwd_kernel"), mf, fo))
    if mb:
        cand.append(("gpa_bwd_tmem_kernel" if R in FIXED_RADII else "gpa_bwd_kernel", mb, bo))
    name, ms, ops = max(cand, key=lambda c: c[1])
    achieved = ops / (ms * 1e-3) / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as fh:
            tj = json.load(fh)
        ent = tj.get(name)
        if ent and ent.get("size") == S and ent.get("N") == N and ent.get("radius") == R:
            traffic = ent.get("bytes")
    roofline = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": fpeak / 1e12,
                "unit": "TFLOP/s", "frac": achieved * 1e12 / fpeak, "traffic": traffic,
                "peak_src": "FP32 pipe: %d SMs x 128 lanes x %.0f MHz (%s sm_max_mhz); one FMA = "
                            "one op" % (props.multi_processor_count, sm_max, pk_src),
                "ops_per_launch": ops, "launch_ms": ms}
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    hbm = None
    if mf:
        gbs = px * 12.0 / (mf * 1e-3) / 1e9  # read f, write out and Q'
        hbm = {"fwd_algorithmic_gbs": gbs, "frac_of_measured_hbm": gbs / hbm_peak,
               "peak_gbs": hbm_peak, "peak_src": pk_src}
    del xs, gs_, outs, qs, gins, ws, fws
    torch.cuda.empty_cache()

    # ---- the small-N HBM study at 4096^2 (box W = 3, sigma_r = 40, N = 1; inputs
    # larger than L2): a batch of 8 same-sized images in one call (one launch of
    # the warp-strip box kernel), and one image alone: single launches after an L2
    # flush, and back to back over the 8 images
    hbm_4096 = hbm_4096_single = None
    if world == 1 and not args.no_hbm_study:
        K4, S4 = 8, 4096
        xb = torch.from_numpy(np.stack([synth.blocks_image(S4, S4, 64, 10.0, seed=3000 + k)
                                        for k in range(K4)])).to(dev)
        ob = torch.empty_like(xb)
        ms4 = _time_ms(lambda: bf.gpa_forward_many(xb, bf.BOX, 40.0, 1, radius=3, out=ob), 5,
                       stream, flush) / K4
        gbs4 = 8.0 * S4 * S4 / (ms4 * 1e-3) / 1e9
        hbm_4096 = {"workload": "8 x 4096x4096 blocks(64)+N(0,10^2); box W=3, sigma_r=40, N=1; "
                                "one bf_fast_forward_many call (one launch)",
                    "ms_per_image": ms4, "algorithmic_bytes_per_px": 8,
                    "algorithmic_gbs": gbs4, "frac_of_measured_hbm": gbs4 / hbm_peak,
                    "peak_gbs": hbm_peak, "peak_src": pk_src}
        # single launches of ~30 us: the median of 20 timed launches (a mean would
        # carry the occasional launch that waits on the host)
        def med_ms(fn, fl, reps=20):
            fn()
            torch.cuda.synchronize(dev)
            ts = []
            for k in range(reps):
                fl.fill_(float(k))
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            return statistics.median(ts)
        box1 = lambda: bf.gpa_forward(xb[0], bf.BOX, 40.0, 1, radius=3, out=ob[0])  # noqa: E731
        one = med_ms(box1, flush)
        for k in range(K4):
            bf.gpa_forward(xb[k], bf.BOX, 40.0, 1, radius=3, out=ob[k])
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for r in range(3):
            for k in range(K4):
                bf.gpa_forward(xb[k], bf.BOX, 40.0, 1, radius=3, out=ob[k])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        b2b = e0.elapsed_time(e1) / (3 * K4)
        # the same single launch after a write flush followed by a 256 MB read: L2 then
        # holds clean lines, so the launch does not also write back the flush's dirty data
        rbuf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

        class CleanFlush:
            def fill_(self, v):
                flush.fill_(v)
                rbuf.sum()
        clean = med_ms(box1, CleanFlush())
        cp_dirty = med_ms(lambda: ob[0].copy_(xb[0]), flush)
        cp_clean = med_ms(lambda: ob[0].copy_(xb[0]), CleanFlush())
        del rbuf
        frac = lambda ms: 8.0 * S4 * S4 / (ms * 1e-3) / 1e9 / hbm_peak  # noqa: E731
        hbm_4096_single = {
            "workload": "one 4096x4096 blocks(64)+N(0,10^2) image; box W=3, sigma_r=40, N=1; "
                        "bf_fast_forward (one warp-strip launch)",
            "single_launch_ms": one, "single_launch_frac_of_measured_hbm": frac(one),
            "single_launch_clean_l2_ms": clean,
            "single_launch_clean_l2_frac_of_measured_hbm": frac(clean),
            "back_to_back_ms": b2b, "back_to_back_frac_of_measured_hbm": frac(b2b),
            "copy_reference": {"single_launch_frac": frac(cp_dirty),
                               "single_launch_clean_l2_frac": frac(cp_clean)},
            "flush": "single_launch: after a 512 MB write (L2 left full of dirty lines, which the "
                     "launch writes back); clean_l2: the same write then a 256 MB read; "
                     "single launches: median of 20",
            "peak_gbs": hbm_peak, "peak_src": pk_src}
        del xb, ob
        torch.cuda.empty_cache()

    # ---- the other workloads (each timed on its own; errors from the CPU leg)
    studies = {}
    if world == 1 and not args.no_studies and args.only == "all" and (S, kind, R) == (2048, 1, 9):
        studies["equal_error"] = study_equal_error(bf, base_np[0], x0, g0, kind, R, ss, sr, N, dev,
                                                   stream, flush, keep)
        if direct:
            ee = studies["equal_error"]
            ee["direct_fwd_bwd_ms"] = direct["fwd_ms"] + (direct["bwd_ms"] or float("nan"))
            ee["speedup_vs_direct_fwd_bwd"] = ee["direct_fwd_bwd_ms"] / ee["fast_fwd_bwd_ms"]
        del x0, out0, g0
        torch.cuda.empty_cache()
        studies["large_8192"] = study_large8192(bf, synth, dev, stream, flush, fpeak, keep)
        studies["grad_512x32"] = study_grad512(bf, synth, dev, stream, flush, keep)
        studies["batch_256"] = study_batch256(bf, synth, dev, stream, flush, keep)

    cpu = None
    if not args.no_cpu_baseline and world == 1 and args.only == "all":
        cpu, _ = cpu_baseline(base_np[0], kind, R, ss, sr, N)
        cpu["parity"] = cpu_parity(keep)

    default = (S, kind, R, ss, sr, N, args.only, B) == (2048, 1, 9, 3.0, 30.0, 40, "all", 96)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if default else
                       workload(S, kind, R, ss, sr, N, args.only, B),
                       "image": "%dx%d" % (S, S), "images_per_step": B,
                       "kind": "gaussian" if kind == 1 else "box", "radius": R, "sigma_s": ss,
                       "sigma_r": sr, "N": N, "only": args.only, "l2": L2_NOTE,
                       "parallelism": "dp%d (each rank its own images)" % world},
            "fwd_mpx_s": fwd_mpx, "fwd_ms": mf, "bwd_ms": mb, "order_selection_ms": order_ms,
            "direct": direct, "hbm": hbm, "hbm_4096_batch": hbm_4096,
            "hbm_4096_single": hbm_4096_single, "clocks": clocks, "e2e": e2e,
            "gpu_launches": launches_per * args.steps, "roofline": roofline,
            "cpu_baseline": cpu, "wall_s_timed_region": wall}
    line.update(studies)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
