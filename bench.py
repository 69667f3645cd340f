"""Benchmark of the PXST main loop on GB300. The default workload is the 2-D precision scan
(400 frames of 1024 x 1024 on a 20 x 20 grid of 4 px steps, reference 1200 x 1200, window
+-16 x +-16), synthetic data from the seeded generator. A step is one main-loop iteration
(make_object_map, then update_pixel_map with the 3x3 fit) from the scan's initial map.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pxst|reference]
                    [--workload NAME] [--form all|fp32|bf16|tf32]

Prints one JSON line (rank 0). With --form all (the default) the plain FP32 form and the
tensor-core BF16 and TF32 forms are timed on the same device-resident scan; `value` and
`ms_per_step` are the BF16 form's (pixel-shift-frame evaluations per second over the whole
job; iteration time), and `forms` carries every form's time, rooflines, launches, end-to-end
rate and its error against the FP64 oracle on stated row stripes. Under torchrun each rank
runs its own scan (seed + rank): weak scaling, no collective on the data path.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gen  # noqa: E402

METRIC = "PXST iteration time & pixel·shift·frame evals/s; served scans/s, p50/p99"
UNIT = "pixel·shift·frame evals/s"
# the sources each timed kernel group is built from (a recorded DRAM traffic is used only
# while their hash is unchanged)
KERNEL_SOURCES = {
    "upm_search": ["paper_2003_12726_gb300/csrc/upm.cu", "paper_2003_12726_gb300/csrc/pxst_common.cuh"],
    "upm_rescore": ["paper_2003_12726_gb300/csrc/upm.cu", "paper_2003_12726_gb300/csrc/pxst_common.cuh"],
    "omap_scatter": ["paper_2003_12726_gb300/csrc/omap.cu", "paper_2003_12726_gb300/csrc/pxst_common.cuh"],
    "tensor_search": ["paper_2003_12726_gb300/csrc/tensor.cu", "paper_2003_12726_gb300/csrc/tc_ptx.cuh",
                      "paper_2003_12726_gb300/csrc/pxst_common.cuh"],
}


FORMS = {"fp32": 0, "bf16": 1, "tf32": 2}
WORKLOADS = {"lens1d": (gen.config_lens1d, 1), "small": (gen.config_small, 0),
             "precision2d": (gen.config_precision2d, 2), "precision2d-256": (gen.config_precision2d, 2),
             "precision2d-512": (gen.config_precision2d, 2), "lens1d-256": (gen.config_lens1d, 1),
             "batch64": (None, 3), "serve": (None, 4)}


def make_workload(name, rank):
    fn, idx = WORKLOADS[name]
    seed = gen.BASE_SEED + idx + 1000 * rank
    if name == "small":
        return gen.tiny2d(seed=seed, name="2d-16x64x64-w4")
    if name == "precision2d-256":        # the 2-D precision scan on a 256 x 256 detector (profiling)
        return fn(det=256, ref=400, seed=seed)
    if name == "precision2d-512":        # 512 x 512: frames (420 MB) still larger than L2 (profiling)
        return fn(det=512, ref=680, seed=seed)
    if name == "lens1d-256":             # 256 rows of the lens scan: frames (190 MB) larger than L2 (profiling)
        return fn(ny=256, seed=seed)
    return fn(seed=seed)


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value of x over the ranks (x itself on one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step, world, ms_total, steps):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank_step * world * steps / (ms_total / 1e3)


def evals_per_step(s):
    Sy, Sx = s.window
    return int(s.M.sum()) * (2 * Sy + 1) * (2 * Sx + 1) * s.frames.shape[0]


def kernel_hash(name):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(name, []):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                self.rows.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        rows = [p for (t, p) in self.rows if (t0 is None or t >= t0) and (t1 is None or t <= t1)]
        busy = [p for p in rows if p[4].isdigit() and int(p[4]) > 0] or rows
        if not busy:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(p[1]) for p in busy if num(p[1]) is not None]
        mx = [num(p[2]) for p in busy if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in busy for i in range(4) if p[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(busy)}


# ---------------------------------------------------------------------------------------
def cpu_sample(s, target_s=12.0, max_rows=None, threads=None):
    """The oracle as it stands on a stripe of detector rows: make_object_map from the
    stripe's pixels, then update_pixel_map of the stripe. Rows are added until about
    target_s seconds of CPU work; returns (evals/s, rows, seconds, threads)."""
    import oracle
    threads = threads or oracle.default_threads()
    ny = s.frames.shape[1]
    rows_active = np.flatnonzero(s.M.any(axis=1))
    r0 = int(rows_active[0]) if rows_active.size else 0
    n_rows, spent, evals = 1, 0.0, 0
    Sy, Sx = s.window
    nwin = (2 * Sy + 1) * (2 * Sx + 1)
    while True:
        r1 = min(ny, r0 + n_rows)
        sl = slice(r0, r1)
        fr = np.ascontiguousarray(s.frames[:, sl])
        t = time.perf_counter()
        Iref, w = oracle.make_object_map(fr, s.W[sl], s.M[sl], s.u_init[:, sl], s.delta, s.ref_shape)
        oracle.update_pixel_map(fr, s.W[sl], s.M[sl], Iref, w, s.delta, s.u_init[:, sl], s.window,
                                threads=threads)
        dt = time.perf_counter() - t
        spent, evals = dt, int(s.M[sl].sum()) * nwin * s.frames.shape[0]
        if dt >= target_s * 0.5 or r1 >= ny or (max_rows and n_rows >= max_rows):
            break
        n_rows = max(n_rows + 1, int(n_rows * min(8.0, target_s / max(dt, 1e-3))))
    return evals / spent, r1 - r0, spent, threads


def reference_step(s, threads=None):
    """One step of the reference arm: the oracle as it stands on the sample the pxst arm's
    cpu_baseline uses (make_object_map of the whole scan, then update_pixel_map with the 3x3
    fit of the pixels of the row stripes), extrapolated to the whole iteration by the
    good-pixel count. Returns (evals/s, seconds spent, threads, sample description)."""
    import oracle
    threads = threads or oracle.default_threads()
    rows = stripe_rows(s)
    nx = s.frames.shape[2]
    pix = np.array([r * nx + c for r in rows for c in range(nx) if s.M[r, c]], dtype=np.int64)
    t0 = time.perf_counter()
    Io, wo = oracle.make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    t_omap = time.perf_counter() - t0
    I64, w64 = Io.astype(np.float32).astype(np.float64), wo.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    oracle.update_pixels(s.frames, s.W, s.M, I64, w64, s.delta, s.u_init, s.window, pix, quadratic=True,
                         threads=threads)
    t_upm = time.perf_counter() - t0
    Sy, Sx = s.window
    n_good = int(s.M.sum())
    rate = n_good * (2 * Sy + 1) * (2 * Sx + 1) * s.frames.shape[0] / (t_omap + t_upm * n_good / max(pix.size, 1))
    sample = (f"make_object_map of the whole scan + update_pixel_map with the 3x3 fit of {pix.size} good pixels "
              f"in detector rows {rows[0]}-{rows[len(rows) // 2 - 1]} and {rows[len(rows) // 2]}-{rows[-1]}, "
              f"extrapolated to all {n_good} good pixels (the pxst arm's cpu_baseline sample)")
    return rate, t_omap + t_upm, threads, sample


def reference_arm(args, rank, world):
    if rank != 0:
        return
    s = make_workload(args.workload, 0)
    per_step = []
    for k in range(args.warmup + args.steps):
        rate, sec, threads, sample = reference_step(s)
        if k >= args.warmup:
            per_step.append((rate, sec))
    value = float(np.mean([r for r, _ in per_step]))
    ms = float(np.mean([t for _, t in per_step]) * 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": s.name, "frames": int(s.frames.shape[0]), "detector": list(s.frames.shape[1:]),
                       "window": list(s.window), "reference": list(s.ref_shape)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
def load_traffic(workload, name):
    """DRAM bytes per launch of kernel group `name` on `workload` from profiles/traffic.json,
    or None when none is recorded for the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(workload, {}).get(name)
        if e and e.get("kernel_hash") == kernel_hash(name):
            return e.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def stripe_rows(s, rows_per_stripe=4):
    """The detector rows the accuracy comparison and the oracle's timed sample use: the first
    rows holding good pixels (where candidates read uncovered reference pixels) and the
    central rows."""
    ny = s.frames.shape[1]
    active = np.flatnonzero(s.M.any(axis=1))
    top = int(active[0]) if active.size else 0
    mid = max(top + rows_per_stripe, ny // 2 - rows_per_stripe // 2)
    rows = sorted(set(range(top, min(ny, top + rows_per_stripe))) |
                  set(range(mid, min(ny, mid + rows_per_stripe))))
    return rows


def oracle_leg(s, threads=None):
    """The oracle on a bounded sample of one main-loop iteration: make_object_map of the whole
    scan, then update_pixel_map (integer and with the 3x3 fit) of the pixels of a few row
    stripes. Returns the oracle's results (for the per-form accuracy below) and its timing,
    from which the whole iteration's CPU time is extrapolated by the good-pixel count."""
    import oracle
    threads = threads or oracle.default_threads()
    rows = stripe_rows(s)
    nx = s.frames.shape[2]
    pix = np.array([r * nx + c for r in rows for c in range(nx) if s.M[r, c]], dtype=np.int64)
    t0 = time.perf_counter()
    Io, wo = oracle.make_object_map(s.frames, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    t_omap = time.perf_counter() - t0
    I32, w32 = Io.astype(np.float32), wo.astype(np.float32)
    I64, w64 = I32.astype(np.float64), w32.astype(np.float64)
    t0 = time.perf_counter()
    uo_q, eo_q = oracle.update_pixels(s.frames, s.W, s.M, I64, w64, s.delta, s.u_init, s.window, pix,
                                      quadratic=True, threads=threads)
    t_upm = time.perf_counter() - t0
    uo_i, eo_i = oracle.update_pixels(s.frames, s.W, s.M, I64, w64, s.delta, s.u_init, s.window, pix,
                                      quadratic=False, threads=threads)
    Sy, Sx = s.window
    nwin = (2 * Sy + 1) * (2 * Sx + 1)
    n_good = int(s.M.sum())
    t_iter = t_omap + t_upm * n_good / max(pix.size, 1)
    rate = n_good * nwin * s.frames.shape[0] / t_iter
    return dict(Io=Io, wo=wo, I32=I32, w32=w32, pix=pix, rows=rows, uo_q=uo_q.T, eo_q=eo_q, uo_i=uo_i.T,
                eo_i=eo_i, rate=rate, t_omap=t_omap, t_upm=t_upm, threads=threads,
                sample=f"make_object_map of the whole scan ({t_omap:.1f} s) + update_pixel_map with the 3x3 fit of "
                       f"{pix.size} good pixels in detector rows {rows[0]}-{rows[len(rows) // 2 - 1]} and "
                       f"{rows[len(rows) // 2]}-{rows[-1]} ({t_upm:.1f} s), extrapolated to all {n_good} good pixels")


def accuracy(s, orc, u_int, e_int, u_q):
    """The GPU's update against the oracle's on the stripe pixels, both searching the oracle's
    reference image (rounded to float32): integer argmin agreement, the pixels where they differ
    and whether each is a near-tie (the oracle's own error at the GPU's pick within
    1e-5 e_min + 1e-7 sum I^2 / var of its minimum), and the sub-pixel map difference where the
    integer picks agree."""
    import oracle
    pix = orc["pix"]
    nx = s.frames.shape[2]
    ug_i = u_int.reshape(2, -1)[:, pix]
    ug_q = u_q.reshape(2, -1)[:, pix]
    eg_i = e_int.ravel()[pix]
    same = np.all(ug_i == orc["uo_i"], axis=0)
    bad = np.flatnonzero(~same)
    Sy, Sx = s.window
    I64, w64 = orc["I32"].astype(np.float64), orc["w32"].astype(np.float64)
    ties = 0
    for k in bad[:200]:
        p = int(pix[k])
        e, (ci, cj) = oracle.pixel_window(s.frames, s.W, s.M, I64, w64, s.delta, s.u_init, s.window, p)
        a_ = int(round(ug_i[0, k])) - ci + Sy
        b_ = int(round(ug_i[1, k])) - cj + Sx
        if not (0 <= a_ <= 2 * Sy and 0 <= b_ <= 2 * Sx):
            continue
        I = s.frames[:, p // nx, p % nx].astype(np.float64)
        Wv = float(s.W.ravel()[p])
        scale = float(np.sum(I * I) / max(np.sum((I - Wv) ** 2), 1e-300))
        emin = float(np.min(e))
        ties += int(e[a_, b_] - emin <= 1e-5 * emin + 1e-7 * scale)
    du = np.abs(ug_q - orc["uo_q"])[:, same]
    fin = same & np.isfinite(orc["eo_i"])
    rel = np.abs(eg_i[fin] - orc["eo_i"][fin]) / np.maximum(np.abs(orc["eo_i"][fin]), 1e-30)
    return {"pixels": int(pix.size), "argmin_agree": float(same.mean()) if pix.size else 1.0,
            "differing": int(bad.size), "differing_near_ties": ties,
            "u_max_abs_err_px": float(du.max()) if du.size else 0.0,
            "u_rms_err_px": float(np.sqrt(np.mean(du ** 2))) if du.size else 0.0,
            "err_max_rel": float(rel.max()) if rel.size else 0.0}


def kernel_roofline(name, avg_ms, s, ev_step, form, pk, basis, sms, sm_mhz, extra=None):
    """Algorithmic work of one launch of kernel group `name` over its average launch time,
    against the peak that bounds it. extra: the full loop's translation window (tw), map
    filter radius (filter_r) and conjugate-gradient steps per integration (integ_steps)."""
    extra = extra or {}
    N = s.frames.shape[0]
    P = s.frames.shape[1] * s.frames.shape[2]
    R = s.ref_shape[0] * s.ref_shape[1]
    n_good = int(s.M.sum())
    alu = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    alu_basis = f"{sms} SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz ({basis} max clock)"
    # FP64: 2 DFMA per clock per SM on this GPU (the DFMA peak ncu reports for it)
    fp64 = sms * 2 * 2 * sm_mhz * 1e6 / 1e12
    fp64_basis = f"{sms} SMs x 2 FP64 FMA x 2 flop x {sm_mhz:.0f} MHz ({basis} max clock)"
    if name == "tensor_search":
        work, unit, bound = 2.0 * ev_step / 1e12, "TFLOP/s", "tensor"        # cross term: one multiply-add per eval
        peak = float(pk["bf16_tflops"]) * (0.5 if form == 2 else 1.0)
        pb = f"{basis} dense bf16 cuBLAS burst" + (" x 0.5 (nominal tf32/bf16 ratio)" if form == 2 else "")
    elif name == "upm_search":
        work, unit, bound, peak, pb = 4.0 * ev_step / 1e12, "TFLOP/s", "alu", alu, alu_basis   # 2 FMA per eval
    elif name == "upm_rescore":
        # at least the 3x3 about each pixel's first candidate: 2 FMA per pixel, frame and point
        work, unit, bound, peak, pb = 4.0 * 9 * n_good * N / 1e12, "TFLOP/s", "alu", alu, alu_basis
    elif name == "tensor_gtable":
        # G~ and V written once per reference pixel and frame (2 x element size), the reference read
        es = 4 if form == 2 else 2
        work, unit, bound = (2.0 * es * R * N + 8.0 * R) / 1e9, "GB/s", "hbm"
        peak, pb = float(pk["hbm_gbs"]), f"{basis} HBM copy bandwidth"
    elif name == "tensor_prep":
        es = 4 if form == 2 else 2
        work, unit, bound = (4.0 * N * P + es * N * P + 5.0 * P) / 1e9, "GB/s", "hbm"
        peak, pb = float(pk["hbm_gbs"]), f"{basis} HBM copy bandwidth"
    elif name == "integrate":
        # per pixel and conjugate-gradient step: the 5-point normal operator (5 flop), three
        # vector updates and two dot products (2 flop each)
        work = 17.0 * n_good * max(extra.get("integ_steps", 0), 1) / 1e12
        unit, bound, peak, pb = "TFLOP/s", "fp64", fp64, fp64_basis
    elif name == "filter_map":
        # per good pixel: two passes of 2r + 1 taps, 3 FMA each
        work = 12.0 * (2 * extra.get("filter_r", 4) + 1) * n_good / 1e12
        unit, bound, peak, pb = "TFLOP/s", "fp64", fp64, fp64_basis
    elif name == "update_translations":
        # per pixel, frame and shift: the masked bilinear read (4 FMA) and the squared,
        # normalised residual added to the shift's sum (2 FMA)
        ty, tx = extra.get("tw") or (1, 1)
        work = 12.0 * N * n_good * (2 * ty + 1) * (2 * tx + 1) / 1e12
        unit, bound, peak, pb = "TFLOP/s", "alu", alu, alu_basis
    elif name == "calc_error":
        # frames read twice (var(x), then the errors), the map, W, M, var and the pixel error per
        # pixel, the reference-plane sums and error per reference pixel
        work, unit, bound = (8.0 * N * P + 33.0 * P + 12.0 * R) / 1e9, "GB/s", "hbm"
        peak, pb = float(pk["hbm_gbs"]), f"{basis} HBM copy bandwidth"
    else:
        # make_object_map: frames once, the map, W and M per pixel, FP64 flush and the outputs
        work, unit, bound = (4.0 * N * P + 21.0 * P + 32.0 * R) / 1e9, "GB/s", "hbm"
        peak, pb = float(pk["hbm_gbs"]), f"{basis} HBM copy bandwidth"
    achieved = work / (avg_ms * 1e-3)
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "kernel": name, "avg_launch_ms": avg_ms, "peak_basis": pb}


def time_form(args, s, base, u0, form_name, dist, world, orc, sampler):
    """Autotune, warm up and time one arithmetic form on the device-resident scan; then the
    same steps end to end from pinned host buffers. A step is one main-loop iteration
    (make_object_map, update_pixel_map) from the initial map u0."""
    import torch
    import paper_2003_12726_gb300 as px
    form = FORMS[form_name]
    rec = px.Reconstruction.from_device(base.frames, base.W, base.M, base.delta, u0, s.ref_shape, s.window,
                                        form=form)
    stream = torch.cuda.current_stream()
    tuned = None
    if not args.no_autotune:
        rec.run(1)                       # a reference image to search against; the map is restored
        tile, tms = px.autotune(rec, trials=3)
        tuned = {"tile": tile, "update_ms": tms}

    # the paper's full iteration adds the map filter, the translation update (iii) and the
    # figures of merit (iv); --frac replaces the 3x3 fit by fractional candidates
    full, frac = args.loop == "full", args.frac
    delta0 = rec.delta.clone()
    tw, integ = None, [None]
    if full:
        tw = (0, 2) if s.window[0] <= 1 else (1, 1)
        pe_t = torch.empty((rec.dims.ny, rec.dims.nx), dtype=torch.float32, device="cuda")
        fe_t = torch.empty(rec.dims.n_frames, dtype=torch.float64, device="cuda")
        tot_t = torch.empty(1, dtype=torch.float64, device="cuda")
        re_t = torch.empty(tuple(s.ref_shape), dtype=torch.float32, device="cuda")

    def step():
        rec.u.copy_(u0)
        if full:
            rec.delta.copy_(delta0)
        if frac:
            px.make_object_map(rec.dims, rec.frames, rec.W, rec.M, rec.u, rec.delta, rec.I_ref, rec.w, rec.ws)
            px.update_pixel_map_fractional(rec.dims, rec.opts, frac, rec.frames, rec.W, rec.M, rec.I_ref, rec.w,
                                           rec.delta, rec.u, rec.ws, rec.err)
        else:
            rec.run(1)
        if full:
            px.filter_map(rec.dims, 1.0, rec.M, rec.u, rec.ws)
            integ[0] = px.integrate_map(rec.dims, rec.M, rec.u, rec.ws, max_iter=200, tol=1e-8)
            px.update_translations(rec.dims, tw, rec.frames, rec.W, rec.M, rec.I_ref, rec.w, rec.u, rec.delta,
                                   rec.ws, fe_t)
            px.calc_error(rec.dims, rec.frames, rec.W, rec.M, rec.I_ref, rec.w, rec.u, rec.delta, rec.ws, pe_t,
                          fe_t, tot_t, re_t)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    code, bits = px.get_status(rec.ws)
    if code != 0:
        raise RuntimeError(f"{form_name}: device status {code} bits {bits}")

    # ---- device-resident timed region -----------------------------------------------------
    px.timing_enable(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = px.launch_count()
    t_wall0 = time.time()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall1 = time.time()
    launches = px.launch_count() - n0
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    ktimes = px.timing_read()
    px.timing_enable(False)
    n_exact = px.last_exact_count(rec.ws)
    code, bits = px.get_status(rec.ws)
    if code != 0:
        raise RuntimeError(f"{form_name}: device status {code} bits {bits} after the timed steps")

    rec.delta.copy_(delta0)
    sweep = None
    if full:
        # initialisation: fit_defocus_registration over 5 x 5 map scales (timed once, warm)
        sc = [0.96, 0.98, 1.0, 1.02, 1.04]
        Ib, wb = torch.empty_like(rec.I_ref), torch.empty_like(rec.w)
        px.defocus_sweep(rec.dims, rec.frames, rec.W, rec.M, u0, rec.delta, sc, sc, Ib, wb, rec.ws)
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        cmap = px.defocus_sweep(rec.dims, rec.frames, rec.W, rec.M, u0, rec.delta, sc, sc, Ib, wb, rec.ws)
        d1.record(stream)
        torch.cuda.synchronize()
        best = divmod(int(torch.argmax(cmap).item()), len(sc))
        sweep = {"pairs": len(sc) ** 2, "ms": d0.elapsed_time(d1), "best_scales": [sc[best[0]], sc[best[1]]]}

    # ---- the configuration's 10 iterations in one pxst_iterate call ------------------------
    rec.u.copy_(u0)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    rec.run(s.n_iter)
    g1.record(stream)
    torch.cuda.synchronize()
    ms_iter10 = g0.elapsed_time(g1) / s.n_iter

    # ---- end to end through the public API with pinned host buffers ------------------------
    pinned = rec.pin_host_buffers(s.frames, s.W, s.M, s.delta, s.u_init)
    hs = px.HostStream(rec, pinned)
    h2d, d2h = hs.run(2)
    hs.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(hs.copy)
    hs.compute.wait_stream(hs.copy)
    ev_steps = []
    for _ in range(args.steps):
        hs.run(1)
        ev_steps.append(torch.cuda.Event(enable_timing=True))
        ev_steps[-1].record(hs.compute)
    f1.record(hs.compute)
    hs.synchronize()
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(f0.elapsed_time(f1), dist, "cuda")
    # what bounds it: each step's completion interval, and the inputs' host-to-device copy
    # alone (no compute beside it)
    e2e_steps = [f0.elapsed_time(ev_steps[0])] + [ev_steps[k - 1].elapsed_time(ev_steps[k])
                                                  for k in range(1, len(ev_steps))]
    h2d_alone = []
    for _ in range(3):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(hs.copy)
        with torch.cuda.stream(hs.copy):
            for key in ("frames", "W", "M", "delta", "u"):
                hs.bufs[1][key].copy_(pinned[key], non_blocking=True)
        c1.record(hs.copy)
        c1.synchronize()
        h2d_alone.append(c0.elapsed_time(c1))
    hs = None

    # ---- accuracy on the oracle's stripes: both sides search the oracle's reference --------
    acc = None
    if orc is not None:
        Id = torch.as_tensor(orc["I32"]).cuda()
        wd = torch.as_tensor(orc["w32"]).cuda()
        out = {}
        for q in (False, True):
            o = px.Options(s.window[0], s.window[1], q, form, tile=rec.opts.tile)
            ud = u0.clone()
            err = torch.empty((rec.dims.ny, rec.dims.nx), dtype=torch.float32, device="cuda")
            px.update_pixel_map(rec.dims, o, rec.frames, rec.W, rec.M, Id, wd, rec.delta, ud, err, rec.ws)
            code, bits = px.get_status(rec.ws)
            if code != 0:
                raise RuntimeError(f"{form_name}: device status {code} bits {bits} in the accuracy run")
            out[q] = (ud.cpu().numpy(), err.cpu().numpy().astype(np.float64))
        acc = accuracy(s, orc, out[False][0], out[False][1], out[True][0])
    res = {"ms_per_step": ms / args.steps, "ms_per_iteration_10": ms_iter10, "tuned": tuned,
           "ktimes": ktimes, "launches": launches, "exact_pixels": n_exact, "e2e_ms": ms_e2e / args.steps,
           "e2e_steps_ms": e2e_steps, "h2d_alone_ms": float(np.median(h2d_alone)),
           "h2d": h2d, "d2h": d2h, "t_wall": (t_wall0, t_wall1), "accuracy": acc, "sweep": sweep,
           "extra": {"tw": tw, "filter_r": 4,
                     "integ_steps": int(integ[0][0].item()) if integ[0] is not None else 0}}
    del rec
    torch.cuda.empty_cache()
    return res


def full_loop_entry(r, s, ev_step, form, pk, basis, sms, sm_mhz, sampler=None):
    """The full-iteration run of time_form (loop = full) as an entry of the bench line: per
    kernel group its average time per launch and roofline, the dominant group, the launches."""
    kt = {k: (v[1] / v[0] if v[0] else 0.0) for k, v in r["ktimes"].items() if v[0]}
    roofs = {k: kernel_roofline(k, kt[k], s, ev_step, FORMS[form], pk, basis, sms, sm_mhz, r.get("extra"))
             for k in kt if k not in ("prepare", "omap_normalise", "upm_exact")}
    dom = max(kt, key=lambda k: kt[k] * r["ktimes"][k][0])
    extra = r.get("extra") or {}
    return {"form": form, "ms_per_step": r["ms_per_step"], "steps": 5, "warmup": 3,
            "step": "one full iteration from the scan's initial map and translations: reference image, pixel map "
                    "(3x3 fit), map filter (sigma 1), integration (at most 200 conjugate-gradient steps, tolerance "
                    "1e-8), translation update, figures of merit",
            "translation_window": list(extra.get("tw") or ()), "integrate_steps": extra.get("integ_steps"),
            "dominant_kernel": dom, "roofline": roofs.get(dom), "kernel_ms": kt, "kernel_rooflines": roofs,
            "gpu_launches": r["launches"], "defocus_sweep": r.get("sweep"),
            "clocks": sampler.summary(r["t_wall"][0] - 0.2, r["t_wall"][1] + 0.2) if sampler else None}


def pxst_arm(args, rank, world, local_rank):
    import torch
    import paper_2003_12726_gb300 as px

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    s = make_workload(args.workload, rank)
    ev_step = evals_per_step(s)
    forms = ["fp32", "bf16", "tf32"] if args.form == "all" else [args.form]
    headline = "bf16" if "bf16" in forms else forms[0]
    # the scan's inputs stay resident; every form runs on the same device arrays
    base = px.Reconstruction(s.frames, s.W, s.M, s.delta, s.u_init, s.ref_shape, s.window)
    u0 = base.u.clone()
    orc = None
    if world == 1 and not args.no_cpu_baseline:
        orc = oracle_leg(s)
    sampler = ClockSampler(local_rank) if rank == 0 else None
    iref_err = None
    if orc is not None:
        # the reference image of the first iteration (the same kernels serve every form)
        Ig = torch.empty(tuple(s.ref_shape), dtype=torch.float32, device="cuda")
        wg = torch.empty_like(Ig)
        px.make_object_map(base.dims, base.frames, base.W, base.M, u0, base.delta, Ig, wg, base.ws)
        Ig, wg = Ig.cpu().numpy().astype(np.float64), wg.cpu().numpy().astype(np.float64)
        sel = orc["wo"] > 1e-4 * orc["wo"].max()
        rl2 = lambda a, b: float(np.sqrt(np.sum((a - b) ** 2) / max(np.sum(b ** 2), 1e-300)))
        iref_err = {"iref_rel_l2": rl2(Ig[sel], orc["Io"][sel]), "w_rel_l2": rl2(wg, orc["wo"]),
                    "coverage_mismatch": int(np.count_nonzero((wg > 0) != (orc["wo"] > 0))),
                    "over": "reference pixels with oracle weight > 1e-4 max (I_ref); all (w)"}
    results = {f: time_form(args, s, base, u0, f, dist, world, orc, sampler) for f in forms}
    # the paper's full iteration in the headline form, beside the main-loop line (one GPU)
    full = None
    if world == 1 and args.form == "all" and args.loop == "main" and not args.frac and not args.no_full_loop:
        fa = argparse.Namespace(**vars(args))
        fa.loop, fa.steps, fa.warmup, fa.no_autotune = "full", 5, 3, True
        full = time_form(fa, s, base, u0, headline, dist, world, None, sampler)
    if sampler:
        sampler.stop()
    # the batched and served workloads of the same run (one GPU, the default line only)
    batch = serve = None
    if world == 1 and args.form == "all" and args.workload == "precision2d" and not args.no_extra:
        del base
        torch.cuda.empty_cache()
        batch = run_batch(FORMS["bf16"], steps=5, warmup=3)
        batch.pop("_scans")
        torch.cuda.empty_cache()
        pool = ServePool()
        serve = {}
        for fname, n_req in (("bf16", 120), ("fp32", 60)):
            cap = run_serve(FORMS[fname], pool, n_req, 0.0, args.mem_gb, realtime=False)
            sub = run_serve(FORMS[fname], pool, n_req, 0.5 * cap["scans_per_s"], args.mem_gb, realtime=True,
                            seed_offset=45)
            serve[fname] = {"capacity": cap, "half_capacity": sub}
        del pool
        torch.cuda.empty_cache()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    pk, basis = peaks()
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    per_form = {}
    for f, r in results.items():
        kt = {k: (v[1] / v[0] if v[0] else 0.0) for k, v in r["ktimes"].items() if v[0]}
        roofs = {k: kernel_roofline(k, kt[k], s, ev_step, FORMS[f], pk, basis, sms, sm_mhz, r.get("extra"))
                 for k in kt if k not in ("prepare", "omap_normalise", "upm_exact")}
        dom = max(kt, key=lambda k: kt[k] * r["ktimes"][k][0])
        roofs[dom]["traffic"] = load_traffic(args.workload + ("" if f == "fp32" else "-" + f), dom)
        clocks = sampler.summary(r["t_wall"][0] - 0.2, r["t_wall"][1] + 0.2) if sampler else None
        per_form[f] = {"ms_per_step": r["ms_per_step"], "value": job_rate(ev_step, world, r["ms_per_step"], 1),
                       "ms_per_iteration_of_10": r["ms_per_iteration_10"],
                       "e2e": {"value": job_rate(ev_step, world, r["e2e_ms"], 1), "ms_per_step": r["e2e_ms"]},
                       "dominant_kernel": dom, "roofline": roofs[dom], "kernel_rooflines": roofs,
                       "kernel_ms": kt, "gpu_launches": r["launches"], "autotuned": r["tuned"],
                       "exact_path_pixels": r["exact_pixels"], "accuracy_vs_oracle": r["accuracy"],
                       "clocks": clocks}
        if r["sweep"]:
            per_form[f]["defocus_sweep"] = r["sweep"]
    h = per_form[headline]
    rh = results[headline]
    cpu = None
    if orc is not None:
        cpu = {"value": orc["rate"], "unit": UNIT, "cores": orc["threads"], "kind": "oracle", "sample": orc["sample"]}
    clocks = sampler.summary(min(r["t_wall"][0] for r in results.values()) - 0.2,
                             max(r["t_wall"][1] for r in results.values()) + 0.2) if sampler else None
    dt = {"fp32": "f32", "bf16": "bf16/f32", "tf32": "tf32/f32"}
    line = {"metric": METRIC, "value": h["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dt[headline], "data": "synthetic",
            "config": {"workload": s.name, "frames": int(s.frames.shape[0]), "detector": list(s.frames.shape[1:]),
                       "window": list(s.window), "reference": list(s.ref_shape), "form": headline,
                       "forms_timed": forms, "quadratic": True, "evals_per_step": ev_step,
                       "parallelism": f"replicas{world}",
                       "step": "one main-loop iteration (make_object_map, update_pixel_map with the 3x3 fit) from "
                               "the scan's initial map, restored on the device before each step",
                       "subpixel": f"fractional candidates, 1/{args.frac} grid" if args.frac else "3x3 paraboloid",
                       "loop": "full: reference image, pixel map, map filter (sigma 1), integration (at most 200 "
                               "conjugate-gradient steps, tolerance 1e-8), translations, figures of merit"
                               if args.loop == "full" else "reference image, pixel map",
                       "l2": f"inputs larger than L2 (frames {s.frames.nbytes / 1e6:.0f} MB per step)"},
            "roofline": h["roofline"], "cpu_baseline": cpu,
            "e2e": {"value": h["e2e"]["value"], "unit": UNIT, "h2d_bytes_per_step": rh["h2d"],
                    "d2h_bytes_per_step": rh["d2h"], "ms_per_step": h["e2e"]["ms_per_step"],
                    "step_ms": [round(x, 3) for x in rh["e2e_steps_ms"]], "h2d_alone_ms": rh["h2d_alone_ms"],
                    "api": "HostStream: every step copies the frames, whitefield, mask, translations and initial "
                           "map from pinned host memory, runs pxst_iterate for one iteration and copies the map and "
                           "error back; the next step's copy overlaps this step's compute"},
            "gpu_launches": h["gpu_launches"], "kernel_ms": h["kernel_ms"], "exact_path_pixels": h["exact_path_pixels"],
            "forms": per_form, "iref_error_vs_oracle": iref_err, "clocks": clocks}
    if full:
        line["full_loop"] = full_loop_entry(full, s, ev_step, headline, pk, basis, sms, sm_mhz, sampler)
    if batch:
        line["batch64"] = dict(batch, form="bf16", workload="64 scans of the batched configuration")
    if serve:
        line["serve"] = dict(serve, workload="Poisson stream, sizes log-uniform between the small configuration and "
                                              "the 2-D precision scan, 1-D or 2-D, 10 iterations each; capacity: every "
                                              "request at t = 0; half_capacity: arrivals at half that rate")
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _host_scan(sc):
    """A GPU-rendered scan as host arrays (for the oracle's timed sample)."""
    from types import SimpleNamespace
    return SimpleNamespace(name=sc.name, frames=sc.frames.cpu().numpy(), W=sc.W.cpu().numpy(), M=sc.M.cpu().numpy(),
                           u_init=sc.u_init.cpu().numpy(), delta=sc.delta.cpu().numpy(), ref_shape=sc.ref_shape,
                           window=sc.window)


def run_batch(form, steps, warmup, branches=8, n_scans=64):
    """The batched workload: 64 scans of uneven size (frames U[16, 400], sides U[128, 1024],
    windows U{4..16}) iterated together; a step is one iteration of every scan, one graph
    launch of pxst_batch_run. Tile shapes come from the autotuner. Returns a summary dict."""
    import torch
    import gen.gpu as gg
    import paper_2003_12726_gb300 as px
    specs = gg.batch_specs(n_scans)
    scans = [gg.render(sp) for sp in specs]
    torch.cuda.synchronize()
    recs = [px.Reconstruction.from_device(sc.frames, sc.W, sc.M, sc.delta, sc.u_init, sc.ref_shape, sc.window,
                                          form=form) for sc in scans]
    ev_step = sum(sc.evals for sc in scans)
    t_plan = time.time()
    b = px.Batch(recs, n_iter=1, n_branches=branches, autotune=True)
    t_plan = time.time() - t_plan
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    for _ in range(warmup):
        b.run()
    torch.cuda.synchronize()
    for r in recs:
        code, bits = px.get_status(r.ws)
        if code != 0:
            raise RuntimeError(f"device status {code} bits {bits}")
    torch.cuda.synchronize()
    t_wall0 = time.time()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        b.run()
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    ms = e0.elapsed_time(e1)
    sampler.stop()
    tiles = {}
    for r in recs:
        tiles[r.opts.tile] = tiles.get(r.opts.tile, 0) + 1
    out = {"value": ev_step / (ms / 1e3) * steps, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
           "scans": len(scans), "scan_iterations_per_s": len(scans) * steps / (ms / 1e3),
           "frames_range": [min(s.frames.shape[0] for s in scans), max(s.frames.shape[0] for s in scans)],
           "side_range": [min(s.frames.shape[1] for s in scans), max(s.frames.shape[1] for s in scans)],
           "window_range": [min(s.window[0] for s in scans), max(s.window[0] for s in scans)],
           "evals_per_step": ev_step, "branches": branches, "plan_s": t_plan,
           "tiles_chosen": {str(k): v for k, v in sorted(tiles.items())},
           "step": "one iteration of every scan: one cudaGraphLaunch of pxst_batch_run",
           "l2": f"inputs larger than L2 (frames {sum(s.frames.numel() for s in scans) * 4 / 1e9:.1f} GB)",
           "clocks": sampler.summary(t_wall0 - 0.2, t_wall1 + 0.2), "_scans": scans}
    b.close()
    return out


def batch_arm(args):
    form = FORMS[args.form]
    res = run_batch(form, args.steps, args.warmup, args.branches)
    scans = res.pop("_scans")
    cpu = None
    if not args.no_cpu_baseline:
        small = min(range(len(scans)), key=lambda k: scans[k].evals)
        rate, rows, sec, threads = cpu_sample(_host_scan(scans[small]), target_s=args.cpu_s)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{rows} detector rows of scan {scans[small].name}: make_object_map + update_pixel_map "
                         f"of the stripe, {sec:.1f} s"}
    line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {0: "f32", 1: "bf16/f32", 2: "tf32/f32"}[form],
            "data": "synthetic (rendered on the GPU)",
            "config": {"workload": "batch-64-scans", "form": args.form,
                       **{k: res[k] for k in ("scans", "frames_range", "side_range", "window_range", "evals_per_step",
                                               "branches", "tiles_chosen", "plan_s", "l2")},
                       "parallelism": "one graph launch per step"},
            "scan_iterations_per_s": res["scan_iterations_per_s"], "roofline": None, "cpu_baseline": cpu, "e2e": None,
            "gpu_launches": None, "clocks": res["clocks"]}
    print(json.dumps(line), flush=True)


class ServePool:
    """Host-resident scans for the served workload: the size parameter tau of the stream's
    log-uniform mix, binned to `levels` values, for each geometry, rendered once on the GPU
    and kept in pinned host memory; a request takes the template of its bin and geometry, and
    the server copies it to the device at admission (inside the request's latency)."""

    def __init__(self, levels=8, device="cuda"):
        import torch
        import gen.gpu as gg
        self.levels = levels
        self.tmpl = {}
        for kind in ("2d", "1d"):
            for k in range(levels):
                tau = k / (levels - 1)
                sp = self._spec(kind, tau, seed=12726 * 100 + k + (0 if kind == "2d" else 50))
                sc = gg.render(sp, device=device)
                pin = lambda t: t.cpu().pin_memory()
                self.tmpl[(kind, k)] = SimpleNamespace(frames=pin(sc.frames), W=pin(sc.W), M=pin(sc.M),
                                                       delta=pin(sc.delta), u_init=pin(sc.u_init),
                                                       ref_shape=sc.ref_shape, window=sc.window, spec=sp)
                del sc
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    @staticmethod
    def _spec(kind, tau, seed):
        frames = int(round(16 * 25 ** tau))
        side = int(round(64 * 16 ** tau))
        if kind == "2d":
            return dict(kind="2d", n_side=max(4, int(round(frames ** 0.5))), det=side, window=int(round(4 + 12 * tau)),
                        seed=seed)
        return dict(kind="1d", n_frames=frames, ny=max(16, side // 2), nx=max(96, (3 * side) // 2), seed=seed)

    def template(self, spec):
        # the bin of the spec's size parameter: 16 * 25^tau frames and 64 * 16^tau pixels
        import math
        if spec["kind"] == "2d":
            tau = math.log(max(spec["det"], 64) / 64.0) / math.log(16.0)
        else:
            tau = math.log(max(spec["nx"] * 2 // 3, 64) / 64.0) / math.log(16.0)
        k = min(self.levels - 1, max(0, int(round(tau * (self.levels - 1)))))
        return self.tmpl[(spec["kind"], k)]


def run_serve(form, pool, n_requests, rate, mem_gb, realtime=True, seed_offset=44):
    """The served workload: a Poisson stream (rate per second; realtime=False: every request
    arrives at once, so the throughput is the capacity) of scans drawn from the log-uniform
    mix between the small configuration and the 2-D precision scan, 10 iterations each,
    through the continuous-batching server with admission by device memory; each request's
    data is copied from pinned host memory at admission."""
    import gen.gpu as gg
    from paper_2003_12726_gb300.serve import Request, Server, estimate_bytes, poisson_arrivals
    specs = gg.serve_specs(n_requests)
    arr = poisson_arrivals(len(specs), rate, seed=gen.BASE_SEED + seed_offset) if realtime else [0.0] * len(specs)

    def reqs(sp_list, times):
        out = []
        for k, (sp, t) in enumerate(zip(sp_list, times)):
            tp = pool.template(sp)
            n, ny, nx = (int(v) for v in tp.frames.shape)
            dims = (n, ny, nx, int(tp.ref_shape[0]), int(tp.ref_shape[1]))
            out.append(Request(rid=k, arrival=float(t), make=(lambda tp=tp: tp),
                               est_bytes=estimate_bytes(dims, tp.window, form), n_iter=10, form=form))
        return out
    server = Server(mem_budget=int(mem_gb * (1 << 30)), n_streams=8, max_active=32)
    server.run(reqs(specs[:8], [0.0] * 8), realtime=False)          # warm-up
    sampler = ClockSampler(0)
    t_wall0 = time.time()
    R = reqs(specs, arr)
    st = server.run(R, realtime=realtime)
    t_wall1 = time.time()
    sampler.stop()
    h2d = sum(r.make().frames.numel() * 4 for r in R)
    return {"scans_per_s": st["scans_per_s"], "requests": len(R), "rate_per_s": rate if realtime else "all at t=0",
            "latency_s": {"p50": st["p50_s"], "p99": st["p99_s"], "mean": st["mean_s"]},
            "evals_per_s": st["evals_per_s"], "span_s": st["span_s"], "peak_active": st["peak_active"],
            "peak_bytes": st["peak_bytes"], "h2d_frame_bytes": h2d, "iterations": 10, "mem_budget_gb": mem_gb,
            "clocks": sampler.summary(t_wall0, t_wall1)}


def serve_arm(args):
    form = FORMS[args.form]
    pool = ServePool()
    st = run_serve(form, pool, args.requests, args.rate, args.mem_gb)
    line = {"metric": METRIC, "value": st["scans_per_s"], "unit": "scans/s", "n_gpus": 1, "steps": st["requests"],
            "warmup": 8, "ms_per_step": 1e3 / st["scans_per_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {0: "f32", 1: "bf16/f32", 2: "tf32/f32"}[form],
            "data": "synthetic (rendered once on the GPU, kept in pinned host memory, copied at admission)",
            "config": {"workload": f"serve-{st['requests']}-scans", "rate_per_s": args.rate, "iterations": 10,
                       "form": args.form, "mem_budget_gb": args.mem_gb, "streams": 8, "max_active": 32,
                       "parallelism": "continuous batching over streams"},
            "latency_s": st["latency_s"], "evals_per_s": st["evals_per_s"], "span_s": st["span_s"],
            "peak_active": st["peak_active"], "roofline": None, "cpu_baseline": None, "e2e": None,
            "gpu_launches": None, "clocks": st["clocks"]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="pxst", choices=["pxst", "reference"])
    ap.add_argument("--workload", default="precision2d", choices=sorted(WORKLOADS),
                    help="precision2d (the benchmark workload: the largest single-GPU scan) or another scan")
    ap.add_argument("--form", default="all", choices=["all"] + sorted(FORMS),
                    help="arithmetic of the candidate search: all three, fp32 (CUDA cores) or the tensor-core "
                         "bf16/tf32")
    ap.add_argument("--cpu-s", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-full-loop", action="store_true",
                    help="with --form all: skip the full-iteration run of the headline form")
    ap.add_argument("--no-extra", action="store_true",
                    help="default line without the batched and served workloads")
    ap.add_argument("--branches", type=int, default=8, help="batch64: parallel graph branches")
    ap.add_argument("--no-autotune", action="store_true", help="keep the automatic tile shape")
    ap.add_argument("--frac", type=int, default=0, help="fractional candidates on a 1/FRAC grid instead of the fit")
    ap.add_argument("--loop", default="main", choices=["main", "full"],
                    help="main: steps (i)+(ii) of the main loop; full: + translations and figures of merit")
    ap.add_argument("--requests", type=int, default=500, help="serve: number of scans")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: mean arrivals per second")
    ap.add_argument("--mem-gb", type=float, default=96.0, help="serve: device memory budget")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.form == "all" and args.workload in ("batch64", "serve"):
        args.form = "bf16"
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference" and args.workload in ("batch64", "serve"):
        ap.error("the reference arm times the oracle on the single-scan workloads")
    if args.impl == "reference":
        reference_arm(args, rank, world)
    elif args.workload == "batch64":
        batch_arm(args)
    elif args.workload == "serve":
        serve_arm(args)
    else:
        pxst_arm(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
