#!/usr/bin/env python
"""Throughput benchmark of the ray-tracing path on one GB300 per rank.

A step traces the 512^2 sweep of six images ({Einasto, cored-NFW, Kerr} x
inclination {17, 80} deg, spin 0.9, +-12 M, 4x4 refinement to 3 levels) in
one batched call: launch, Dormand-Prince integration, crossings, redshift,
intensity, refinement and assembly, all in the library's kernels.  The
headline value is geodesic rays integrated per second (base + refined rays),
whole job; images/s, the FP64 comparison and the roofline of the dominant
kernel (the persistent trace kernel) ride along.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank traces its own batch
(independent images, no collective on the data path); weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "geodesic rays/s & images/s at 512^2, mixed vs FP64 at <=1e-4 rel intensity err"
WORKLOAD = ("512x512 sweep: {Einasto lam_E=0.1, cored-NFW eta=0.02 lam_c=10, Kerr} x incl "
            "{17,80} deg, a=0.9, R_o=1000, +-12 M, 4x4 refinement x3 levels, thin disk from r_ISCO")
WORKLOAD_VOL = WORKLOAD.replace("thin disk from r_ISCO",
                                "volumetric layer from r_ISCO (Eqs. 83-88, H0=h=0.05)")
# Algorithmic FP64/FP32 operations per accepted Dormand-Prince step: six
# right-hand-side evaluations (84 each for the Kerr lapse, counted from the
# separated Hamilton equations) plus the stage combinations, the 5th-order
# update and the error norm (504).  Rejected steps are overhead and not
# counted; the Einasto / cored-NFW lapses add work that is not counted either.
FLOP_PER_STEP = 6 * 84 + 504
FP64_PEAK_FLOPS = 1.25e12          # GB300 nominal FP64 vector rate
KEYS_CAP = 1 << 23                 # refinement-pattern keys kept per image
# DRAM bytes (read + write) per bench step of each trace kernel's launches
# on the 512^2 six-image mixed thin-disk sweep, from one ncu capture of the
# current kernels (dram__bytes_read.sum + dram__bytes_write.sum over the
# kernel's launches of one plan launch); to be retaken whenever a trace kernel
# changes.  Not measured for the volumetric layer, which reports null.
TRAFFIC_PER_STEP = {"trace_fp64_kernel": 2.14e9, "trace_mixed_kernel": 2.15e9}
FP32_PEAK_FLOPS = 152 * 128 * 2 * 2.07e9   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None
        self.first = 0

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi takes a moment to start: wait (bounded) for its first
        # sample, then count only the samples taken after this point, i.e.
        # inside the timed region that follows
        t_end = time.time() + 5.0
        while not self.lines and time.time() < t_end and self.proc.poll() is None:
            time.sleep(0.01)
        self.first = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return summarise_clocks(self.lines[self.first:])


def summarise_clocks(lines):
    """Median SM clock, maximum clock and the throttle reasons seen in the
    nvidia-smi CSV lines (index, clocks.sm, clocks.max.sm, power.draw,
    active reasons, hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown,
    sw_power_cap); None without a sample."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def default_steps(workload: str) -> int:
    """Timed steps when --steps is not given: 5, or enough of the
    millisecond-long calls to last about a second (so that the clock sampler
    has samples inside the timed region)."""
    return {"vis1024": 1000, "viscurves": 300, "kerr64": 30}.get(workload, 5)


def aggregate_ranks(rays: float, ms: float, world: int, device):
    """Whole-job aggregation across ranks: the sum of the rays every rank
    traced and the longest rank's timed duration (the job ends with it)."""
    import torch
    import torch.distributed as dist
    tot = torch.tensor([float(rays), float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        r_sum = tot[0:1].clone()
        t_max = tot[1:2].clone()
        dist.all_reduce(r_sum, op=dist.ReduceOp.SUM)
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
        tot = torch.cat([r_sum, t_max])
    return float(tot[0]), float(tot[1])


def cpu_baseline(flats, seconds: float, seed: int = 7):
    """The oracle (plain FP64 C, OpenMP over pixels) on a bounded random sample
    of base pixels of the same images, each with its refinement subtree."""
    import numpy as np

    import oracle

    oracle.build()
    rng = np.random.default_rng(seed)
    rays, elapsed, pixels = 0, 0.0, 0
    t_end = time.time() + seconds
    while time.time() < t_end:
        for d in flats:
            P = oracle.problem(**{k: v for k, v in d.items() if k in oracle.DEFAULTS})
            ij = np.stack([rng.integers(0, d["nx"], 16), rng.integers(0, d["ny"], 16)], 1)
            t0 = time.perf_counter()
            r = oracle.trace_pixels(P, ij)
            elapsed += time.perf_counter() - t0
            rays += int(r["rays"].sum())
            pixels += len(ij)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": rays / elapsed, "unit": "rays/s", "cores": cores, "kind": "oracle",
            "sample": f"{pixels} random base pixels (16 per image per round, {len(flats)} images) with "
                      f"their on-screen neighbours and refinement subtrees, {rays} rays, "
                      f"{elapsed:.1f} s of oracle time"}


METRIC_SWEEP96 = "images/s, 96-image sweep at 256^2 (batched, graph-captured) vs single-image FP64"
WORKLOAD_SWEEP96 = ("96 images: {Kerr, Einasto lam_E=0.1, cored-NFW eta=0.02 lam_c=10} x a in "
                    "{0,0.3,0.5,0.7,0.8,0.9,0.94,0.98} x incl {17,30,50,80} deg, halo x U(0.8,1.2) "
                    "(seed 20260513), 256^2 over +-12 M, 4x4 refinement x3 levels")
METRIC_VIS = "visibilities/s, 1024^2 image x 65536 baselines (Eq. 108), split BF16 tensor cores"
WORKLOAD_VIS = ("1024^2 cored-NFW a=0.94 incl 17 deg +-12 M refined image; 65536 (u,v) with "
                "|b| ~ U(0,15) G-lambda, PA ~ U(0,pi), theta_g = 3.8 uas (seed 20260515)")


def _events_ms(stream, fn, reps):
    import torch
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(reps):
        fn()
    t1.record(stream)
    t1.synchronize()
    return t0.elapsed_time(t1) / reps


def _compare_images(a, b):
    """Intensity error of a against b relative to b's maximum over pixels
    whose class and refinement depth agree."""
    import torch
    same = ((a["status"] == b["status"]) & (a["ncross"] == b["ncross"]) &
            (a["refine_level"] == b["refine_level"]))
    d = (a["I"].double() - b["I"].double()).abs() / b["I"].double().abs().max()
    return (float(d[same].max()), float(torch.quantile(d.flatten()[::7], 0.999)),
            int((~same).sum()))


def _subtree_changed(a, b, nx, ny):
    """Pixels whose set of refined cells differs between two outputs."""
    import numpy as np
    ka = a["refine_keys"][: int(a["refine_keys_count"][0])].cpu().numpy()
    kb = b["refine_keys"][: int(b["refine_keys_count"][0])].cpu().numpy()
    diff = np.setxor1d(ka, kb)
    mask = np.zeros(nx * ny, dtype=bool)
    mask[np.unique(diff >> 16)] = True
    return mask.reshape(ny, nx)


def _run_plan_once(B, flats, dev, stream):
    """One launch of a plan over ``flats``: (plan, stats, seconds)."""
    import torch
    plan = B.Plan([B.from_flat(d) for d in flats], device=dev, keys_cap=KEYS_CAP)
    with torch.cuda.stream(stream):
        torch.cuda.synchronize(dev)
        c0 = time.perf_counter()
        plan.launch(stream=stream)
        st = plan.stats(stream)
        c1 = time.perf_counter()
    plan.check(stream)
    return plan, st, c1 - c0


def compare_with_fp64(B, workloads, flats, plan, dev, stream, value, mixed_s_per_step):
    """The mixed images against the all-FP64 path at its own tolerance (rtol
    1e-10), pixel by pixel over every pixel of every image: the intensity
    error relative to each image's maximum with no pixel exempt
    (``within_bar``: all pixels within 1e-4), the pixels whose base class,
    refinement depth or refined subtree differ (counted), and the two speed
    ratios: against FP64 at rtol 1e-10 (precision and tolerance together) and
    against FP64 at the mixed path's own tolerances (precision alone)."""
    import torch
    rp, st, s64 = _run_plan_once(B, [dict(d, **workloads.FP64_INTEG) for d in flats], dev, stream)
    errs, p999, p9999, over, cls_changed, tree_changed, total = [], [], [], 0, 0, 0, 0
    worst = None
    for img, (a, b) in enumerate(zip(plan.outputs, rp.outputs)):
        same = ((a["status"] == b["status"]) & (a["ncross"] == b["ncross"]) &
                (a["refine_level"] == b["refine_level"]))
        tree = same & ~torch.from_numpy(_subtree_changed(a, b, flats[img]["nx"],
                                                         flats[img]["ny"])).to(same.device)
        d = (a["I"].double() - b["I"].double()).abs() / b["I"].double().abs().max()
        k = int(torch.argmax(d))
        jj, ii = divmod(k, d.shape[1])
        if worst is None or float(d.flatten()[k]) > worst["err"]:
            worst = {"err": float(d.flatten()[k]), "image": img, "i": ii, "j": jj,
                     "I_mixed": float(a["I"][jj, ii]), "I_fp64": float(b["I"][jj, ii]),
                     "ncross": int(b["ncross"][jj, ii]), "status": int(b["status"][jj, ii]),
                     "level": int(b["refine_level"][jj, ii]),
                     "class_or_depth_changed": bool(not same[jj, ii]),
                     "subtree_changed": bool(same[jj, ii] and not tree[jj, ii])}
        errs.append(float(d.max()))
        over += int((d > 1e-4).sum())
        flat = d.flatten()
        p999.append(float(torch.quantile(flat[::3], 0.999)))
        p9999.append(float(torch.quantile(flat[::3], 0.9999)))
        cls_changed += int((~same).sum())
        tree_changed += int((same & ~tree).sum())
        total += same.numel()
    fp64_rate = sum(st["rays"]) / s64
    rp.close()
    # FP64 at the mixed path's own tolerances: the same images with only the
    # arithmetic precision changed
    mp, mst, s64m = _run_plan_once(B, [dict(d, precision=0) for d in flats], dev, stream)
    mp.close()
    return {"fp64_rtol": workloads.FP64_INTEG["rtol"], "fp64_rays_per_s": fp64_rate,
            "fp64_s_per_step": s64, "mixed_over_fp64": value / fp64_rate,
            "fp64_at_mixed_tolerances_s_per_step": s64m,
            "mixed_over_fp64_same_tolerances": s64m / mixed_s_per_step,
            "within_bar": over == 0,
            "max_rel_intensity_err_vs_fp64": max(errs),
            "pixels_over_1e-4": over,
            "p99_9_rel_intensity_err_all_pixels": max(p999),
            "p99_99_rel_intensity_err_all_pixels": max(p9999),
            "pixels_with_class_or_depth_change": cls_changed,
            "pixels_with_refined_subtree_change": tree_changed, "pixels": total,
            "worst_pixel": worst}


def run_sweep96(args, B, workloads, dev, stream):
    """The 96-image sweep in one batched plan, autotuned and replayed as a
    CUDA graph; single-image FP64 tracing of a sample of the images is the
    comparison."""
    import torch
    prec = B.MIXED if args.precision == "mixed" else B.FP64
    base = workloads.sweep_96()
    flats = [dict(d, **(workloads.MIXED_INTEG if prec == B.MIXED else workloads.FP64_INTEG))
             for d in base]
    items = [B.from_flat(d) for d in flats]
    plan = B.Plan(items, device=dev)
    with torch.cuda.stream(stream):
        plan.launch(stream=stream)
        plan.check(stream)
        tune = plan.autotune(stream=stream) if args.autotune else None
        # one timed eager launch for the per-kernel split (roofline)
        plan.set_timing(True)
        plan.launch(stream=stream)
        st = plan.stats(stream)
        plan.set_timing(False)
        for _ in range(args.warmup):
            plan.launch(use_graph=True, stream=stream)
        plan.check(stream)
        sampler = ClockSampler(dev.index or 0)
        torch.cuda.synchronize(dev)
        sampler.start()
        ms = _events_ms(stream, lambda: plan.launch(use_graph=True, stream=stream), args.steps)
        clocks = sampler.stop()
        plan.check(stream)
        rays = sum(plan.stats(stream)["rays"])
    images_per_s = len(items) / (ms / 1e3)
    steps32, ms32 = st["accepted_fp32"], st["fp32_ms"]
    steps64, ms64 = st["accepted_fp64"], st["fp64_ms"]
    tot_ms = ms32 + ms64

    def roof(steps, kms, peak, kern, lanes):
        ach = steps * FLOP_PER_STEP / (kms / 1e3) / 1e12 if kms > 0 else 0.0
        return {"bound": "alu", "achieved": ach, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": ach * 1e12 / peak, "traffic": None, "kernel": kern,
                "kernel_share_of_step": kms / tot_ms if tot_ms > 0 else None,
                "accepted_steps": steps, "flop_per_accepted_step": FLOP_PER_STEP,
                "lane_util": st[lanes]}
    r64 = roof(steps64, ms64, FP64_PEAK_FLOPS, "trace_fp64_kernel", "lane_util_fp64")
    if prec == B.FP64:
        roofline = r64
    else:
        # the dominant trace kernel of the step, the other alongside
        r32 = roof(steps32, ms32, FP32_PEAK_FLOPS, "trace_mixed_kernel", "lane_util_fp32")
        roofline, other = (r64, r32) if ms64 >= ms32 else (r32, r64)
        roofline = dict(roofline, other_trace_kernel=other)
    # single-image FP64 tracing of a sample (one image per spin, all metrics)
    sample = list(range(0, len(base), 12))
    t_single, errs, p999, changed = [], [], [], 0
    for k in sample:
        it = B.from_flat(dict(base[k], **workloads.FP64_INTEG))
        with torch.cuda.stream(stream):
            torch.cuda.synchronize(dev)
            c0 = time.perf_counter()
            ref = B.trace_batch([it], device=dev, stream=stream)[0]
            torch.cuda.synchronize(dev)
            t_single.append(time.perf_counter() - c0)
        e, p, c = _compare_images(plan.outputs[k], ref)
        errs.append(e)
        p999.append(p)
        changed += c
    fp64_images_per_s = len(sample) / sum(t_single)
    line = {
        "metric": METRIC_SWEEP96, "value": images_per_s, "unit": "images/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == B.FP64 else "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_SWEEP96, "images": len(items), "nx": 256, "ny": 256,
                   "levels": 3, "precision": args.precision, "graph": True,
                   "autotuned": tune is not None,
                   "l2": "working set > L2 (refinement records ~GBs); no flush",
                   "parallelism": "dp1"},
        "rays_per_s": rays / (ms / 1e3), "rays_per_step": rays, "tune": tune,
        "roofline": roofline, "clocks": clocks, "gpu_launches": st["kernel_launches"],
        "compare": {"fp64_single_image_images_per_s": fp64_images_per_s,
                    "batched_over_fp64_single": images_per_s / fp64_images_per_s,
                    "sampled_images": sample,
                    "max_rel_intensity_err_vs_fp64": max(errs),
                    "p99_9_rel_intensity_err": max(p999),
                    "pixels_with_class_or_depth_change": changed},
    }
    print(json.dumps(line), flush=True)
    plan.close()


def run_vis1024(args, B, workloads, dev, stream):
    """Eq. (108) for 65,536 baselines of a traced 1024^2 image on the tensor
    cores (split BF16 and FP16), against the FP64 direct sum on a sample."""
    import numpy as np
    import torch
    flat = workloads.vis_1024()
    item = B.from_flat(flat)
    cam = item[1]
    with torch.cuda.stream(stream):
        I = B.trace_batch([item], device=dev, stream=stream)[0]["I"]
    K = 65536
    uv_np = workloads.uv_points(K, seed=20260515)
    uv = torch.from_numpy(uv_np).to(dev)
    imax = float(I.abs().max())
    vout = torch.empty(K, 2, dtype=torch.float64, device=dev)
    res = {}
    with torch.cuda.stream(stream):
        for mode, name in ((B.VIS_BF16, "bf16"), (B.VIS_FP16, "fp16")):
            def call():
                B.visibilities(I, cam, uv, mode=mode, image_max=imax, stream=stream, out=vout,
                               check=False)
            for _ in range(args.warmup):
                call()
            torch.cuda.synchronize(dev)
            sampler = ClockSampler(dev.index or 0)
            sampler.start()
            ms = _events_ms(stream, call, args.steps)
            clocks = sampler.stop()
            V = torch.view_as_complex(vout.clone())
            res[name] = {"ms": ms, "clocks": clocks, "V": V}
        ks = torch.arange(0, K, 16, device=dev)
        ref = B.visibilities_fp64(I, cam, uv[ks], stream=stream)
        torch.cuda.synchronize(dev)
        V0 = abs(complex(B.visibilities_fp64(I, cam, torch.zeros(1, 2, dtype=torch.float64,
                                                                  device=dev))[0]))
    n = flat["nx"]
    tc_flop = 3 * 4.0 * n * n * K        # three split products of the two real GEMMs
    alg_flop = 4.0 * n * n * K
    ms = res["bf16"]["ms"]
    errs = {k: float((v["V"][ks] - ref).abs().max() / V0) for k, v in res.items()}
    achieved = tc_flop / (ms / 1e3) / 1e12
    peak = _measured_peak("bf16_tflops") or 1900.0
    # end to end: host image in, visibilities out, through the public call
    I_host = I.cpu().pin_memory()
    V_host = torch.empty(K, 2, dtype=torch.float64, pin_memory=True)
    with torch.cuda.stream(stream):
        torch.cuda.synchronize(dev)
        w0 = time.perf_counter()
        for _ in range(args.steps):
            Id = I_host.to(dev, non_blocking=True)
            B.visibilities(Id, cam, uv, mode=B.VIS_BF16, image_max=imax, stream=stream,
                           out=vout, check=False)
            V_host.copy_(vout, non_blocking=True)
            torch.cuda.synchronize(dev)
        w1 = time.perf_counter()
    e2e = {"value": K * args.steps / (w1 - w0), "unit": "visibilities/s",
           "h2d_bytes_per_step": I_host.numel() * 4, "d2h_bytes_per_step": K * 16}
    # oracle: the direct per-baseline sum on the host for a bounded sample
    from oracle.visibility import visibilities as vis_oracle
    Ih = I.double().cpu().numpy()
    c0 = time.perf_counter()
    kk = 0
    while time.perf_counter() - c0 < args.cpu_seconds and kk < K:
        vis_oracle(Ih, flat["x_min"], flat["x_max"], flat["y_min"], flat["y_max"], uv_np[kk:kk + 8])
        kk += 8
    cpu_s = time.perf_counter() - c0
    line = {
        "metric": METRIC_VIS, "value": K / (ms / 1e3), "unit": "visibilities/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3 split -> f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_VIS, "nx": n, "ny": n, "baselines": K,
                   "l2": "image 4 MB, phases generated on chip; inputs stay resident",
                   "parallelism": "dp1"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "vis_tc_kernel",
                     "tensor_flop_per_launch": tc_flop, "algorithmic_flop": alg_flop,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)"},
        "fp16_split": {"ms": res["fp16"]["ms"], "max_err_vs_fp64_over_V0": errs["fp16"]},
        "max_err_vs_fp64_over_V0": errs["bf16"], "fp64_sample": int(ks.numel()),
        "clocks": res["bf16"]["clocks"], "e2e": e2e,
        # per call: workspace header, image split, contraction
        "gpu_launches": 3 * args.steps,
        "cpu_baseline": {"value": kk / cpu_s, "unit": "visibilities/s", "cores": 1,
                         "kind": "oracle", "sample": f"{kk} baselines of the same image, numpy "
                         f"direct sum (Eq. 108), {cpu_s:.1f} s"},
    }
    print(json.dumps(line), flush=True)


METRIC_ADJ = "gradients/s of image loss w.r.t. 10 parameters at 256^2 (discrete adjoint)"
WORKLOAD_ADJ = ("{Kerr, cored-NFW eta=0.02 lam_c=10} a=0.7 incl 50 deg, 256^2 over +-12 M, one "
                "refinement level, FP64, R_in = R_+ + dR_in; loss = sum w I (w ~ N(0,1)) + "
                "diagnostics and 8 visibility amplitudes (uv seed 20260514)")


def run_adjoint(args, B, workloads, dev, stream):
    """One gradient of an image loss by the discrete adjoint, against the
    FP64 forward trace of the same image; the gradient against free central
    differences of the GPU FP64 forward image (the adaptive decisions are
    not frozen there, so agreement is to about the step-selection noise)."""
    import numpy as np
    import torch
    names = ["chi", "incl", "halo1", "halo2", "j0", "p", "R_s", "sigma_in", "sigma_out", "R_out"]
    flat_keys = {0: "chi", 1: "incl", 4: "j0", 5: "p", 6: "R_s", 7: "sigma_in", 8: "sigma_out",
                 9: "R_out"}
    uv8 = workloads.uv_points(8, seed=20260514)
    rows, times, fwd_times, clocks = [], [], [], []
    for metric in (workloads.KERR, workloads.CNFW):
        flat = dict(workloads.kerr_64(), metric=metric, chi=0.7, incl=math.radians(50.0), nx=256,
                    ny=256, x_min=-12.0, x_max=12.0, y_min=-12.0, y_max=12.0, levels=1,
                    r_in_mode=1, **workloads.HALO[metric])
        keys = dict(flat_keys)
        if metric == workloads.CNFW:
            keys.update({2: "eta", 3: "lam_c"})
        rng = np.random.default_rng(20260514 + metric)
        w = torch.from_numpy(rng.normal(size=(256, 256))).float().to(dev)
        st, cam, em, it = B.from_flat(flat)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                B.trace_backward(st, cam, em, it, dL_dI=w, stream=stream)
            torch.cuda.synchronize(dev)
            sampler = ClockSampler(dev.index or 0)
            sampler.start()
            res = {}

            def grad_call():
                res["g"] = B.trace_backward(st, cam, em, it, dL_dI=w, stream=stream)
            times.append(_events_ms(stream, grad_call, args.steps) / 1e3)
            clocks.append(sampler.stop())
            grad, diag, img = res["g"]

            def loss(d):
                out = B.trace_batch([B.from_flat(d)], device=dev, stream=stream)[0]
                return float((out["I"].double() * w.double()).sum())
            L0 = loss(flat)          # warm-up (workspace allocation)
            torch.cuda.synchronize(dev)
            f0 = time.perf_counter()
            for _ in range(3):
                L0 = loss(flat)
            torch.cuda.synchronize(dev)
            fwd_times.append((time.perf_counter() - f0) / 3)
            fd = {}
            for k, key in keys.items():
                x0 = flat[key]
                h = 1e-4 * max(abs(x0), 1.0)
                fd[names[k]] = (loss(dict(flat, **{key: x0 + h})) -
                                loss(dict(flat, **{key: x0 - h}))) / (2 * h)
        rel = {n: abs(grad[names.index(n)] - v) / max(abs(v), 1e-30) for n, v in fd.items()}
        rows.append({"metric": ["kerr", "einasto", "cnfw"][metric], "loss": L0,
                     "grad": {n: float(grad[i]) for i, n in enumerate(names)},
                     "free_fd": fd, "rel_err_vs_free_fd": rel,
                     "median_rel_err_vs_free_fd": float(np.median(list(rel.values())))})
    t = sum(times) / len(times)
    seen = [c for c in clocks if c]
    line = {
        "metric": METRIC_ADJ, "value": 1.0 / t, "unit": "gradients/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_ADJ, "nx": 256, "ny": 256, "levels": 1,
                   "parallelism": "dp1"},
        "forward_fp64_ms": 1e3 * sum(fwd_times) / len(fwd_times),
        "backward_over_forward": t / (sum(fwd_times) / len(fwd_times)),
        "per_metric": rows,
        "clocks": ({"sm_mhz": min(c["sm_mhz"] for c in seen),
                    "sm_max_mhz": max(c["sm_max_mhz"] for c in seen),
                    "reasons": sorted({x for c in seen for x in c["reasons"]}),
                    "samples": sum(c["samples"] for c in seen)} if seen else None),
        # per gradient: the forward plan (workspace header, level-0 and level-1
        # traces, refinement marking, assembly), image moments, radial
        # profile, per-pixel adjoint and the ray adjoint; both spacetimes
        "gpu_launches": 9 * args.steps * 2,
        "note": ("the adjoint differentiates the algorithm with its adaptive decisions frozen; "
                 "free differences of the pixel-sampled image also contain the motion of class "
                 "boundaries (shadow edge, photon-ring orders) across pixels, so they agree only "
                 "for parameters that move no boundary (the emissivity parameters); the "
                 "frozen-decision finite differences against the FP64 oracle are the parity "
                 "check (tests/test_gpu_adjoint.py)"),
    }
    print(json.dumps(line), flush=True)


METRIC_C1 = "geodesic rays/s, Kerr 64^2 parity case (FP64), with the oracle's time for the image"
WORKLOAD_C1 = ("Kerr a=0.5 incl 17 deg, R_o=1000, 64x64 cell-centred over [-10,10]^2, no "
               "refinement, FP64 rtol 1e-10 (the oracle-sized parity case)")


def run_kerr64(args, B, workloads, dev, stream):
    """The small parity case: one 64^2 Kerr image in FP64, timed on the GPU,
    and the whole image by the oracle on the host cores."""
    import torch

    import oracle
    flat = workloads.kerr_64()
    items = [B.from_flat(flat)]
    plan = B.Plan(items, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.launch(stream=stream)
        plan.check(stream)
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(dev.index or 0)
        sampler.start()
        ms = _events_ms(stream, lambda: plan.launch(stream=stream), args.steps)
        clocks = sampler.stop()
        st = plan.stats(stream)
    rays = sum(st["rays"])
    steps_acc = st["accepted_fp64"]
    plan.close()
    ach = steps_acc * FLOP_PER_STEP / (ms / 1e3) / 1e12
    oracle.build()
    P = oracle.problem(**{k: v for k, v in flat.items() if k in oracle.DEFAULTS})
    t0 = time.perf_counter()
    oracle.trace_image(P)
    t_or = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "metric": METRIC_C1, "value": rays / (ms / 1e3), "unit": "rays/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD_C1, "nx": 64, "ny": 64,
                                        "parallelism": "dp1"},
        "note": "4096 rays fill 3 % of the GPU's resident threads: a latency figure, not a "
                "throughput one",
        "cpu_baseline": {"value": rays / t_or, "unit": "rays/s", "cores": cores,
                         "kind": "oracle", "sample": f"the whole image, {t_or:.2f} s"},
        "oracle_seconds_for_image": t_or,
        "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_FLOPS / 1e12,
                     "unit": "TFLOP/s", "frac": ach * 1e12 / FP64_PEAK_FLOPS, "traffic": None,
                     "kernel": "trace_fp64_kernel", "flop_per_accepted_step": FLOP_PER_STEP,
                     "accepted_steps": steps_acc,
                     "peak_source": "nominal GB300 FP64 1.25 TFLOP/s"},
        "clocks": clocks, "gpu_launches": st["kernel_launches"] * args.steps,
    }
    print(json.dumps(line), flush=True)


METRIC_SHADOW = "shadow-boundary points/s (Fig. 5: 3 metrics x 4096 directions, b to 1e-10)"
WORKLOAD_SHADOW = ("Fig. 5 shadow boundaries: {Kerr, Einasto lam_E=0.3, cored-NFW eta=0.02 "
                   "lam_c=10} at a=0.5, incl 60 deg, R_o=1000; 4096 directions each, b in "
                   "[1, 9] bracketed to 1e-10, FP64 rtol 1e-10")


def run_shadow(args, B, workloads, dev, stream):
    """One step brackets the shadow boundary of the three Fig. 5 spacetimes
    along 4096 screen directions each (three calls on one stream)."""
    import numpy as np
    import torch

    import oracle
    flats, psi, lo, hi, tol = workloads.shadow_fig5()
    items = [B.from_flat(d) for d in flats]
    n = len(psi)
    psi_d = torch.tensor(psi, dtype=torch.float64, device=dev)
    stats = [torch.zeros(3, dtype=torch.int64, device=dev) for _ in items]
    res = [None] * len(items)

    def step():
        for i, (st, cam, _, it) in enumerate(items):
            res[i] = B.shadow_boundary(st, cam, it, psi_d, lo, hi, tol, device=dev, stream=stream,
                                       stats=stats[i])

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(dev.index or 0)
        sampler.start()
        ms = _events_ms(stream, step, args.steps)
        clocks = sampler.stop()
        counts = np.sum([s.cpu().numpy() for s in stats], axis=0)   # the last step's
        flags = np.concatenate([r[2].cpu().numpy() for r in res])
        b_in = [r[0].cpu().numpy() for r in res]
        b_out = [r[1].cpu().numpy() for r in res]
        # end to end: directions from pinned host memory, brackets back to the host
        psi_h = torch.tensor(psi, dtype=torch.float64).pin_memory()
        host = [torch.empty(n, dtype=torch.float64, pin_memory=True)
                for _ in range(2 * len(items))]
        torch.cuda.synchronize(dev)
        n_e2e = max(1, min(3, args.steps))
        w0 = time.perf_counter()
        for _ in range(n_e2e):
            pd = psi_h.to(dev, non_blocking=True)
            for i, (st, cam, _, it) in enumerate(items):
                bi, bo, _ = B.shadow_boundary(st, cam, it, pd, lo, hi, tol, device=dev,
                                              stream=stream)
                host[2 * i].copy_(bi, non_blocking=True)
                host[2 * i + 1].copy_(bo, non_blocking=True)
            torch.cuda.synchronize(dev)
        w1 = time.perf_counter()
    points = len(items) * n
    value = points / (ms / 1e3)
    ach = counts[1] * FLOP_PER_STEP / (ms / 1e3) / 1e12
    # the oracle's bisection on a bounded sample of the same directions
    oracle.build()
    rng = np.random.default_rng(7)
    t_end = time.time() + args.cpu_seconds
    cpu_pts, cpu_t, worst = 0, 0.0, 0.0
    while time.time() < t_end:
        for i, d in enumerate(flats):
            k = rng.choice(n, 8, replace=False)
            P = oracle.problem(**{kk: v for kk, v in d.items() if kk in oracle.DEFAULTS})
            t0 = time.perf_counter()
            r = oracle.shadow_boundary(P, np.asarray(psi)[k], lo, hi, tol)
            cpu_t += time.perf_counter() - t0
            cpu_pts += len(k)
            mid_o = 0.5 * (r["b_in"] + r["b_out"])
            mid_g = 0.5 * (b_in[i][k] + b_out[i][k])
            worst = max(worst, float(np.max(np.abs(mid_g - mid_o))))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "metric": METRIC_SHADOW, "value": value, "unit": "boundary points/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_SHADOW, "directions": n, "spacetimes": len(items),
                   "l2": "ALU-bound, ray state in registers, 32 KB of inputs; no flush",
                   "parallelism": "dp1"},
        "rays_per_step": int(counts[0]), "rays_per_s": counts[0] / (ms / 1e3),
        "accepted_steps_per_step": int(counts[1]),
        "flags_nonzero": int(np.count_nonzero(flags)),
        "max_abs_b_diff_vs_oracle_sample": worst,
        "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_FLOPS / 1e12,
                     "unit": "TFLOP/s", "frac": ach * 1e12 / FP64_PEAK_FLOPS, "traffic": None,
                     "kernel": "shadow_kernel", "flop_per_accepted_step": FLOP_PER_STEP,
                     "peak_source": "nominal GB300 FP64 1.25 TFLOP/s"},
        "cpu_baseline": {"value": cpu_pts / cpu_t, "unit": "boundary points/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{cpu_pts} random directions of the same three spacetimes "
                                   f"(bisection, 8 per spacetime per round), {cpu_t:.1f} s"},
        "clocks": clocks,
        "e2e": {"value": n_e2e * points / (w1 - w0), "unit": "boundary points/s",
                "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": 2 * points * 8},
        # per spacetime and step: workspace header and the boundary kernel
        "gpu_launches": 2 * len(items) * args.steps,
    }
    print(json.dumps(line), flush=True)


METRIC_SCAN = "spacetimes classified/s (Figs. 3-4 grids: horizon, extremal spin, 16-angle R_s)"
WORKLOAD_SCAN = ("Einasto (chi, lambda_E) in [0,1.2]x[0.05,1] and cored-NFW (chi, eta) in "
                 "[0,1.2]x[0,0.3] at lambda_c=10, 1024^2 each; R_+, chi_e, R_e and R_s at 16 "
                 "polar angles in [0, pi/2]")
# Hand count of FP64 operations per lapse evaluation R^2 H(R) in the scan
# (exp by reduction and a degree-13 polynomial, log1p by its atanh series,
# reciprocals by two Newton steps): Einasto 42, cored-NFW 66; the bench grid
# is half of each.
SCAN_FLOP_PER_EVAL = 54


def run_scan(args, B, workloads, dev, stream):
    """One step classifies the two Figs. 3-4 parameter grids (2 x 1024^2
    spacetimes) in one bh_geometry_scan call."""
    import numpy as np
    import torch

    import oracle
    metric, chi, lam_E, eta, lam_c, theta = workloads.geometry_grid()
    n = metric.shape[0]
    rec = np.zeros(n, dtype=np.dtype([("metric", "<i4"), ("reserved", "<i4"), ("chi", "<f8"),
                                      ("lambda_E", "<f8"), ("eta", "<f8"),
                                      ("lambda_c", "<f8")]))
    rec["metric"], rec["chi"], rec["lambda_E"], rec["eta"], rec["lambda_c"] = (
        metric, chi, lam_E, eta, lam_c)
    raw = rec.view(np.uint8)
    st_d = torch.from_numpy(raw.copy()).to(dev)
    stats = torch.zeros(2, dtype=torch.int64, device=dev)
    res = {}

    def step():
        res.update(B.geometry_scan(st_d, theta, device=dev, stream=stream, stats=stats))

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(dev.index or 0)
        sampler.start()
        ms = _events_ms(stream, step, args.steps)
        clocks = sampler.stop()
        evals = int(stats.sum())                     # the last step's
        out = {k: v.cpu().numpy() for k, v in res.items()}
        # end to end: parameters from pinned host memory, results back
        host_in = torch.from_numpy(raw.copy()).pin_memory()
        torch.cuda.synchronize(dev)
        n_e2e = max(1, min(3, args.steps))
        w0 = time.perf_counter()
        for _ in range(n_e2e):
            r = B.geometry_scan(host_in.to(dev, non_blocking=True), theta, device=dev,
                                stream=stream)
            {k: v.to("cpu", non_blocking=True) for k, v in r.items()}
            torch.cuda.synchronize(dev)
        w1 = time.perf_counter()
    value = n / (ms / 1e3)
    ach = evals * SCAN_FLOP_PER_EVAL / (ms / 1e3) / 1e12
    # the oracle (plain C scans at its own 1e-3 / 1e-4 grids) on a bounded sample
    oracle.build()
    rng = np.random.default_rng(11)
    t_end = time.time() + args.cpu_seconds
    cpu_n, cpu_t, worst = 0, 0.0, 0.0
    while time.time() < t_end:
        i = int(rng.integers(0, n))
        P = oracle.problem(metric=int(metric[i]), chi=float(chi[i]), lam_E=float(lam_E[i]),
                           eta=float(eta[i]), lam_c=float(lam_c[i]))
        t0 = time.perf_counter()
        ce, _ = oracle.extremal_spin(P)
        rp = oracle.horizon(P)
        rs = [oracle.ergosurface(P, float(t)) for t in theta]
        cpu_t += time.perf_counter() - t0
        cpu_n += 1
        # chi_e = 0 where -R^2 H never becomes positive (the oracle returns
        # round-off there): an absolute difference
        d = abs(out["chi_e"][i] - ce)
        worst = max(worst, d / ce if ce > 1e-8 else d)
        if rp is not None and abs(chi[i]) < ce - 1e-3:
            worst = max(worst, abs(out["r_plus"][i] - rp) / rp)
    line = {
        "metric": METRIC_SCAN, "value": value, "unit": "spacetimes/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_SCAN, "spacetimes": n, "angles": len(theta),
                   "l2": "ALU-bound; 84 MB of parameters read once per step, no flush",
                   "parallelism": "dp1"},
        "lapse_evaluations_per_step": evals,
        "black_holes": int(np.count_nonzero(out["flags"] == 0)),
        "max_rel_diff_vs_oracle_sample": worst,
        "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_FLOPS / 1e12,
                     "unit": "TFLOP/s", "frac": ach * 1e12 / FP64_PEAK_FLOPS, "traffic": None,
                     "kernel": "scan_kernel",
                     "flop_per_lapse_evaluation": SCAN_FLOP_PER_EVAL,
                     "peak_source": "nominal GB300 FP64 1.25 TFLOP/s"},
        "cpu_baseline": {"value": cpu_n / cpu_t, "unit": "spacetimes/s", "cores": 1,
                         "kind": "oracle",
                         "sample": f"{cpu_n} random grid points, one at a time (the oracle's "
                                   f"scans are serial), {cpu_t:.1f} s"},
        "clocks": clocks,
        "e2e": {"value": n_e2e * n / (w1 - w0), "unit": "spacetimes/s",
                "h2d_bytes_per_step": int(raw.nbytes),
                "d2h_bytes_per_step": int(n * (3 * 8 + 4 + 8 * len(theta)))},
        "gpu_launches": args.steps,  # one scan kernel per step
    }
    print(json.dumps(line), flush=True)


METRIC_VISCURVES = ("amplitude-curve points/s (Fig. 12: V(q) and the u cut, 256 q x 256 angles, "
                    "split BF16 tensor cores)")
WORKLOAD_VISCURVES = ("Fig. 12 images: {Kerr, Einasto lam_E=0.1, cored-NFW eta=0.02 lam_c=10} "
                      "at a=0.95, incl 70 deg, 1024^2 over +-12 M, 3 refinement levels (mixed "
                      "path); 256 radii q in (0, 0.5] cycles/M, 256 position angles each")


def run_viscurves(args, B, workloads, dev, stream):
    """Sec. 6.4's azimuthally averaged amplitude and horizontal cut of the three
    Fig. 12 images, 256 radii x 256 angles each, on the split BF16 tensor-core
    path; the FP64 direct mode on the same call is the accuracy reference."""
    import numpy as np
    import torch

    from oracle.visibility import amplitude_curves
    flats = workloads.fig12_images()
    items = [B.from_flat(d) for d in flats]
    with torch.cuda.stream(stream):
        imgs = [o["I"] for o in B.trace_batch(items, device=dev, stream=stream)]
    n_q, n_phi = 256, 256
    q = np.linspace(0.5 / n_q, 0.5, n_q)
    K = n_q * (n_phi + 1) + 1
    imax = [float(I.abs().max()) for I in imgs]
    out = [None] * len(imgs)

    def step():
        for i, I in enumerate(imgs):
            out[i] = B.visibility_curves(I, items[i][1], q, n_phi=n_phi, mode=B.VIS_BF16,
                                         image_max=imax[i], stream=stream, check=False)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(dev.index or 0)
        sampler.start()
        ms = _events_ms(stream, step, args.steps)
        clocks = sampler.stop()
        bf = [(a.cpu().numpy(), c.cpu().numpy()) for a, c in out]
        t0 = time.perf_counter()
        ref = [B.visibility_curves(I, items[i][1], q, n_phi=n_phi, mode=B.VIS_FP64,
                                   image_max=imax[i], stream=stream) for i, I in enumerate(imgs)]
        torch.cuda.synchronize(dev)
        fp64_s = time.perf_counter() - t0
        ref = [(a.cpu().numpy(), c.cpu().numpy()) for a, c in ref]
        # end to end: the images from pinned host memory, the curves back
        host = [I.cpu().pin_memory() for I in imgs]
        torch.cuda.synchronize(dev)
        n_e2e = max(1, min(3, args.steps))
        w0 = time.perf_counter()
        for _ in range(n_e2e):
            for i, h in enumerate(host):
                a, c = B.visibility_curves(h.to(dev, non_blocking=True), items[i][1], q,
                                           n_phi=n_phi, mode=B.VIS_BF16, image_max=imax[i],
                                           stream=stream, check=False)
                a.cpu(), c.cpu()
            torch.cuda.synchronize(dev)
        w1 = time.perf_counter()
    err = max(float(np.max(np.abs(b[0] - r[0]))) for b, r in zip(bf, ref))
    err_cut = max(float(np.max(np.abs(b[1] - r[1]))) for b, r in zip(bf, ref))
    n = flats[0]["nx"]
    tc_flop = len(imgs) * 3 * 4.0 * n * n * K     # three split products per image
    achieved = tc_flop / (ms / 1e3) / 1e12
    peak = _measured_peak("bf16_tflops") or 1900.0
    # the oracle's direct sums on a bounded sample: a few radii of one image
    I0 = imgs[0].double().cpu().numpy()
    g = flats[0]
    t_end = time.time() + args.cpu_seconds
    cpu_pts, cpu_t = 0, 0.0
    rng = np.random.default_rng(3)
    while time.time() < t_end:
        qs = q[rng.integers(0, n_q, 1)]
        t0 = time.perf_counter()
        amplitude_curves(I0, g["x_min"], g["x_max"], g["y_min"], g["y_max"], qs, 16)
        cpu_t += time.perf_counter() - t0
        cpu_pts += 17 / (n_phi + 1)      # 16 angles and the cut of one radius
    line = {
        "metric": METRIC_VISCURVES, "value": len(imgs) * n_q / (ms / 1e3),
        "unit": "curve points/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3 split, f32 accumulate", "data": "synthetic",
        "config": {"workload": WORKLOAD_VISCURVES, "images": len(imgs), "n_q": n_q,
                   "n_phi": n_phi, "baselines_per_image": K,
                   "l2": "images 4 MB each, re-read per 256-baseline tile; no flush",
                   "parallelism": "dp1"},
        "visibilities_per_s": len(imgs) * K / (ms / 1e3),
        "max_abs_err_avg_vs_fp64": err, "max_abs_err_cut_vs_fp64": err_cut,
        "fp64_direct_s_for_same_curves": fp64_s,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "vis_tc_kernel",
                     "tensor_flop_per_step": tc_flop,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)"},
        "cpu_baseline": {"value": cpu_pts / cpu_t, "unit": "curve points/s", "cores": 1,
                         "kind": "oracle",
                         "sample": f"direct FP64 sums (numpy) at random radii of the Kerr image, "
                                   f"16 angles + cut each, scaled to {n_phi} angles; "
                                   f"{cpu_t:.1f} s"},
        "clocks": clocks,
        "e2e": {"value": n_e2e * len(imgs) * n_q / (w1 - w0), "unit": "curve points/s",
                "h2d_bytes_per_step": int(len(imgs) * n * n * 4 + len(imgs) * n_q * 8),
                "d2h_bytes_per_step": int(len(imgs) * 2 * n_q * 8)},
        # per image and step: (u, v) set, header, image split, contraction, reduction
        "gpu_launches": 5 * len(imgs) * args.steps,
    }
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """One fixed case run a few times for profiling a kernel in isolation
    (``ncu ... python bench.py --profile-case CASE``); prints a one-line
    summary, no bench line.  Cases: ``kerr128`` (Kerr a = 0.5, i = 17 deg,
    128^2 over [-10, 10]^2, no refinement), ``sweep512`` (the first image of
    the 512^2 sweep, with refinement), ``sweep512l0`` (the same image without
    refinement), ``shadow512`` (the Fig. 5 cored-NFW shadow boundary along
    512 directions to 1e-10, FP64), ``scan64k`` (65,536 spacetimes of the
    Figs. 3-4 grids with 16 angles).  Tracing cases use the chosen
    precision's integrator settings."""
    import torch

    from paper_2605_05635_gb300 import bhrt, workloads
    case = args.profile_case
    if case == "shadow512":
        flats, psi, lo, hi, tol = workloads.shadow_fig5(512)
        st, cam, _, it = bhrt.from_flat(flats[2])
        for _ in range(args.repeat):
            b_in, b_out, fl = bhrt.shadow_boundary(st, cam, it, psi, lo, hi, tol)
        torch.cuda.synchronize()
        print(f"case shadow512: {int((fl != 0).sum())} flagged, mean b "
              f"{float((b_in + b_out).mean() / 2):.9f}")
        return 0
    if case == "scan64k":
        metric, chi, lam_E, eta, lam_c, theta = workloads.geometry_grid(256)
        sts = [bhrt.Spacetime(metric=int(metric[i]), chi=float(chi[i]),
                              lambda_E=float(lam_E[i]), eta=float(eta[i]),
                              lambda_c=float(lam_c[i])) for i in range(0, metric.shape[0], 2)]
        arr = bhrt.spacetime_array(sts)
        for _ in range(args.repeat):
            res = bhrt.geometry_scan(arr, theta)
        torch.cuda.synchronize()
        print(f"case scan64k: {len(sts)} spacetimes, {int((res['flags'] == 0).sum())} black holes")
        return 0
    prec = bhrt.FP64 if args.precision == "fp64" else bhrt.MIXED
    integ = workloads.FP64_INTEG if prec == bhrt.FP64 else workloads.MIXED_INTEG
    if case == "kerr128":
        flat = dict(workloads.kerr_64(), nx=128, ny=128, **integ)
    elif case in ("einasto128", "cnfw128"):
        # the same screen through the two halo metrics at a = 0.5, i = 17 deg
        metric = workloads.EINASTO if case == "einasto128" else workloads.CNFW
        flat = dict(workloads.kerr_64(), nx=128, ny=128, metric=metric, **workloads.HALO[metric],
                    **integ)
    else:
        flat = dict(workloads.sweep_512()[0], **integ)
        if case == "sweep512l0":
            flat["levels"] = 0
    plan = bhrt.Plan([bhrt.from_flat(flat)])
    for _ in range(args.repeat):
        plan.launch()
    torch.cuda.synchronize()
    plan.check()
    st = plan.stats()
    print(f"case {case} {args.precision} (last launch): rays {sum(st['rays'])} accepted fp32 "
          f"{st['accepted_fp32']} rejected fp32 {st['rejected_fp32']} fp64 "
          f"{st['accepted_fp64']} rejected fp64 {st['rejected_fp64']} promoted "
          f"{st['promoted_rays']} lane utilisation fp32 {st['lane_util_fp32']:.3f} "
          f"fp64 {st['lane_util_fp64']:.3f}")
    plan.close()
    return 0


def _measured_peak(key):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        v = d.get(key)
        return float(v) if v is not None else None
    except (OSError, ValueError, TypeError):
        return None


def run_reference(args, rank, world):
    """--impl reference: the oracle on the host cores, same metric/config."""
    if rank != 0:
        return
    from paper_2605_05635_gb300 import workloads
    flats = workloads.sweep_512(precision=0)
    per_step = max(5.0, min(30.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(flats, per_step / 4)
    vals = [cpu_baseline(flats, per_step, seed=11 + k) for k in range(args.steps)]
    v = sum(x["value"] for x in vals) / len(vals)
    base = vals[-1]
    rays_per_image = None
    line = {"metric": METRIC, "value": v, "unit": "rays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "images": len(flats), "nx": 512, "ny": 512,
                       "levels": 3, "sample": "bounded oracle sample per step"},
            "cpu_baseline": {"value": v, "unit": "rays/s", "cores": base["cores"],
                             "kind": "oracle", "sample": base["sample"]},
            "e2e": {"value": v, "unit": "rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "images_per_s": rays_per_image}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 5; for the millisecond-long visibility, amplitude-"
                         "curve and 64^2 calls, enough calls to last about a second, so that the "
                         "clock sampler sees the timed region)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--workload", choices=["sweep512", "sweep96", "vis1024", "adjoint256", "kerr64",
                                           "shadow", "scan", "viscurves"],
                    default="sweep512",
                    help="sweep512: the headline line; sweep96 and vis1024: the batched-sweep "
                         "and visibility measurements")
    ap.add_argument("--emission", choices=["thin", "volumetric"], default="thin",
                    help="sweep512: thin disk (the headline) or the volumetric layer (Eq. 88)")
    ap.add_argument("--autotune", action="store_true", help="sweep96: autotune the plan first")
    ap.add_argument("--no-autotune", action="store_true",
                    help="sweep512: keep the default launch shapes")
    ap.add_argument("--profile-case", default=None,
                    choices=["kerr128", "einasto128", "cnfw128", "sweep512", "sweep512l0",
                             "shadow512", "scan64k"],
                    help="run one fixed case --repeat times for a profiler and exit")
    ap.add_argument("--repeat", type=int, default=2, help="--profile-case: launches")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.steps is None:
        args.steps = default_steps(args.workload)

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist

    import paper_2605_05635_gb300 as B
    from paper_2605_05635_gb300 import workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    prec = B.MIXED if args.precision == "mixed" else B.FP64
    try:
        B.lib()
    except Exception as e:  # the CUDA library is the product; no fallback
        raise SystemExit(f"libbhrt unavailable: {e}")
    stream = torch.cuda.Stream(device=dev)
    if args.workload != "sweep512":
        if world > 1:
            raise SystemExit(f"--workload {args.workload} runs on one GPU")
        fn = {"sweep96": run_sweep96, "vis1024": run_vis1024,
              "adjoint256": run_adjoint, "kerr64": run_kerr64,
              "shadow": run_shadow, "scan": run_scan,
              "viscurves": run_viscurves}[args.workload]
        return fn(args, B, workloads, dev, stream)
    vol = args.emission == "volumetric"
    flats = workloads.sweep_512(precision=prec, volumetric=vol)
    items = [B.from_flat(d) for d in flats]
    plan = B.Plan(items, device=dev, keys_cap=KEYS_CAP)

    with torch.cuda.stream(stream):
        # setup, untimed: the plan's autotuner picks the persistent grids
        # and kernel builds on this workload
        tune = plan.autotune(stream=stream) if not args.no_autotune else None
        for _ in range(args.warmup):
            plan.launch(use_graph=False, stream=stream)
        plan.check(stream)
        plan.set_timing(True)
        sampler = ClockSampler(local)
        barrier()
        torch.cuda.synchronize(dev)
        sampler.start()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        rays = 0
        steps_acc = 0
        trace_ms = 0.0
        steps64, ms64, promoted = 0, 0.0, 0
        max_steps_ray = 0
        launches = 0
        for _ in range(args.steps):
            plan.launch(stream=stream)
            st = plan.stats(stream)          # blocking copy of the counters
            rays += sum(st["rays"])
            if prec == B.FP64:
                steps_acc += st["accepted_fp64"]
                trace_ms += st["fp64_ms"]
            else:
                steps_acc += st["accepted_fp32"]
                trace_ms += st["fp32_ms"]
                steps64 += st["accepted_fp64"]
                ms64 += st["fp64_ms"]
                promoted += st["promoted_rays"]
            launches += st["kernel_launches"]
            max_steps_ray = max(max_steps_ray, st["max_ray_steps"])
            if st["status"] != 0:
                raise SystemExit(f"device status {st['status']}")
        t1.record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop()
        barrier()
        ms = t0.elapsed_time(t1)
    plan.set_timing(False)

    all_rays, max_ms = aggregate_ranks(rays, ms, world, dev)
    value = all_rays / (max_ms / 1e3)
    images_per_s = world * len(items) * args.steps / (max_ms / 1e3)

    # roofline of the dominant kernel: the trace kernel with the larger share
    # of the step (summed over its launches: levels and passes); the other
    # trace kernel of the mixed path rides along
    def kernel_roof(steps, kms, peak, name, source):
        ach = steps * FLOP_PER_STEP / (kms / 1e3) / 1e12 if kms > 0 else 0.0
        return {"bound": "alu", "achieved": ach, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": ach * 1e12 / peak, "traffic": None, "kernel": name,
                "kernel_share_of_step": kms / ms, "accepted_steps": steps,
                "flop_per_accepted_step": FLOP_PER_STEP, "peak_source": source}
    fp64_src = "nominal GB300 FP64 1.25 TFLOP/s (an FMA-chain probe measured 1.19)"
    fp32_src = "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (an FMA-chain probe measured 74.6)"
    if prec == B.FP64:
        roofline = kernel_roof(steps_acc, trace_ms, FP64_PEAK_FLOPS, "trace_fp64_kernel", fp64_src)
    else:
        r32 = kernel_roof(steps_acc, trace_ms, FP32_PEAK_FLOPS, "trace_mixed_kernel", fp32_src)
        r64 = kernel_roof(steps64, ms64, FP64_PEAK_FLOPS, "trace_fp64_kernel", fp64_src)
        for r in (r32, r64):
            r["traffic"] = None if vol else TRAFFIC_PER_STEP.get(r["kernel"])
            r["traffic_unit"] = "bytes per step (all of the kernel's launches of one step)"
        r64["promoted_rays"] = promoted
        r64["pass"] = "FP64 promoted pass of the mixed path"
        r32["pass"] = "FP32 main and demoted passes of the mixed path"
        roofline, other = (r64, r32) if ms64 >= trace_ms else (r32, r64)
        roofline = dict(roofline, other_trace_kernel=other)

    # end to end through the public API with host buffers
    e2e = None
    with torch.cuda.stream(stream):
        outs = plan.outputs
        # the image planes come back to the host (the refinement-key buffers stay)
        planes = [{k: v for k, v in o.items() if k != "refine_keys"} for o in outs]
        host = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in o.items()}
                for o in planes]
        d2h = sum(v.numel() * v.element_size() for o in planes for v in o.values())
        h2d = len(items) * 512  # per-image constants + output pointers uploaded per call
        ws = plan.workspace
        n_e2e = max(1, min(3, args.steps))
        torch.cuda.synchronize(dev)
        barrier()
        w0 = time.perf_counter()
        e_rays = 0
        for _ in range(n_e2e):
            res = B.trace_batch(items, device=dev, stream=stream, outputs=outs, workspace=ws,
                                check=False)
            for o, h in zip(res, host):
                for k in h:
                    h[k].copy_(o[k], non_blocking=True)
            torch.cuda.synchronize(dev)
            e_rays += rays / args.steps
        w1 = time.perf_counter()
        barrier()
        e2e = {"value": world * e_rays / (w1 - w0), "unit": "rays/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    compare = None
    if prec == B.MIXED and not args.no_compare:
        compare = compare_with_fp64(B, workloads, flats, plan, dev, stream, value,
                                    max_ms / args.steps / 1e3)

    if rank == 0:
        cpu = cpu_baseline(flats, args.cpu_seconds) if world == 1 else None
        line = {
            "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == B.FP64 else "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_VOL if vol else WORKLOAD, "images": len(items),
                       "nx": 512, "ny": 512,
                       "levels": 3, "precision": "fp64" if prec == B.FP64 else "mixed",
                       "l2": "working set > L2 (refinement records ~GBs); no flush",
                       "parallelism": f"dp{world}"},
            "images_per_s": images_per_s,
            "rays_per_step": all_rays / args.steps / world,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "e2e": e2e,
            "gpu_launches": launches, "compare": compare, "longest_ray_steps": max_steps_ray,
            "tune": tune,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
