#!/usr/bin/env python
"""Throughput of the non-sequential photon trace on one or more GB300s.

Workload (a step): the LST-like segmented parabolic dish -- 198 hexagonal
spherical facets on a 28 m paraboloid, four masts, a camera box, a 3 m focal
plane -- lit by 1e7 photons at each of the field angles 0, 0.5, 1, 1.5 and
2 deg (5e7 photons, wavelength uniform over 300-600 nm, facet tilt errors
0.1 mrad, roughness 0.3 mrad).  One step traces every photon to termination
in ONE persistent launch and reduces the spot diagram (centroid, R80) of each
field angle.  Metric: photon-bounces/s (sum of per-photon interaction counts
divided by the device time of the step).  Inputs are resident in HBM and
larger than L2 (1.4 GB for FP32).

The FP32 step runs with the accuracy guard: every photon whose running error
estimate exceeds 1e-6 f (position) or 1e-5 rad (direction) is re-traced in
FP64 by a second launch inside the step.

Reported beside it: the FP64 form of the same step; the two-mirror aspheric
(Schwarzschild-Couder-like) system, 1e7 photons at each of 8 field angles, in
FP32 and FP64; the GCT-like dual-mirror system (1e7 photons at each of 5
field angles, FP32); the batched concentrator study; the misalignment sweep; the
gradient batch; the end-to-end rate through the host-buffer entry point
(inputs copied in and results copied out inside the timed region); the ALU
roofline of each trace form and, at one GPU, the CPU oracle timed on the host
cores together with each form's error against it on fixed photon windows.

Multi-GPU (torchrun): photons are independent, so every rank traces its own
full workload with its own photon-id range (weak scaling, no collective in
the data path); a barrier brackets the timed region and the slowest rank's
time is used.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "photon-bounces/s on 1 GB300 (FP32 vs FP64 form, fraction of roofline); grad evals/s"
UNIT = "photon-bounces/s"
ANGLES = W.LST_ANGLES_DEG

# Algorithmic FP operations per counted work unit (add, mul, compare = 1;
# FMA = 2; div, sqrt, log, sin/cos = 1).  Units and figures are listed in the
# design notes: per ray-box test 12, quadric root solve 20 + sqrt, hexagon
# aperture 15, cylinder 25, aspheric Newton iteration 35, Bezier wall 30,
# reflection 8, Fresnel + Snell 35, plus the frame transform (33) and the
# roughness perturbation (36).  Philox is integer work and counts 0 here.
UNIT_FLOPS = {"aabb": 12, "sag": 21, "newton": 35, "aperture": 15, "cylinder": 25, "box": 20, "hexwall": 30,
              "reflect": 8, "refract": 35, "rough": 36, "philox": 0, "rebase": 33, "refine": 120}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(n_per_angle):
    return {"workload": "lst_dish_198_facets_masts_camera_5_field_angles", "photons_per_step": n_per_angle * len(ANGLES),
            "photons_per_angle": n_per_angle, "field_angles_deg": list(ANGLES), "wavelength_nm": [300, 600],
            "facet_tilt_sigma_mrad": 0.1, "roughness_sigma_mrad": 0.3, "max_bounces": 100,
            "outputs": "status, bounce count, focal-plane (x, y) per photon; per-angle centroid and R80",
            "accuracy_bound": "FP32: final positions 1e-6 f, directions 1e-5 rad (FP64 re-trace of photons over it)",
            "l2": "inputs larger than L2 (no flush)"}


def cpu_oracle_rate(n_target_s=15.0, cap=2_000_000, seed=0):
    """The oracle as it stands, on a bounded sample of the same workload."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    # calibrate on a small sample, then size the sample for ~n_target_s seconds
    sc, b = W.lst_workload(4_000, seed=seed)
    t0 = time.perf_counter()
    r = oracle.trace(sc, b.rounded_to(np.float32), seed=seed, eps=oracle.default_eps(sc, 32), n_threads=cores)
    dt = time.perf_counter() - t0
    per_photon = dt / b.n
    n_per_angle = int(min(cap, max(20_000, n_target_s / per_photon)) // len(ANGLES))
    sc, b = W.lst_workload(n_per_angle, seed=seed)
    t0 = time.perf_counter()
    r = oracle.trace(sc, b.rounded_to(np.float32), seed=seed, eps=oracle.default_eps(sc, 32), n_threads=cores)
    dt = time.perf_counter() - t0
    bounces = int(r["bounces"].astype(np.int64).sum())
    return {"value": bounces / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_per_angle} photons per field angle x {len(ANGLES)} angles of the same workload "
                      f"(FP32-rounded inputs, brute-force FP64 oracle, {cores} threads), {dt:.1f} s"}


def _compare(g, r, precision, f, windows, status_det=1):
    """Per-photon error of a GPU trace against the oracle's on the same photons, and the relative
    error of each window's R80, effective area (detected count) and collection efficiency."""
    from oracle import metrics
    same_st = g["status"] == r["status"]
    same = same_st & (g["bounces"] == r["bounces"]) & (g["last_surface"] == r["last_surface"])
    eh = np.abs(g["hit"].astype(np.float64) - r["hit"]).max(axis=0)
    ed = np.abs(g["dir"].astype(np.float64) - r["dir"]).max(axis=0)
    bad = np.where(~same)[0]
    rep = {"photons": int(g["status"].shape[0]), "max_pos_err_over_f": float(eh[same].max(initial=0.0) / f),
           "max_dir_err_rad": float(ed[same].max(initial=0.0)),
           "status_mismatch_frac": float(1.0 - same_st.mean()), "path_mismatches": int(bad.size),
           "path_mismatch_max_edge_margin": float(r["edge_margin"][bad].max()) if bad.size else None}
    r80e, ne, cee = [], [], []
    for s0, c in windows:
        sl = slice(s0, s0 + c)
        mg = metrics.psf(g["status"][sl], g["focal_xy"][:, sl])
        mr = metrics.psf(r["status"][sl], r["focal_xy"][:, sl])
        if mr["n_detected"] > 0:
            r80e.append(abs(mg["r80"] - mr["r80"]) / max(mr["r80"], 1e-300))
            ne.append(abs(mg["n_detected"] - mr["n_detected"]) / mr["n_detected"])
            cee.append(abs((g["status"][sl] == status_det).mean() - (r["status"][sl] == status_det).mean()) /
                       max((r["status"][sl] == status_det).mean(), 1e-300))
    rep.update(r80_rel_err_max=float(max(r80e)) if r80e else None,
               a_eff_rel_err_max=float(max(ne)) if ne else None, ce_rel_err_max=float(max(cee)) if cee else None)
    if "retraced" in g:
        rep["fp64_retraced"] = int(np.asarray(g["retraced"]).ravel()[0])
    return rep


def accuracy_leg(checks):
    """Each form's error against the FP64 oracle on a fixed window of its photon ids (outside
    every timed region; part of the CPU-baseline leg, the one place the bench runs the oracle).
    checks: name -> callable returning (gpu outputs, oracle outputs, precision, f, windows)."""
    out = {}
    for name, fn in checks.items():
        try:
            g, r, precision, f, wins = fn()
            rep = _compare(g, r, precision, f, wins)
            rep["window"] = f"{len(wins)} windows of {wins[0][1]} photons"
            out[name] = rep
        except Exception as e:  # a failed check is reported, not fatal to the bench line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    n_per_angle = args.ref_photons_per_angle
    sc, b = W.lst_workload(n_per_angle, seed=0)
    bb = b.rounded_to(np.float32)
    eps = oracle.default_eps(sc, 32)
    for _ in range(args.warmup):
        oracle.trace(sc, bb, seed=0, eps=eps, n_threads=cores)
    total_b, t = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.trace(sc, bb, seed=0, eps=eps, n_threads=cores)
        t += time.perf_counter() - t0
        total_b += int(r["bounces"].astype(np.int64).sum())
    value = total_b / t
    cfg = workload_config(n_per_angle)
    cfg["note"] = "each step traces a bounded sample of the workload with the CPU oracle"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n_per_angle} photons per field angle x {len(ANGLES)} angles per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def roofline_of(units, kernel_ms, peak, label, peak_source):
    """ALU roofline of a trace launch: algorithmic FLOPs (work units x per-unit figure) over the
    launch's CUDA-event time, against the measured FMA peak."""
    flops = sum(units.get(k, 0) * UNIT_FLOPS[k] for k in UNIT_FLOPS)
    achieved = flops / (kernel_ms * 1e-3)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak, "kernel": label, "kernel_ms": kernel_ms, "flops_per_launch": flops,
            "work_units_per_launch": units, "peak_source": peak_source}


def measure_batched(args, geom_dev, stream, ws, rank, max_over_ranks, sum_over_ranks, barrier, peak32):
    """Batched concentrator study: 64 Bezier-cone variants x 41 incidence angles
    (0-40 deg) x photons per group generated on the device, all in ONE
    persistent launch (plus the FP32 accuracy guard's FP64 re-trace launch),
    replayed from a captured CUDA graph; launch shape from the autotuner.
    Metric: photon-bounces/s; result: collection efficiency per (variant, angle)."""
    import torch
    import paper_1508_07803_gb300 as robast
    from paper_1508_07803_gb300 import autotune

    scene, groups = W.cone_batch(n_variants=64, angles_deg=W.CONE_ANGLES_DEG,
                                 n_per_group=args.batch_photons_per_group, seed=0)
    geom = robast.build_geometry(scene)
    if args.batch_shape:
        (block, bps, rfm), table = _shape(args.batch_shape), {}
    elif args.no_autotune:
        (block, bps, rfm), table = (0, 0, 0), {}
    else:
        (block, bps, rfm), table = autotune.tune_sources(geom, groups, precision=32, max_bounces=30, stream=stream)
    src = robast.sources_create(geom, groups)
    counts = torch.zeros((src.n_groups, 8), dtype=torch.int64, device=geom_dev)
    retraced = torch.zeros(2, dtype=torch.int64, device=geom_dev)
    first_id = rank * src.n_photons

    # one small eager launch with the guard on loads both kernels (trace and FP64 re-trace) before
    # the capture; the full-size launch runs only from the graph
    tiny = robast.sources_create(geom, [dict(groups[0], n=4096)])
    robast.trace_sources(geom, tiny, torch.zeros((1, 8), dtype=torch.int64, device=geom_dev), seed=0, precision=32,
                         max_bounces=30, stream=stream, block_size=block, blocks_per_sm=bps, refill_min=rfm)
    torch.cuda.synchronize()
    tiny.close()
    # capture on a side stream (graphs cannot be captured on the default stream)
    cap = torch.cuda.Stream(device=geom_dev)
    cap.wait_stream(stream)
    with torch.cuda.stream(cap):
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=cap):
            robast.trace_sources(geom, src, counts, seed=0, precision=32, max_bounces=30, stream=cap,
                                 first_photon_id=first_id, block_size=block, blocks_per_sm=bps, refill_min=rfm,
                                 out={"retraced": retraced})
    graph.replay()  # warm-up replay
    torch.cuda.synchronize()
    counts.zero_()
    retraced.zero_()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.batch_steps):
        graph.replay()
    t1.record(stream)
    barrier()
    ms = max_over_ranks(t0.elapsed_time(t1))
    c = counts.cpu().numpy()
    bounces = sum_over_ranks(float(c[:, 0].sum()))
    ce = (c[:, 1] / c[:, 7]).reshape(64, len(W.CONE_ANGLES_DEG))
    angles = list(W.CONE_ANGLES_DEG)
    summary = {f"{int(a)}deg": {"mean": float(ce[:, i].mean()), "min": float(ce[:, i].min()),
                                "max": float(ce[:, i].max())}
               for i, a in enumerate(angles) if int(a) in (0, 10, 20, 25, 30, 35, 40)}
    # work units of the launch, counted on a 1/20 sample of every group (outside the timed region)
    frac = 20
    sample = [dict(g, n=max(1, g["n"] // frac)) for g in groups]
    ssrc = robast.sources_create(geom, sample)
    units_t = torch.zeros(robast.N_UNITS, dtype=torch.int64, device=geom_dev)
    scounts = torch.zeros((ssrc.n_groups, 8), dtype=torch.int64, device=geom_dev)
    robast.trace_sources(geom, ssrc, scounts, seed=0, precision=32, max_bounces=30, stream=stream,
                         block_size=128, work_units=units_t, accuracy=False)
    torch.cuda.synchronize()
    units = {k: v * frac for k, v in zip(robast.UNIT_NAMES, units_t.cpu().tolist())}
    # the accuracy guard's share, timed on the same sample: the FP32 launch alone, then with the guard
    gms = []
    for acc in (False, None):
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        robast.trace_sources(geom, ssrc, scounts, seed=0, precision=32, max_bounces=30, stream=stream,
                             block_size=block, blocks_per_sm=bps, refill_min=rfm, accuracy=acc)
        g1.record(stream)
        g1.synchronize()
        gms.append(g0.elapsed_time(g1))
    guard = {"sample": "1/20 of every group", "fp32_trace_ms": gms[0], "with_guard_ms": gms[1],
             "guard_ms": gms[1] - gms[0]}
    ssrc.close()
    kern_ms = ms / args.batch_steps
    roof = roofline_of(units, kern_ms, peak32, "robast::trace_kernel<float,SRC> (+ FP64 re-trace)",
                       "FFMA throughput probe robast_measure_alu_peak on this GPU (measured); work units counted "
                       "on a 1/20 sample of every group, times 20")
    rt = retraced.cpu().tolist()
    src.close()
    geom.close()
    return {"value": bounces / (ms * 1e-3), "unit": UNIT, "ms_per_step": kern_ms,
            "steps": args.batch_steps, "photons_per_step": src.n_photons,
            "bounces_per_step": bounces / args.batch_steps / ws,
            "fp64_retraced_per_step": rt[0] // args.batch_steps, "over_bound_not_retraced": rt[1],
            "guard": dict(guard, retraced_fraction=(rt[0] // args.batch_steps) / src.n_photons),
            "roofline": roof,
            "config": {"workload": "hex_bezier_cone_64_variants_x_41_angles", "variants": 64,
                       "angles_deg": [0, 40, 1], "photons_per_group": args.batch_photons_per_group,
                       "max_bounces": 30, "sources": "generated on the device (Philox stream 1)",
                       "launch": "one persistent launch per step (+ the accuracy guard's FP64 re-trace), "
                                 "replayed from a CUDA graph"},
            "autotune": {"block": block, "blocks_per_sm": bps, "refill_min": rfm,
                         "candidates_ms": {f"{b}x{p}/r{r}": round(t, 3) for (b, p, r), t in table.items()}},
            "collection_efficiency": summary}


def batched_accuracy_check(dev, n_window=12_500, n_groups=8):
    """Windows of single groups of the batched study, re-traced on the GPU at their original
    photon ids (source mode, FP32 with the accuracy guard) and by the oracle."""
    import torch
    import oracle
    import paper_1508_07803_gb300 as robast
    scene, groups = W.cone_batch(n_variants=64, angles_deg=W.CONE_ANGLES_DEG, n_per_group=2_000_000, seed=0)
    geom = robast.build_geometry(scene)
    first = np.cumsum([0] + [g["n"] for g in groups])
    rng = np.random.default_rng(11)
    gs, rs = [], []
    for gi in sorted(rng.choice(len(groups), size=n_groups, replace=False).tolist()):
        pid0 = int(first[gi]) + int(rng.integers(0, groups[gi]["n"] - n_window))
        one = [dict(groups[gi], n=n_window)]
        s1 = robast.sources_create(geom, one)
        cnt = torch.zeros((1, 8), dtype=torch.int64, device=dev)
        out = robast.alloc_outputs(n_window, 32, dev)
        robast.trace_sources(geom, s1, cnt, seed=0, precision=32, max_bounces=30, out=out, first_photon_id=pid0)
        torch.cuda.synchronize()
        s1.close()
        bb, var, _ = oracle.generate_sources(one, seed=0, first_photon_id=pid0)
        bundle = W.Bundle(bb["origins"], bb["dirs"], bb["wavelengths"]).rounded_to(np.float32)
        rs.append(oracle.trace(scene, bundle, seed=0, first_photon_id=pid0, max_bounces=30, variant_of_photon=var,
                               eps=oracle.default_eps(scene, 32)))
        gs.append({k: v.cpu().numpy() for k, v in out.items()})
    geom.close()
    cat = lambda ds, k: np.concatenate([d[k] for d in ds], axis=-1)
    g = {k: cat(gs, k) for k in ("status", "bounces", "hit", "dir", "last_surface", "focal_xy")}
    g["retraced"] = np.array([sum(int(d["retraced"][0]) for d in gs)])
    r = {k: cat(rs, k) for k in ("status", "bounces", "hit", "dir", "last_surface", "focal_xy", "edge_margin")}
    return g, r, 32, scene.focal_length, [(k * n_window, n_window) for k in range(n_groups)]


def measure_tolerance(args, dev, stream, ws, rank, max_over_ranks, sum_over_ranks, barrier, peak32):
    """Misalignment study: 64 realisations of the dish with Gaussian facet-tilt
    errors (0.5 mrad per axis), 1e6 photons each at a 1 deg field, all
    realisations in one launch (variants); the step includes the R80 of every
    realisation.  Reports photon-bounces/s and the R80 distribution."""
    import torch
    import paper_1508_07803_gb300 as robast

    nr, m = 64, 1_000_000
    scene, b, vop = W.tolerance_sweep(n_realizations=nr, tilt_sigma=0.5e-3, photons_per_realization=m, seed=rank)
    geom = robast.build_geometry(scene)
    o = torch.from_numpy(b.origins).to(dev, torch.float32)
    d = torch.from_numpy(b.dirs).to(dev, torch.float32)
    w = torch.from_numpy(b.wavelengths).to(dev, torch.float32)
    v = torch.from_numpy(vop).to(dev)
    out = robast.alloc_outputs(b.n, 32, dev, fields=("status", "bounces", "focal_xy", "counters", "retraced"))
    wins = [(k * m, m) for k in range(nr)]

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        robast.trace(geom, o, d, w, seed=0, variant_of_photon=v, out=out, stream=stream,
                     first_photon_id=rank * b.n)
        if ev is not None:
            ev[1].record(stream)
        return robast.psf(geom, out["status"], out["focal_xy"], windows=wins, stream=stream)

    for _ in range(3):
        step()
    units_t = torch.zeros(robast.N_UNITS, dtype=torch.int64, device=dev)
    robast.trace(geom, o, d, w, seed=0, variant_of_photon=v, stream=stream, first_photon_id=rank * b.n,
                 work_units=units_t, block_size=128, accuracy=False,
                 out=robast.alloc_outputs(b.n, 32, dev, fields=("status",)))
    torch.cuda.synchronize()
    units = dict(zip(robast.UNIT_NAMES, units_t.cpu().tolist()))
    out["counters"].zero_()
    out["retraced"].zero_()
    barrier()
    steps = 5
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(steps):
        res = step(evs[k])
    t1.record(stream)
    barrier()
    ms = max_over_ranks(t0.elapsed_time(t1))
    kern_ms = statistics.mean(a.elapsed_time(z) for a, z in evs)
    bounces = sum_over_ranks(float(out["counters"][0].item()))
    r80 = np.array([r[3] for r in res])
    rt = out["retraced"].cpu().tolist()
    geom.close()
    return {"value": bounces / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "photons_per_step": int(b.n), "fp64_retraced_per_step": rt[0] // steps,
            "roofline": roofline_of(units, kern_ms, peak32, "robast::trace_kernel<float,512> (+ sort, FP64 re-trace)",
                                    "FFMA throughput probe robast_measure_alu_peak on this GPU (measured)"),
            "r80_m": {"mean": float(r80.mean()), "std": float(r80.std()), "min": float(r80.min()),
                      "max": float(r80.max())},
            "config": {"workload": "lst_tolerance_64_realisations_tilt_0.5mrad", "realisations": nr,
                       "photons_per_realisation": m, "field_deg": 1.0}}


def tolerance_accuracy_check(dev, n_window=25_000):
    import torch
    import oracle
    import paper_1508_07803_gb300 as robast
    nr, m = 64, 1_000_000
    scene, b, vop = W.tolerance_sweep(n_realizations=nr, tilt_sigma=0.5e-3, photons_per_realization=m, seed=0)
    wins = [(k * m + 4321, n_window) for k in (0, 21, 42, 63)]
    idx = np.concatenate([np.arange(s0, s0 + c) for s0, c in wins])
    return _plain_window_check(dev, scene, b, idx, 32, vop=vop, n_window=n_window)


def _plain_window_check(dev, scene, b, idx, precision, vop=None, n_window=None, max_bounces=100):
    """GPU re-trace (at the original photon ids) and oracle trace of windows of a plain workload;
    idx: the photon indices of the windows, contiguous runs of n_window."""
    import torch
    import oracle
    import paper_1508_07803_gb300 as robast
    geom = robast.build_geometry(scene)
    dt = torch.float32 if precision == 32 else torch.float64
    gs, rs = [], []
    for s0 in idx[::n_window]:
        s0 = int(s0)
        sl = slice(s0, s0 + n_window)
        part = W.Bundle(np.ascontiguousarray(b.origins[:, sl]), np.ascontiguousarray(b.dirs[:, sl]),
                        b.wavelengths[sl].copy())
        if precision == 32:
            part = part.rounded_to(np.float32)
        v = None if vop is None else np.ascontiguousarray(vop[sl])
        o = torch.from_numpy(part.origins).to(dev, dt)
        d = torch.from_numpy(part.dirs).to(dev, dt)
        w = torch.from_numpy(part.wavelengths).to(dev, dt)
        out = robast.trace(geom, o, d, w, seed=0, precision=precision, first_photon_id=s0, max_bounces=max_bounces,
                           variant_of_photon=None if v is None else torch.from_numpy(v).to(dev))
        torch.cuda.synchronize()
        gs.append({k: x.cpu().numpy() for k, x in out.items()})
        rs.append(oracle.trace(scene, part, seed=0, first_photon_id=s0, max_bounces=max_bounces,
                               eps=oracle.default_eps(scene, precision), variant_of_photon=v))
    geom.close()
    cat = lambda ds, k: np.concatenate([x[k] for x in ds], axis=-1)
    g = {k: cat(gs, k) for k in ("status", "bounces", "hit", "dir", "last_surface", "focal_xy")}
    if precision == 32:
        g["retraced"] = np.array([sum(int(x["retraced"][0]) for x in gs)])
    r = {k: cat(rs, k) for k in ("status", "bounces", "hit", "dir", "last_surface", "focal_xy", "edge_margin")}
    nw = len(gs)
    return g, r, precision, scene.focal_length, [(k * n_window, n_window) for k in range(nw)]


# FP64 FLOPs of one re-solved interaction of the gradient pass (frame transform 33, quadric or
# Bezier root and one Newton step ~56, aperture 15, normal ~10, reflection 8, roughness 36), and
# the multiplier of its 16-slot dual form (each operation carries 16 derivative lanes: an add 16
# more, a product 32 more; about 17x on this mix)
GRAD_INTERACTION_FLOPS = 158
GRAD_DUAL_FACTOR = 17


def grad_roofline(units, ms_per_eval, peak64, peak32=None, r64=True):
    """ALU roofline of the gradient launch: the forward pass's interactions run in FP64, the
    replays and the dual-number interactions in the derivative precision (FP32 for an FP32 dish
    batch, FP64 through cone walls).  achieved = FLOPs / time; peak = the FLOP-weighted harmonic
    mean of the two measured peaks (the time the same FLOPs take at peak on each pipe)."""
    fwd, rep, dual = units
    f64 = fwd * GRAD_INTERACTION_FLOPS
    fr = rep * GRAD_INTERACTION_FLOPS + dual * GRAD_INTERACTION_FLOPS * GRAD_DUAL_FACTOR
    if r64 or peak32 is None:
        f64, fr, pr = f64 + fr, 0.0, peak64
    else:
        pr = peak32
    flops = f64 + fr
    t_peak = f64 / peak64 + (fr / pr if fr else 0.0)
    peak = flops / t_peak if t_peak > 0 else peak64
    achieved = flops / (ms_per_eval * 1e-3)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "kernel": "robast::grad_kernel<float, " + ("double" if r64 else "float") + "> (adjoint)",
            "flops_per_eval": flops, "fp64_flops_per_eval": f64,
            "work_units_per_eval": {"fwd_interactions": fwd, "replayed_interactions": rep,
                                    "dual_interactions": dual},
            "peak_source": "DFMA and FFMA throughput probes robast_measure_alu_peak on this GPU (measured), "
                           "weighted by the FP64 and FP32 FLOPs; FLOPs per interaction estimated from the "
                           "operation counts"}


def measure_grad_cone(args, dev, stream, ws, rank, max_over_ranks, barrier):
    """Soft collection efficiency of a Bezier hexagonal cone behind its window and its gradient
    with respect to the 6 control-point coordinates of the wall profile: 1e6 photons over
    incidence angles 0-30 deg (FP32 trace; derivative passes in FP64 through the cone walls, whose
    grazing roots need it).  Metric: gradient evaluations/s."""
    import math
    import torch
    import paper_1508_07803_gb300 as robast
    scene = W.cone_scene(n_variants=1, seed=rank)
    H = W.cone_heights(1)[0]
    m = args.grad_cone_photons // 7
    b = W.concat([W.hexagon_bundle(m, W.CONE_A_IN, H + W.CONE_WINDOW + 1e-4, math.radians(a), seed=rank,
                                   stream=700 + k) for k, a in enumerate(range(0, 31, 5))])
    geom = robast.build_geometry(scene)
    o = torch.from_numpy(b.origins).to(dev, torch.float32)
    d = torch.from_numpy(b.dirs).to(dev, torch.float32)
    w = torch.from_numpy(b.wavelengths).to(dev, torch.float32)
    g = torch.zeros((geom.n_surfaces, robast.N_PARAM), dtype=torch.float64, device=dev)

    def evaluate():
        g.zero_()
        return robast.trace_grad(geom, o, d, w, objective="soft_ce", precision=32, seed=0, max_bounces=30,
                                 stream=stream, out=g)

    for _ in range(2):
        evaluate()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.grad_steps):
        value, _, info = evaluate()
    barrier()
    dt = max_over_ranks(time.perf_counter() - t0)
    units = torch.zeros(3, dtype=torch.int64, device=dev)
    robast.trace_grad(geom, o, d, w, objective="soft_ce", precision=32, seed=0, max_bounces=30, stream=stream,
                      work_units=units, grad=False)
    grad = g[1, 10:16].cpu().tolist()
    geom.close()
    return {"value": ws * args.grad_steps / dt, "unit": "grad evals/s", "ms_per_eval": 1e3 * dt / args.grad_steps,
            "roofline": grad_roofline(units.cpu().tolist(), 1e3 * dt / args.grad_steps, args.peak64),
            "photons_per_eval": int(b.n), "objective": "soft collection efficiency (tau = 0.5 mm), frozen path",
            "objective_value": value, "gradient_P0r_P0z_P1r_P1z_P2r_P2z": grad,
            "config": {"workload": "bezier_hex_cone_soft_ce_7_angles_0_to_30_deg", "photons": int(b.n),
                       "max_bounces": 30, "timing": "host wall clock around the synchronous call"}}


def measure_grad(args, dev, stream, ws, rank, max_over_ranks, barrier):
    """Differentiable batch: 32 LST-like dishes with 60-198 facets, 1e6
    photons each over field angles 0-2 deg, one evaluation = the summed
    mean-squared spot radius of the 32 dishes AND its gradient with respect to
    every facet's two tilts and eight aspheric coefficients, in one launch
    (FP32 trace and derivative passes, FP64 forward values, fixed-point sums).  Dish v is lit at the
    field angle 2 v / 31 deg.  Metric: gradient evaluations/s."""
    import torch
    import paper_1508_07803_gb300 as robast

    scene, b, vop, counts = W.dish_batch(n_dishes=32, photons_per_dish=args.grad_photons_per_dish, seed=rank)
    geom = robast.build_geometry(scene)
    o = torch.from_numpy(b.origins).to(dev, torch.float32)
    d = torch.from_numpy(b.dirs).to(dev, torch.float32)
    w = torch.from_numpy(b.wavelengths).to(dev, torch.float32)
    v = torch.from_numpy(vop).to(dev)
    g = torch.zeros((geom.n_surfaces, robast.N_PARAM), dtype=torch.float64, device=dev)

    def evaluate():
        g.zero_()
        return robast.trace_grad(geom, o, d, w, objective="msr", precision=32, seed=0, variant_of_photon=v,
                                 stream=stream, out=g, coherent_order=args.grad_order)

    for _ in range(2):
        evaluate()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.grad_steps):
        value, _, info = evaluate()
    barrier()
    dt = max_over_ranks(time.perf_counter() - t0)
    gn = float(torch.linalg.vector_norm(g).item())
    layout = robast.param_layout(geom)
    active = sum(1 for p in layout if p[3])
    units = torch.zeros(3, dtype=torch.int64, device=dev)
    robast.trace_grad(geom, o, d, w, objective="msr", precision=32, seed=0, variant_of_photon=v, stream=stream,
                      work_units=units, grad=False)
    geom.close()
    return {"value": ws * args.grad_steps / dt, "unit": "grad evals/s", "ms_per_eval": 1e3 * dt / args.grad_steps,
            "roofline": grad_roofline(units.cpu().tolist(), 1e3 * dt / args.grad_steps, args.peak64, args.peak32, r64=False),
            "photons_per_eval": int(b.n), "photons_per_s": ws * args.grad_steps * b.n / dt,
            "objective": "sum over 32 dishes of the mean-squared spot radius (frozen path, expected weights)",
            "objective_value_m2": value, "gradient_norm": gn, "n_params": int(geom.n_surfaces * robast.N_PARAM),
            "n_params_active": active,
            "n_detected": int(info["n_detected"]), "untracked_photons": int(info["n_untracked"]),
            "config": {"workload": "dish_batch_32_dishes_60_to_198_facets", "facets": [counts[0], counts[-1]],
                       "photons_per_dish": args.grad_photons_per_dish, "field_angle_deg": "2 v / 31 for dish v",
                       "timing": "host wall clock around the synchronous call (value returned to the host)"}}


def _shape(text):
    b, k, r = (int(v) for v in text.split(","))
    return b, k, r


def _hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0  # fallback: an earlier measurement on a GB300


HBM_PEAK_GBS = _hbm_peak()

TRAFFIC_SOURCES = ("trace.cuh", "trace_f32.cu", "order.cu")  # the kernel and the processing order that shapes its DRAM traffic


def traffic_source_hash():
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1508_07803_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def traffic_from_profile(n_photons):
    """DRAM bytes of the trace kernel from the committed ncu summary, if it was
    taken on the current kernel and ordering sources; else None."""
    path = os.path.join(ROOT, "profiles", "trace_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        meta = json.load(open(path))
        if meta.get("sources_sha256") != traffic_source_hash():
            return None
        return meta["dram_bytes_per_photon"] * n_photons
    except Exception:
        return None


def issue_from_profile():
    """Issue and pipe utilisation of the trace kernel from the committed ncu capture
    (profiles/trace_kernel_issue.json, a small case of the same kernel), if it was taken on the
    current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "trace_kernel_issue.json")
    if not os.path.exists(path):
        return None
    try:
        meta = json.load(open(path))
        if meta.get("sources_sha256") != traffic_source_hash():
            return None
        return {k: meta[k] for k in ("issue_active", "ipc_per_sm", "fma_pipe", "alu_pipe", "fp64_pipe",
                                     "warps_active", "lanes_active_per_inst")}
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--photons-per-angle", type=int, default=10_000_000)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--ref-photons-per-angle", type=int, default=20_000)
    ap.add_argument("--sct-photons-per-angle", type=int, default=10_000_000)
    ap.add_argument("--sct-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-sct", action="store_true")
    ap.add_argument("--no-gct", action="store_true")
    ap.add_argument("--gct-photons-per-angle", type=int, default=10_000_000)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-tolerance", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="library launch defaults instead of the tuners (keeps profiler launch counts small)")
    ap.add_argument("--trace-shape", default=None,
                    help="block,blocks_per_sm,refill_min for the plain FP32 traces instead of the tuner (profiler runs)")
    ap.add_argument("--batch-shape", default=None,
                    help="block,blocks_per_sm,refill_min for the batched trace instead of the tuner (profiler runs)")
    ap.add_argument("--grad-photons-per-dish", type=int, default=1_000_000)
    ap.add_argument("--grad-steps", type=int, default=3)
    ap.add_argument("--grad-order", type=int, default=0, choices=[-1, 0, 1],
                    help="processing order of the dish-batch gradient (profiler runs): 0 the library default, "
                         "1 coherent (origin cell), -1 photon id")
    ap.add_argument("--grad-cone-photons", type=int, default=1_000_000)
    ap.add_argument("--batch-photons-per-group", type=int, default=2_000_000)
    ap.add_argument("--batch-steps", type=int, default=1)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1508_07803_gb300 as robast
    from paper_1508_07803_gb300 import shard

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    robast.load()
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return shard.all_reduce_scalar(x, "max", device=dev)

    def sum_over_ranks(x):
        return shard.all_reduce_scalar(x, "sum", device=dev)

    def measure(scene, bundle, npa, n_angles, precision, steps, warmup, want_clocks):
        """One step: coherent-order sort, one trace launch (+ the accuracy guard's FP64 re-trace in
        FP32), spot-diagram reduction of every field angle."""
        geom = robast.build_geometry(scene)
        N = bundle.n
        first_id = shard.replica_first_id(rank, N)
        dt = torch.float32 if precision == 32 else torch.float64
        o = torch.from_numpy(bundle.origins).to(dev, dt)
        d = torch.from_numpy(bundle.dirs).to(dev, dt)
        w = torch.from_numpy(bundle.wavelengths).to(dev, dt)
        # per-photon outputs the spot diagram and the metric need: status, bounce count, focal (x, y)
        fields = ("status", "bounces", "focal_xy", "counters") + (("retraced",) if precision == 32 else ())
        out = robast.alloc_outputs(N, precision, dev, fields=fields)
        counters = out["counters"]
        # per step: the coherent-order sort (init, bounds, count, columns, three scan launches, place), the
        # trace (+ the FP64 re-trace in FP32), and the reduction (sums, finish, histogram, pick, compact,
        # check, candidate r^2, sub-histogram, pick, collect, select; all angles at once)
        order_launches, psf_launches = 8, 11
        trace_launches = 2 if precision == 32 else 1
        wins = [(k * npa, npa) for k in range(n_angles)]
        # launch shape and refill threshold from the autotuner (on the first 2e6 photons, untimed)
        from paper_1508_07803_gb300 import autotune
        if args.trace_shape and precision == 32:
            (blk, bps, rfm), table = _shape(args.trace_shape), {}
        elif args.no_autotune:
            (blk, bps, rfm), table = (0, 0, 0), {}
        else:
            (blk, bps, rfm), table = autotune.tune_trace(geom, o, d, w, precision=precision, stream=stream)

        def step(ev=None):
            if ev is not None:
                ev[0].record(stream)
            robast.trace(geom, o, d, w, seed=0, precision=precision, first_photon_id=first_id, out=out,
                         stream=stream, block_size=blk, blocks_per_sm=bps, refill_min=rfm)
            if ev is not None:
                ev[1].record(stream)
            return robast.psf(geom, out["status"], out["focal_xy"], precision=precision, stream=stream, windows=wins)

        for _ in range(warmup):
            step()
        # work units of one launch (counting build, outside the timed region)
        units = torch.zeros(robast.N_UNITS, dtype=torch.int64, device=dev)
        robast.trace(geom, o, d, w, seed=0, precision=precision, first_photon_id=first_id, stream=stream,
                     work_units=units, block_size=128, accuracy=False,
                     out=robast.alloc_outputs(N, precision, dev, fields=("status",)))
        torch.cuda.synchronize()
        units = dict(zip(robast.UNIT_NAMES, units.cpu().tolist()))
        counters.zero_()
        if "retraced" in out:
            out["retraced"].zero_()
        barrier()
        clocks = ClockSampler(dev.index) if want_clocks else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        barrier()
        t0.record(stream)
        last = None
        for k in range(steps):
            last = step(evs[k])
        t1.record(stream)
        barrier()
        ms = t0.elapsed_time(t1)
        kern_ms = [a.elapsed_time(b) for a, b in evs]
        # whole steps (trace start to the next trace start, the last to the end): a step much
        # longer than its kernels means the device waited on the host
        step_ms = [evs[k][0].elapsed_time(evs[k + 1][0]) for k in range(steps - 1)] + [evs[-1][0].elapsed_time(t1)]
        clk = clocks.stop() if clocks else None
        c = counters.cpu().tolist()
        rt = out["retraced"].cpu().tolist() if "retraced" in out else [0, 0]
        guard = None
        if precision == 32:
            # the accuracy guard's share of the trace: one FP32 launch without it (after the timed region)
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            robast.trace(geom, o, d, w, seed=0, precision=precision, first_photon_id=first_id, out=out,
                         stream=stream, block_size=blk, blocks_per_sm=bps, refill_min=rfm, accuracy=False)
            g1.record(stream)
            g1.synchronize()
            f32_ms = g0.elapsed_time(g1)
            guard = {"fp32_trace_ms": f32_ms, "with_guard_ms": statistics.mean(kern_ms),
                     "guard_ms": statistics.mean(kern_ms) - f32_ms,
                     "retraced_fraction": (rt[0] // steps) / N}
        geom.close()
        return {"ms": ms, "kernel_ms": kern_ms, "bounces": c[0], "counters": c, "units": units, "psf": last,
                "clocks": clk, "launches": steps * (order_launches + trace_launches + psf_launches),
                "retraced_per_step": rt[0] // steps, "over_bound_not_retraced": rt[1], "guard": guard,
                "step_ms": step_ms,
                "autotune": {"block": blk, "blocks_per_sm": bps, "refill_min": rfm,
                             "candidates_ms": {f"{b}x{p}/r{r}": round(t, 3) for (b, p, r), t in table.items()}}}

    def form_of(m, steps, precision, peak, label):
        msx = max_over_ranks(m["ms"])
        v = sum_over_ranks(m["bounces"]) / (msx * 1e-3)
        k = statistics.mean(m["kernel_ms"])
        f = {"value": v, "ms_per_step": msx / steps, "kernel_ms": k, "bounces_per_step": m["bounces"] / steps,
             "step_ms_min_median_max": [min(m["step_ms"]), statistics.median(m["step_ms"]), max(m["step_ms"])],
             "roofline": roofline_of(m["units"], k, peak, label,
                                     ("FFMA" if precision == 32 else "DFMA") +
                                     " throughput probe robast_measure_alu_peak on this GPU (measured)")}
        if precision == 32:
            f["fp64_retraced_per_step"] = m["retraced_per_step"]
            f["over_bound_not_retraced"] = m["over_bound_not_retraced"]
            f["guard"] = m["guard"]
        f["autotune"] = m["autotune"]
        return f

    peak32 = robast.measure_alu_peak(32)
    peak64 = robast.measure_alu_peak(64)
    args.peak64 = peak64
    args.peak32 = peak32
    npa = args.photons_per_angle
    scene, bundle = W.lst_workload(npa, seed=rank)
    N = bundle.n
    fp32 = measure(scene, bundle, npa, len(ANGLES), 32, args.steps, args.warmup, want_clocks=True)
    forms = {"fp32": form_of(fp32, args.steps, 32, peak32, "robast::trace_kernel<float,512> (+ sort, FP64 re-trace)")}
    ms = max_over_ranks(fp32["ms"])
    value = forms["fp32"]["value"]
    roof = dict(forms["fp32"]["roofline"])
    roof["traffic"] = traffic_from_profile(N)
    # the same launch against the copy bandwidth (DRAM bytes of the committed capture over this
    # run's kernel time), and its issue utilisation (ncu, committed small-case capture): the
    # FLOP fraction above counts only algorithmic arithmetic, the issue fraction every instruction
    if roof["traffic"]:
        gbs = roof["traffic"] / (roof["kernel_ms"] * 1e-3) / 1e9
        roof["hbm"] = {"achieved_gbs": gbs, "peak_gbs": HBM_PEAK_GBS, "frac": gbs / HBM_PEAK_GBS,
                       "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"}
    roof["issue"] = issue_from_profile()
    if not args.no_fp64:
        fp64 = measure(scene, bundle, npa, len(ANGLES), 64, args.fp64_steps, 3, want_clocks=False)
        forms["fp64"] = form_of(fp64, args.fp64_steps, 64, peak64, "robast::trace_kernel<double,128> (+ sort)")

    if not args.no_sct:
        snpa = args.sct_photons_per_angle
        sscene, sbundle = W.sct_workload(snpa, seed=rank)
        nang = len(W.SCT_ANGLES_DEG)
        s32 = measure(sscene, sbundle, snpa, nang, 32, args.sct_steps, 3, want_clocks=False)
        forms["sct_fp32"] = form_of(s32, args.sct_steps, 32, peak32, "robast::trace_kernel<float,512> (+ sort, FP64 re-trace)")
        s64 = measure(sscene, sbundle, snpa, nang, 64, max(2, args.sct_steps // 2), 3, want_clocks=False)
        forms["sct_fp64"] = form_of(s64, max(2, args.sct_steps // 2), 64, peak64, "robast::trace_kernel<double,128> (+ sort)")
        for k, m in (("sct_fp32", s32), ("sct_fp64", s64)):
            forms[k]["config"] = {"workload": "sct_two_mirror_aspheric_8_field_angles", "photons_per_angle": snpa,
                                  "field_angles_deg": [round(a, 4) for a in W.SCT_ANGLES_DEG],
                                  "newton": "FP32 bulk, FP64 last Newton step at grazing incidence"}
            forms[k]["psf"] = [{"field_deg": round(a, 4), "n_detected": int(p[0]), "r80_m": p[3]}
                               for a, p in zip(W.SCT_ANGLES_DEG, m["psf"])]
        del sbundle

    if not args.no_gct:
        gnpa = args.gct_photons_per_angle
        gscene, gbundle = W.gct_workload(gnpa, seed=rank)
        g32 = measure(gscene, gbundle, gnpa, len(W.GCT_ANGLES_DEG), 32, args.sct_steps, 3, want_clocks=False)
        forms["gct_fp32"] = form_of(g32, args.sct_steps, 32, peak32, "robast::trace_kernel<float,512> (+ sort, FP64 re-trace)")
        forms["gct_fp32"]["config"] = {"workload": "gct_like_dual_mirror_6_petals_5_field_angles",
                                       "photons_per_angle": gnpa, "field_angles_deg": list(W.GCT_ANGLES_DEG)}
        forms["gct_fp32"]["psf"] = [{"field_deg": a, "n_detected": int(p[0]), "r80_m": p[3]}
                                    for a, p in zip(W.GCT_ANGLES_DEG, g32["psf"])]
        del gbundle

    if not args.no_batched:
        forms["batched_fp32"] = measure_batched(args, geom_dev=dev, stream=stream, ws=ws, rank=rank,
                                                max_over_ranks=max_over_ranks, sum_over_ranks=sum_over_ranks,
                                                barrier=barrier, peak32=peak32)

    if not args.no_tolerance:
        forms["tolerance_fp32"] = measure_tolerance(args, dev=dev, stream=stream, ws=ws, rank=rank,
                                                    max_over_ranks=max_over_ranks, sum_over_ranks=sum_over_ranks,
                                                    barrier=barrier, peak32=peak32)

    if not args.no_grad:
        forms["grad_fp32"] = measure_grad(args, dev=dev, stream=stream, ws=ws, rank=rank,
                                          max_over_ranks=max_over_ranks, barrier=barrier)
        forms["grad_cone_fp32"] = measure_grad_cone(args, dev=dev, stream=stream, ws=ws, rank=rank,
                                                    max_over_ranks=max_over_ranks, barrier=barrier)

    e2e = None
    if not args.no_e2e:
        geom = robast.build_geometry(scene)
        first_id = shard.replica_first_id(rank, N)
        dt = torch.float32
        ho = torch.from_numpy(bundle.origins).to(dt).pin_memory()
        hd = torch.from_numpy(bundle.dirs).to(dt).pin_memory()
        hw = torch.from_numpy(bundle.wavelengths).to(dt).pin_memory()
        hout = {"status": torch.empty(N, dtype=torch.uint8).pin_memory(),
                "bounces": torch.empty(N, dtype=torch.uint8).pin_memory(),
                "focal_xy": torch.empty((2, N), dtype=dt).pin_memory(),
                "counters": torch.zeros(robast.N_COUNTERS, dtype=torch.int64),
                "retraced": torch.zeros(2, dtype=torch.int64)}
        for _ in range(2):
            robast.trace_host(geom, ho, hd, hw, seed=0, out=hout, first_photon_id=first_id)
        hout["counters"].zero_()
        e2e_steps = max(3, args.steps // 4)
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            robast.trace_host(geom, ho, hd, hw, seed=0, out=hout, first_photon_id=first_id)
        barrier()
        et = max_over_ranks(time.perf_counter() - t0)
        eb = sum_over_ranks(float(hout["counters"][0].item()))
        geom.close()
        e2e = {"value": eb / et, "unit": UNIT, "h2d_bytes_per_step": int(N * 7 * 4),
               "d2h_bytes_per_step": int(N * (1 + 1 + 2 * 4)), "steps": e2e_steps,
               "api": "robast_trace_host (pinned host buffers in and out, FP32 with the accuracy guard)"}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    accuracy = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate()
        # each form's error against the oracle, on fixed windows of its photon ids
        m = 20_000
        dish_idx = np.concatenate([np.arange(k * npa + 7777, k * npa + 7777 + m) for k in range(len(ANGLES))])
        checks = {"fp32": lambda: _plain_window_check(dev, scene, bundle, dish_idx, 32, n_window=m)}
        if not args.no_fp64:
            checks["fp64"] = lambda: _plain_window_check(dev, scene, bundle, dish_idx, 64, n_window=m)
        if not args.no_sct:
            sm = 12_500
            sscene, sbundle = W.sct_workload(args.sct_photons_per_angle, seed=0)
            sidx = np.concatenate([np.arange(k * args.sct_photons_per_angle + 555,
                                             k * args.sct_photons_per_angle + 555 + sm)
                                   for k in range(len(W.SCT_ANGLES_DEG))])
            checks["sct_fp32"] = lambda: _plain_window_check(dev, sscene, sbundle, sidx, 32, n_window=sm)
            checks["sct_fp64"] = lambda: _plain_window_check(dev, sscene, sbundle, sidx, 64, n_window=sm)
        if not args.no_gct:
            gm = 20_000
            gscene, gbundle = W.gct_workload(args.gct_photons_per_angle, seed=0)
            gidx = np.concatenate([np.arange(k * args.gct_photons_per_angle + 999,
                                             k * args.gct_photons_per_angle + 999 + gm)
                                   for k in range(len(W.GCT_ANGLES_DEG))])
            checks["gct_fp32"] = lambda: _plain_window_check(dev, gscene, gbundle, gidx, 32, n_window=gm)
        if not args.no_batched:
            checks["batched_fp32"] = lambda: batched_accuracy_check(dev)
        if not args.no_tolerance:
            checks["tolerance_fp32"] = lambda: tolerance_accuracy_check(dev)
        accuracy = accuracy_leg(checks)
        for k, a in accuracy.items():
            if k in forms:
                forms[k]["accuracy"] = a
    psf = [{"field_deg": a, "n_detected": int(p[0]), "cx_m": p[1], "cy_m": p[2], "r80_m": p[3],
            "a_eff_m2": p[0] / npa * math.pi * 12.0 ** 2} for a, p in zip(ANGLES, fp32["psf"])]
    cfg = workload_config(npa)
    cfg["parallelism"] = f"replicas{ws}" if ws > 1 else "single"
    launches = fp32["launches"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg, "forms": forms,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": fp32["clocks"], "psf": psf,
            "accuracy": (accuracy or {}).get("fp32"),
            "status_counts_per_step": [c // args.steps for c in fp32["counters"][1:7]]}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
