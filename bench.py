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

Reported beside it: the FP64 form of the same step, the end-to-end rate
through the host-buffer entry point (inputs copied in and results copied out
inside the timed region), the ALU roofline of the trace kernel and, at one
GPU, the CPU oracle timed on the host cores.

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
              "reflect": 8, "refract": 35, "rough": 36, "philox": 0, "rebase": 33}


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


def measure_batched(args, geom_dev, stream, ws, rank, max_over_ranks, sum_over_ranks, barrier):
    """Batched concentrator study: 64 Bezier-cone variants x 41 incidence angles
    (0-40 deg) x photons per group generated on the device, all in ONE
    persistent launch, replayed from a captured CUDA graph; launch shape from
    the autotuner.  Metric: photon-bounces/s; result: collection efficiency per
    (variant, angle)."""
    import torch
    import paper_1508_07803_gb300 as robast
    from paper_1508_07803_gb300 import autotune

    scene, groups = W.cone_batch(n_variants=64, angles_deg=W.CONE_ANGLES_DEG,
                                 n_per_group=args.batch_photons_per_group, seed=0)
    geom = robast.build_geometry(scene)
    (block, bps), table = autotune.tune_sources(geom, groups, precision=32, max_bounces=30, stream=stream)
    src = robast.sources_create(geom, groups)
    counts = torch.zeros((src.n_groups, 8), dtype=torch.int64, device=geom_dev)
    first_id = rank * src.n_photons

    # capture on a side stream (graphs cannot be captured on the default stream)
    cap = torch.cuda.Stream(device=geom_dev)
    cap.wait_stream(stream)
    with torch.cuda.stream(cap):
        robast.trace_sources(geom, src, counts, seed=0, precision=32, max_bounces=30, stream=cap,
                             first_photon_id=first_id, block_size=block, blocks_per_sm=bps)  # warm-up
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=cap):
            robast.trace_sources(geom, src, counts, seed=0, precision=32, max_bounces=30, stream=cap,
                                 first_photon_id=first_id, block_size=block, blocks_per_sm=bps)
    graph.replay()  # warm-up replay
    torch.cuda.synchronize()
    counts.zero_()
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
    src.close()
    geom.close()
    return {"value": bounces / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / args.batch_steps,
            "steps": args.batch_steps, "photons_per_step": src.n_photons,
            "bounces_per_step": bounces / args.batch_steps / ws,
            "config": {"workload": "hex_bezier_cone_64_variants_x_41_angles", "variants": 64,
                       "angles_deg": [0, 40, 1], "photons_per_group": args.batch_photons_per_group,
                       "max_bounces": 30, "sources": "generated on the device (Philox stream 1)",
                       "launch": "one persistent launch per step, replayed from a CUDA graph"},
            "autotune": {"block": block, "blocks_per_sm": bps,
                         "candidates_ms": {f"{b}x{p}": round(t, 3) for (b, p), t in table.items()}},
            "collection_efficiency": summary}


def measure_tolerance(args, dev, stream, ws, rank, max_over_ranks, sum_over_ranks, barrier):
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
    out = robast.alloc_outputs(b.n, 32, dev, fields=("status", "bounces", "focal_xy", "counters"))
    wins = [(k * m, m) for k in range(nr)]

    def step():
        robast.trace(geom, o, d, w, seed=0, variant_of_photon=v, out=out, stream=stream,
                     first_photon_id=rank * b.n)
        return robast.psf(geom, out["status"], out["focal_xy"], windows=wins, stream=stream)

    for _ in range(3):
        step()
    out["counters"].zero_()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    steps = 5
    t0.record(stream)
    for _ in range(steps):
        res = step()
    t1.record(stream)
    barrier()
    ms = max_over_ranks(t0.elapsed_time(t1))
    bounces = sum_over_ranks(float(out["counters"][0].item()))
    r80 = np.array([r[3] for r in res])
    geom.close()
    return {"value": bounces / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "photons_per_step": int(b.n),
            "r80_m": {"mean": float(r80.mean()), "std": float(r80.std()), "min": float(r80.min()),
                      "max": float(r80.max())},
            "config": {"workload": "lst_tolerance_64_realisations_tilt_0.5mrad", "realisations": nr,
                       "photons_per_realisation": m, "field_deg": 1.0}}


def measure_grad(args, dev, stream, ws, rank, max_over_ranks, barrier):
    """Differentiable batch: 32 LST-like dishes with 60-198 facets, 1e6
    photons each over field angles 0-2 deg, one evaluation = the summed
    mean-squared spot radius of the 32 dishes AND its gradient with respect to
    every facet's two tilts and eight aspheric coefficients, in one launch
    (FP32 trace, FP64 dual re-intersection and sums).  Dish v is lit at the
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
                                 stream=stream, out=g)

    for _ in range(2):
        evaluate()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.grad_steps):
        value, _, info = evaluate()
    barrier()
    dt = max_over_ranks(time.perf_counter() - t0)
    gn = float(torch.linalg.vector_norm(g).item())
    geom.close()
    return {"value": ws * args.grad_steps / dt, "unit": "grad evals/s", "ms_per_eval": 1e3 * dt / args.grad_steps,
            "photons_per_eval": int(b.n), "photons_per_s": ws * args.grad_steps * b.n / dt,
            "objective": "sum over 32 dishes of the mean-squared spot radius (frozen path, expected weights)",
            "objective_value_m2": value, "gradient_norm": gn, "n_params": int(geom.n_surfaces * robast.N_PARAM),
            "n_detected": int(info["n_detected"]), "untracked_photons": int(info["n_untracked"]),
            "config": {"workload": "dish_batch_32_dishes_60_to_198_facets", "facets": [counts[0], counts[-1]],
                       "photons_per_dish": args.grad_photons_per_dish, "field_angle_deg": "2 v / 31 for dish v",
                       "timing": "host wall clock around the synchronous call (value returned to the host)"}}


TRAFFIC_SOURCES = ("trace.cuh", "order.cu")  # the kernel and the processing order that shapes its DRAM traffic


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--photons-per-angle", type=int, default=10_000_000)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--ref-photons-per-angle", type=int, default=20_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-tolerance", action="store_true")
    ap.add_argument("--grad-photons-per-dish", type=int, default=1_000_000)
    ap.add_argument("--grad-steps", type=int, default=3)
    ap.add_argument("--batch-photons-per-group", type=int, default=2_000_000)
    ap.add_argument("--batch-steps", type=int, default=2)
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

    npa = args.photons_per_angle
    N = npa * len(ANGLES)
    scene, bundle = W.lst_workload(npa, seed=rank)
    geom = robast.build_geometry(scene)
    first_id = shard.replica_first_id(rank, N)
    stream = torch.cuda.current_stream(dev)

    def inputs(precision):
        dt = torch.float32 if precision == 32 else torch.float64
        return (torch.from_numpy(bundle.origins).to(dev, dt), torch.from_numpy(bundle.dirs).to(dev, dt),
                torch.from_numpy(bundle.wavelengths).to(dev, dt))

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return shard.all_reduce_scalar(x, "max", device=dev)

    def sum_over_ranks(x):
        return shard.all_reduce_scalar(x, "sum", device=dev)

    def measure(precision, steps, warmup, want_clocks):
        o, d, w = inputs(precision)
        # per-photon outputs the spot diagram and the metric need: status, bounce count, focal (x, y)
        out = robast.alloc_outputs(N, precision, dev, fields=("status", "bounces", "focal_xy", "counters"))
        counters = out["counters"]
        # per step: the coherent-order sort (init, bounds, count, columns, three scan launches, place), the
        # trace, and the reduction (sums, finish, histogram, pick, compact, check, candidate r^2,
        # sub-histogram, pick, collect, select; all angles at once)
        order_launches, psf_launches = 8, 11

        def step(ev=None):
            if ev is not None:
                ev[0].record(stream)
            robast.trace(geom, o, d, w, seed=0, precision=precision, first_photon_id=first_id, out=out,
                         stream=stream)
            if ev is not None:
                ev[1].record(stream)
            return robast.psf(geom, out["status"], out["focal_xy"], precision=precision, stream=stream,
                              windows=[(k * npa, npa) for k in range(len(ANGLES))])

        for _ in range(warmup):
            step()
        # work units of one launch (counting build, outside the timed region)
        units = torch.zeros(robast.N_UNITS, dtype=torch.int64, device=dev)
        robast.trace(geom, o, d, w, seed=0, precision=precision, first_photon_id=first_id, out=out,
                     stream=stream, work_units=units, block_size=128)
        torch.cuda.synchronize()
        units = dict(zip(robast.UNIT_NAMES, units.cpu().tolist()))
        counters.zero_()
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
        clk = clocks.stop() if clocks else None
        c = counters.cpu().tolist()
        bounces = c[0]
        return {"ms": ms, "kernel_ms": kern_ms, "bounces": bounces, "counters": c, "units": units, "psf": last,
                "clocks": clk, "launches": steps * (order_launches + 1 + psf_launches)}

    fp32 = measure(32, args.steps, args.warmup, want_clocks=True)
    ms = max_over_ranks(fp32["ms"])
    bounces_all = sum_over_ranks(fp32["bounces"])
    value = bounces_all / (ms * 1e-3)
    kern_avg_ms = statistics.mean(fp32["kernel_ms"])

    # ALU roofline of the trace kernel (FP32 FMA peak measured on this device)
    peak32 = robast.measure_alu_peak(32)
    flops = sum(fp32["units"][k] * UNIT_FLOPS[k] for k in UNIT_FLOPS)
    achieved = flops / (kern_avg_ms * 1e-3)
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak32 / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak32, "traffic": traffic_from_profile(N),
            "kernel": "robast::trace_kernel<float,512> (with the coherent-order sort)", "kernel_ms": kern_avg_ms,
            "flops_per_launch": flops, "work_units_per_launch": fp32["units"],
            "peak_source": "FFMA throughput probe robast_measure_alu_peak on this GPU (measured)"}

    forms = {"fp32": {"value": value, "ms_per_step": ms / args.steps, "kernel_ms": kern_avg_ms,
                      "bounces_per_step": bounces_all / args.steps / ws}}
    if not args.no_fp64:
        fp64 = measure(64, args.fp64_steps, 3, want_clocks=False)
        ms64 = max_over_ranks(fp64["ms"])
        v64 = sum_over_ranks(fp64["bounces"]) / (ms64 * 1e-3)
        k64 = statistics.mean(fp64["kernel_ms"])
        peak64 = robast.measure_alu_peak(64)
        fl64 = sum(fp64["units"][k] * UNIT_FLOPS[k] for k in UNIT_FLOPS)
        forms["fp64"] = {"value": v64, "ms_per_step": ms64 / args.fp64_steps, "kernel_ms": k64,
                         "roofline": {"bound": "alu", "achieved": fl64 / (k64 * 1e-3) / 1e12, "peak": peak64 / 1e12,
                                      "unit": "TFLOP/s", "frac": fl64 / (k64 * 1e-3) / peak64,
                                      "peak_source": "DFMA throughput probe (measured)"}}

    if not args.no_batched:
        forms["batched_fp32"] = measure_batched(args, geom_dev=dev, stream=stream, ws=ws, rank=rank,
                                                max_over_ranks=max_over_ranks, sum_over_ranks=sum_over_ranks,
                                                barrier=barrier)

    if not args.no_tolerance:
        forms["tolerance_fp32"] = measure_tolerance(args, dev=dev, stream=stream, ws=ws, rank=rank,
                                                    max_over_ranks=max_over_ranks, sum_over_ranks=sum_over_ranks,
                                                    barrier=barrier)

    if not args.no_grad:
        forms["grad_fp32"] = measure_grad(args, dev=dev, stream=stream, ws=ws, rank=rank,
                                          max_over_ranks=max_over_ranks, barrier=barrier)

    e2e = None
    if not args.no_e2e:
        dt = torch.float32
        ho = torch.from_numpy(bundle.origins).to(dt).pin_memory()
        hd = torch.from_numpy(bundle.dirs).to(dt).pin_memory()
        hw = torch.from_numpy(bundle.wavelengths).to(dt).pin_memory()
        hout = {"status": torch.empty(N, dtype=torch.uint8).pin_memory(),
                "bounces": torch.empty(N, dtype=torch.uint8).pin_memory(),
                "focal_xy": torch.empty((2, N), dtype=dt).pin_memory(),
                "counters": torch.zeros(robast.N_COUNTERS, dtype=torch.int64)}
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
        e2e = {"value": eb / et, "unit": UNIT, "h2d_bytes_per_step": int(N * 7 * 4),
               "d2h_bytes_per_step": int(N * (1 + 1 + 2 * 4)), "steps": e2e_steps,
               "api": "robast_trace_host (pinned host buffers in and out)"}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate()
    psf = [{"field_deg": a, "n_detected": int(p[0]), "cx_m": p[1], "cy_m": p[2], "r80_m": p[3],
            "a_eff_m2": p[0] / npa * math.pi * 12.0 ** 2} for a, p in zip(ANGLES, fp32["psf"])]
    cfg = workload_config(npa)
    cfg["parallelism"] = f"replicas{ws}" if ws > 1 else "single"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg, "forms": forms,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": fp32["launches"],
            "clocks": fp32["clocks"], "psf": psf,
            "status_counts_per_step": [c // args.steps for c in fp32["counters"][1:7]]}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
