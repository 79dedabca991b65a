#!/usr/bin/env python3
"""Benchmark: 64-right-hand-side mat-vecs of the layered multiple-scattering operator.

Workload: 10^4 particles (enclosing radius U[0.2, 0.5], packing fraction 0.2; half discs, half stars
r(t) = a (1 + 0.2 cos 5t) of 16 quantised sizes x 2 boundary conditions with random rotations),
omega = 6, expansion order p = 20, N_S = 4800 Sommerfeld nodes on the contour adapted to the cloud's
width, 64 right-hand sides (synthetic, seeded).  The 32 star prototype matrices are seeded dense
stand-ins with the order profile of small-particle scattering matrices (synthetic.surrogate_tables):
the mat-vec's work does not depend on their values.  A step is one application y = x - S (T + R) x of the
whole hot path (precision staging, near-pair translation, FMM far field, multipole-to-Sommerfeld,
reflection, Sommerfeld-to-local, scattering-matrix apply) to the 64-column block, with the FP32
operator on the tensor cores (--no-tensor-cores: CUDA cores).  `value` is mat-vecs per second over
all ranks with inputs resident in HBM; `e2e` repeats the step through the same C-ABI call with the
block copied host->device and the result device->host inside the timed region.  Inputs (0.84 GB)
exceed the 126 MB L2.

Multi-GPU: right-hand-side blocks are independent, so each rank applies the operator to its own
64-column block with no collective (weak scaling, replicas of the geometry).

--impl reference times the FP64 CPU oracle on this host on a bounded sample of the same
mat-vec (a few target particles of the direct sum plus the full spectral part) and extrapolates
to one full mat-vec.  --mode solve times solves to 1e-8 (mixed, and FP64 with --full-fp64);
--mode grad times gradient evaluations of the inverse-scattering workload; --profile runs a small
case for ncu.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "matvecs/s (2D N=1e4, 64 RHS, mixed FP32 operator)"
UNIT = "matvec/s"


def star_tables(wl, seed: int = 77):
    """Seeded stand-in prototype matrices for timing: row/column order profile (k_b R_q / 2)^|n| / |n|!
    with R_q the prototype's enclosing radius and k_b the lower layer's wavenumbers."""
    import synthetic as syn
    if wl.n_proto == 0:
        return None
    kp = wl.omega / math.sqrt(wl.media.lam_l + 2 * wl.media.mu_l)
    ks = wl.omega / math.sqrt(wl.media.mu_l)
    R = wl.proto_shape[:, 0] + wl.proto_shape[:, 1]
    ratio = np.stack([kp * R / 2, ks * R / 2], 1)
    return syn.surrogate_tables(seed, ratio, wl.p)


def workload():
    import synthetic as syn
    wl = syn.config3()
    return wl, star_tables(wl)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(wl, tables, targets: int, nrhs: int, spectral_cols: int = 8):
    """Time the FP64 oracle on `targets` target particles of the direct translation sum (nrhs
    columns) and on the full spectral part (multipole-to-Sommerfeld, reflection, Sommerfeld-to-local)
    for `spectral_cols` columns; extrapolate linearly to one full 64-column mat-vec.
    Returns (matvecs/s, cores, sample text, quadrature nodes of the oracle's rule)."""
    import synthetic as syn
    from oracle import system
    ref = system.Problem(wl, proto_S=tables)
    x = syn.random_coeffs(99, wl.M, wl.p, nrhs)
    idx = list(range(targets))
    t0 = time.perf_counter()
    ref.apply_S(ref.translate(x, targets=idx), targets=idx)
    t1 = time.perf_counter()
    ref.reflect(x[..., :spectral_cols], targets=idx)
    t2 = time.perf_counter()
    t_full = (t1 - t0) / targets * wl.M * (64 / nrhs) + (t2 - t1) * (64 / spectral_cols)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = (f"oracle FP64 numpy/scipy: direct Graf sum and scattering-matrix apply for {targets} of {wl.M} "
              f"targets with {nrhs} columns "
              f"and the full spectral part with {spectral_cols} columns, extrapolated linearly to one "
              f"64-column mat-vec ({t1 - t0:.1f} s + {t2 - t1:.1f} s measured)")
    return 1.0 / t_full, cores, sample, len(ref.xi)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl, tables = workload()
    vals = []
    cores = 0
    sample = ""
    nodes = 0
    # warm-up steps run the same oracle code on a minimal sample (one target, one spectral column):
    # they only bring the code and the tables in; the timed steps are the full bounded samples
    for _ in range(args.warmup):
        oracle_sample(wl, tables, targets=1, nrhs=8, spectral_cols=1)
    for _ in range(max(args.steps, 1)):
        v, cores, sample, nodes = oracle_sample(wl, tables, targets=2, nrhs=64)
        vals.append(v)
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "M": wl.M, "p": wl.p, "nrhs": 64,
                                            "n_nodes": nodes},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "projected": True,
            "projection": ("value and ms_per_step are projected linearly from each step's bounded sample to one "
                           "full 64-column mat-vec; the run itself lasts steps x the sample's time")}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2608_26875_b300 as P
    import synthetic as syn

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    wl, tables = workload()
    prec = P.MS_PREC_FP32 if args.prec == "fp32" else P.MS_PREC_FP64
    solver = P.Solver.from_workload(wl, proto_S=tables, leaf_target=args.leaf_target,
                                    tensor_cores=args.tensor_cores, store_near=args.store_near)
    stored = solver.near_stored_bytes()
    nrhs = 64
    x = torch.as_tensor(syn.random_coeffs(1000 + rank, wl.M, wl.p, nrhs), device="cuda")
    y = torch.empty_like(x)
    st = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        solver.apply(x, prec=prec, out=y)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(st)
        for _ in range(args.steps):
            solver.apply(x, prec=prec, out=y)
        ev1.record(st)
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    t = torch.tensor([ms], device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    value = world / (ms / 1000.0)

    # per-part times through the operator-parts view (each call also runs the two staging passes):
    # near-pair Graf sum, FMM far field, and the layered part (M2S, reflect, S2L)
    def part_time(parts):
        solver.operator(x, parts, prec=prec)
        torch.cuda.synchronize()
        n = max(1, min(args.steps, 3))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(n):
            solver.operator(x, parts, prec=prec)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n / 1000.0

    t_near = part_time(P.MS_PART_T_NEAR)
    t_far = part_time(P.MS_PART_T_FAR) if solver.fmm_levels else 0.0
    t_refl = part_time(P.MS_PART_R)
    t_sapply = part_time(P.MS_PART_S)
    pairs = solver.near_pairs
    work = solver.work()                                              # complex MACs per column, by part
    flops_near = work["near"] * nrhs * 8.0                            # complex MAC = 8 real flops
    flops_far = work["far"] * nrhs * 8.0
    flops_refl = work["refl"] * nrhs * 8.0
    pk, src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2032.0))
    fp32_peak = 148 * 128 * 2 * sm_max * 1e6 / 1e12                  # TFLOP/s of the FP32 CUDA-core pipes
    tf32_peak = float(pk.get("bf16_tflops", 1800.0)) * 0.5             # dense TF32 = bf16 x 1.1/2.25 (nominal)
    tc = args.tensor_cores and prec == P.MS_PREC_FP32
    near_kernel = ("k_list_stored (stored 3xTF32 tiles by cp.async.bulk, tcgen05 kind::tf32) near pairs"
                   if stored else "k_list_tc (tcgen05 kind::tf32, 3xTF32) near pairs")
    cand = [("near", t_near, flops_near, near_kernel if tc else "k_translate<float> near pairs"),
            ("refl", t_refl, flops_refl,
             "k_m2s_tc + k_reflect + k_s2l_tc (tcgen05 kind::tf32, 3xTF32)" if tc else "k_m2s + k_reflect + k_s2l")]
    name, t_dom, flops_dom, kname = max(cand, key=lambda c: c[1])
    achieved = flops_dom / t_dom / 1e12
    part_peak = tf32_peak if tc else fp32_peak
    if tc:
        peak, bound = tf32_peak, "tensor"
        peak_src = f"TF32 dense = measured bf16 {pk.get('bf16_tflops')} TFLOP/s x 0.5 (nominal ratio); {src}"
    else:
        peak, bound = fp32_peak, "alu"
        peak_src = f"148 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz ({src} clock)"
    hbm_peak = float(pk.get("hbm_gbs", 6400.0))
    # stored near tiles: one pass over them per application, plus the FP32 staged block in and out
    near_bytes = stored + 2 * wl.M * 2 * (2 * wl.p + 1) * nrhs * 8 if (tc and stored) else None
    if name == "near" and near_bytes and near_bytes / t_dom / 1e9 / hbm_peak > achieved / peak:
        achieved, peak, bound = near_bytes / t_dom / 1e9, hbm_peak, "hbm"
        peak_src = f"measured HBM copy {hbm_peak} GB/s ({src})"
    traffic = None
    tpath = os.path.join(ROOT, "profiles", f"{name}_traffic.json")
    if os.path.exists(tpath):
        traffic = json.load(open(tpath)).get("bytes_per_launch")

    # end to end: host block in, host block out, through the same call
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    xd = torch.empty_like(x)
    ev4 = torch.cuda.Event(enable_timing=True)
    ev5 = torch.cuda.Event(enable_timing=True)
    ne = max(1, min(args.steps, 3))
    barrier()
    ev4.record(st)
    for _ in range(ne):
        xd.copy_(xh, non_blocking=True)
        solver.apply(xd, prec=prec, out=y)
        yh.copy_(y, non_blocking=True)
    ev5.record(st)
    barrier()
    e2e_ms = ev4.elapsed_time(ev5) / ne
    te = torch.tensor([e2e_ms], device="cuda")
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_val = world / (float(te.item()) / 1000.0)
    nbytes = x.numel() * 16

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, _ = oracle_sample(wl, tables, targets=2, nrhs=64)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if prec == P.MS_PREC_FP32 else "f64", "data": "synthetic",
                "config": {"workload": wl.name, "M": wl.M, "p": wl.p, "nrhs": nrhs,
                           "stars": int((wl.proto >= 0).sum()), "prototypes": wl.n_proto,
                           "n_nodes": solver.n_nodes, "omega": wl.omega,
                           "near_pairs": pairs, "fmm_levels": solver.fmm_levels,
                           "leaf_target": args.leaf_target, "contour_depth": wl.depth,
                           "tensor_cores": bool(args.tensor_cores),
                           "near_stored_gb": stored / 1e9,
                           "l2": "inputs 0.84 GB > 126 MB L2, no flush",
                           "parallelism": f"rhs-replicas x{world}"},
                "roofline": {"bound": bound, "kernel": kname + f" (timed via ms_operator, part {name})",
                             "achieved": achieved, "peak": peak, "unit": "GB/s" if bound == "hbm" else "TFLOP/s",
                             "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                             "flops": "algorithmic complex MACs x 8 (the 3xTF32 split issues 3 MMAs per product)"
                             if tc else "algorithmic complex MACs x 8",
                             "bytes": (f"stored near tiles {stored} B + FP32 block in and out"
                                       if bound == "hbm" else None)},
                "parts_ms": {"near": t_near * 1e3, "far": t_far * 1e3, "refl": t_refl * 1e3,
                             "sapply": t_sapply * 1e3,
                             "note": "each part timed through ms_operator, staging in and out included"},
                "parts_roofline": {
                    k: {"tflops_algorithmic": f / 1e12, "achieved_tflops": (f / t / 1e12) if t > 0 else None,
                        "frac": (f / t / 1e12 / part_peak) if t > 0 else None}
                    for k, t, f in (("near", t_near, flops_near), ("far", t_far, flops_far),
                                    ("refl", t_refl, flops_refl))},
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
                "gpu_launches": launches_per_step(solver, tc) * args.steps,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_solve(args):
    """Time to solution at relative residual 1e-8 for plane-wave right-hand sides at the 10^4-particle
    workload's density (radii U[0.2, 0.5], packing 0.2, omega = 6, p = 20; discs, whose closed-form
    scattering matrices are physical, unlike the stand-in star tables of the mat-vec), with --M particles and
    --nrhs columns: the mixed form (FP32 operator, FP64 refinement) and, with --full-fp64, the FP64
    form, both measured; otherwise the FP64 form is extrapolated from its mat-vec time and the
    mat-vecs the mixed solve needed.  GMRES restart and iteration cap from --restart, --max-iters."""
    import torch

    import paper_2608_26875_b300 as P
    import synthetic as syn
    wl = syn.config3_discs(M=args.M or 10000, nrhs=args.nrhs)
    kinds, angles = wl.inc_kind[:args.nrhs], wl.inc_angle[:args.nrhs]
    if args.far_diag:
        # FP32-vs-FP64 far field on the physical right-hand side b and on the library's test blocks, for
        # tree variants: the default, the CUDA-core M2L, and larger leaves (fewer levels)
        out = []
        for name, kw in (("default", {}), ("cuda-core", {"tensor_cores": False}), ("leaf40", {"leaf_target": 40})):
            sw = P.Solver.from_workload(wl, store_near=0, **kw)
            b = sw.rhs(kinds, angles)
            xr = torch.as_tensor(syn.random_coeffs(7, wl.M, wl.p, len(kinds)), device="cuda")
            row = {"variant": name, "fmm_levels": sw.fmm_levels}
            for lab, v in (("rhs", b), ("random", xr)):
                y64 = sw.operator(v, P.MS_PART_T_FAR, prec=P.MS_PREC_FP64)
                y32 = sw.operator(v, P.MS_PART_T_FAR, prec=P.MS_PREC_FP32)
                row[lab] = float(torch.linalg.norm(y64 - y32) / torch.linalg.norm(y64))
            out.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
            sw.close()
        print(json.dumps({"mode": "far-diag", "workload": wl.name, "rows": out}), flush=True)
        return
    if args.iter_sweep:
        rows = []
        for cap in [int(c) for c in args.iter_sweep.split(",")]:
            sw = P.Solver.from_workload(wl, leaf_target=args.leaf_target, restart=args.restart, max_iters=cap,
                                        precond_group=args.precond_group, store_near=args.store_near)
            xs, inf = sw.solve(kinds, angles, tol=1e-8, prec=P.MS_PREC_FP32)
            # how far the FP32 operator is from the FP64 one on this iterate, part by part
            parts = {"near": P.MS_PART_T_NEAR | P.MS_PART_S, "far": P.MS_PART_T_FAR | P.MS_PART_S,
                     "refl": P.MS_PART_R | P.MS_PART_S, "all": P.MS_PART_T | P.MS_PART_R | P.MS_PART_S}
            disc = {}
            for k, pt in parts.items():
                y64 = sw.operator(xs, pt, prec=P.MS_PREC_FP64)
                y32 = sw.operator(xs, pt, prec=P.MS_PREC_FP32)
                disc[k] = float(torch.linalg.norm(y64 - y32) / torch.linalg.norm(y64))
            inf["fp32_vs_fp64_operator_on_iterate"] = disc
            rows.append({"max_iters": cap, **inf})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            sw.close()
        print(json.dumps({"mode": "solve-sweep", "workload": wl.name, "restart": args.restart,
                          "precond_group": args.precond_group, "rows": rows}), flush=True)
        return
    t0 = time.perf_counter()
    s = P.Solver.from_workload(wl, leaf_target=args.leaf_target, tensor_cores=args.tensor_cores,
                               restart=args.restart, max_iters=args.max_iters, inner_tol=args.inner_tol,
                               block_krylov=not args.per_column, precond_group=args.precond_group,
                               store_near=args.store_near)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    g, info = s.solve(kinds, angles, tol=1e-8, prec=P.MS_PREC_FP32)
    torch.cuda.synchronize()
    out = {"mode": "solve", "workload": wl.name, "M": wl.M, "nrhs": len(kinds), "tol": 1e-8,
           "krylov": "per-column GMRES" if args.per_column else "block GMRES over the right-hand sides",
           "restart": args.restart, "max_iters": args.max_iters, "tensor_cores": bool(args.tensor_cores),
           "inner_tol": args.inner_tol or "default", "precond_group": args.precond_group,
           "setup_s": setup_s, "setup_note": "ms_setup incl. tables, tree and the preconditioner's inverses",
           "mixed": info}
    x = torch.empty_like(g)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.apply(g, prec=P.MS_PREC_FP64, out=x)
    torch.cuda.synchronize()
    ev0.record()
    s.apply(g, prec=P.MS_PREC_FP64, out=x)
    ev1.record()
    torch.cuda.synchronize()
    t64 = ev0.elapsed_time(ev1) / 1000.0
    out["fp64_matvec_s"] = t64
    ev0.record()
    s.apply(g, prec=P.MS_PREC_FP32, out=x)
    ev1.record()
    torch.cuda.synchronize()
    out["fp32_matvec_s"] = ev0.elapsed_time(ev1) / 1000.0
    if args.skip_fp64:
        pass
    elif args.full_fp64:
        g64, info64 = s.solve(kinds, angles, tol=1e-8, prec=P.MS_PREC_FP64)
        out["fp64"] = info64
        out["rel_diff_mixed_vs_fp64"] = float(torch.linalg.norm(g - g64) / torch.linalg.norm(g64))
    else:
        out["fp64_extrapolated_s"] = t64 * info["matvecs"]
        out["fp64_extrapolation"] = "FP64 mat-vec time x mat-vecs of the mixed solve"
    print(json.dumps(out), flush=True)


def run_grad(args):
    """Gradients per second on the inverse-scattering workload: 2000 rigid discs, p = 16, omega = 4,
    32 plane P-waves, 128 receivers on y = -0.5.  The data are the receiver fields of the same discs
    with centres moved by N(0, 0.05^2) (synthetic truth); one gradient is the whole evaluation at the
    current centres: ms_setup, the forward solve, the receiver fields, and ms_grad (adjoint solve plus
    the centre, radius and frequency derivatives), both solves to --tol with --restart / --max-iters,
    in the precisions of --grad-prec."""
    import copy

    import torch

    import paper_2608_26875_b300 as P
    import synthetic as syn
    wl = syn.config4() if args.M in (None, 2000) else syn.config4(M=args.M)
    rx = wl.receivers
    truth = copy.deepcopy(wl)
    truth.centres = syn.perturb_centres(wl.centres, wl.radius, 0.05, 3001)
    st = P.Solver.from_workload(truth, restart=args.restart, precond_group=args.precond_group)
    gt, _ = st.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP32)     # refined to 1e-10 in FP64
    d = st.fields(gt, rx)
    st.close()
    out = {"mode": "grad", "workload": wl.name, "M": wl.M, "nrhs": wl.nrhs, "receivers": int(rx.shape[0])}
    precs = {"mixed": [("mixed", P.MS_PREC_FP32)], "fp64": [("fp64", P.MS_PREC_FP64)],
             "both": [("mixed", P.MS_PREC_FP32), ("fp64", P.MS_PREC_FP64)]}[args.grad_prec]
    out.update({"tol": args.tol, "restart": args.restart, "max_iters": args.max_iters,
                "precond_group": args.precond_group})
    for name, prec in precs:
        times = []
        for it in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = P.Solver.from_workload(wl, tensor_cores=args.tensor_cores, restart=args.restart,
                                       max_iters=args.max_iters, precond_group=args.precond_group)
            g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=args.tol, prec=prec)
            u = s.fields(g, rx)
            w = (u - d).contiguous()
            gc, gr, gw, ginfo = s.grad(wl.inc_kind, wl.inc_angle, g, w, rx, tol=args.tol, prec=prec)
            loss = 0.5 * float(torch.sum(torch.abs(w) ** 2))
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            s.close()
            if it >= args.warmup:
                times.append(dt)
        out[name] = {"grads_per_s": len(times) / sum(times), "s_per_grad": sum(times) / len(times),
                     "forward": info, "adjoint": ginfo, "loss": loss,
                     "max_abs_dL_dcentre": float(gc.abs().max()), "dL_domega": gw}
        # each precision's result as soon as it is known (a slow FP64 pass must not hide the mixed one)
        print(json.dumps({"partial": name, **out[name]}), file=sys.stderr, flush=True)
    print(json.dumps(out), flush=True)


def run_3d(args):
    """The 3D workload (Sec. 6): 500 rigid spheres of radius U[0.3, 0.5] in [-15, 15]^2 x [-12, -1], p = 8,
    16 plane waves, polar Sommerfeld rule 128 x 64 with contour depth 3 / (horizontal extent) (the 2D
    reading for wide clouds).  Times the FP64 mat-vec and its parts, then the block-GMRES solve to
    --tol; algorithmic complex multiply-adds per application are counted from the sizes."""
    import torch

    import paper_2608_26875_b300 as P
    import synthetic as syn
    from paper_2608_26875_b300 import _native as nat
    wl = syn.spheres3d(M=args.M or 500)
    ext = float(np.hypot(np.ptp(wl.centres[:, 0]), np.ptp(wl.centres[:, 1])))
    alpha = min(1.0, 3.0 / ext)
    t0 = time.perf_counter()
    s = P.Solver3(wl.centres, wl.radius, wl.bc, wl.media, wl.omega, wl.p, n_r=128, n_theta=64, n_panels=4,
                  t_max=10.0, alpha=alpha, beta=1.0, restart=args.restart, max_iters=args.max_iters)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    nrhs = wl.nrhs
    x = s.rhs(wl.inc_kind, wl.inc_theta, wl.inc_phi)
    y = torch.empty_like(x)

    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n / 1000.0

    n = max(1, args.steps)
    t_all32 = timed(lambda: s.apply(x, prec=P.MS_PREC_FP32, out=y), n)
    t_all = timed(lambda: s.apply(x, out=y), n)
    t_T = timed(lambda: s.operator(x, nat.MS3_PART_T, out=y), n)
    t_R = timed(lambda: s.operator(x, nat.MS3_PART_R, out=y), n)
    p, M, NS = wl.p, wl.M, s.n_nodes
    nl, nmn, K2 = (p + 1) ** 2, p * (p + 2), (p + 2) ** 2
    T = 2 * nmn + nl
    cmac_T = M * (M - 1) * (3 * K2 * nl + nl * nl) * nrhs
    cmac_R = NS * M * (nl + 4 * nmn) * nrhs + M * NS * 3 * T * nrhs
    fp64_peak = 1.13e12           # measured FP64 FMA-chain rate of this GPU (design notes)
    out = {"mode": "3d", "workload": wl.name, "M": M, "p": p, "nrhs": nrhs, "n_nodes": NS, "contour_alpha": alpha,
           "setup_s": setup_s, "matvec_s": t_all, "matvecs_per_s": 1.0 / t_all, "fp32_matvec_s": t_all32,
           "free_space_s": t_T,
           "reflected_s": t_R, "dtype": "f64",
           "roofline": {"bound": "alu", "unit": "TFLOP/s", "peak": fp64_peak / 1e12,
                        "free_space": {"achieved": 8 * cmac_T / t_T / 1e12, "frac": 8 * cmac_T / t_T / fp64_peak},
                        "reflected": {"achieved": 8 * cmac_R / t_R / 1e12, "frac": 8 * cmac_R / t_R / fp64_peak},
                        "flops": "complex MACs of the contractions x 8 (translation-coefficient generation not counted)"}}
    if args.no_solve:
        print(json.dumps(out), flush=True)
        return
    gm, info_m = s.solve(wl.inc_kind, wl.inc_theta, wl.inc_phi, tol=args.tol, prec=P.MS_PREC_FP32)
    out["solve_mixed"] = info_m
    if not args.skip_fp64:
        g, info = s.solve(wl.inc_kind, wl.inc_theta, wl.inc_phi, tol=args.tol)
        out["solve_fp64"] = info
        out["rel_diff_mixed_vs_fp64"] = float(torch.linalg.norm(gm - g) / torch.linalg.norm(g))
    print(json.dumps(out), flush=True)


def launches_per_step(solver, tensor_cores=False):
    """Kernels of one ms_apply: staging in/out, near sum (2 waves; one tensor-core launch for both),
    FMM (per wave: P2M, M2M per level, M2L per level, L2L per level, L2P), M2S, reflect, S2L (plus
    the FP32 amplitude copy on the tensor-core path), S-apply of the discs and of the prototypes."""
    L = solver.fmm_levels
    fmm = 0 if L == 0 else 2 * (1 + (L - 2) + (L - 1) + (L - 2) + 1)
    proto = 1 if getattr(solver, "has_proto", False) else 0
    if tensor_cores:
        return 2 + 1 + fmm + 4 + 1 + proto
    return 2 + 2 + fmm + 3 + 1 + proto


def run_profile(args):
    """Small case for ncu: M particles at the bench's density, 64 columns, `--part` of the operator
    applied `--steps` times (near: direct near-pair sum; far: FMM far field; refl: spectral part;
    all: the whole mat-vec)."""
    import torch

    import paper_2608_26875_b300 as P
    import synthetic as syn
    wl = syn.config3(M=args.M or 2500, nrhs=64)
    prec = P.MS_PREC_FP32 if args.prec == "fp32" else P.MS_PREC_FP64
    s = P.Solver.from_workload(wl, proto_S=star_tables(wl), tensor_cores=args.tensor_cores,
                               store_near=args.store_near)
    x = torch.as_tensor(syn.random_coeffs(5, wl.M, wl.p, 64), device="cuda")
    parts = {"near": P.MS_PART_T_NEAR, "far": P.MS_PART_T_FAR, "refl": P.MS_PART_R | P.MS_PART_S,
             "sapply": P.MS_PART_S}
    for _ in range(args.steps):
        if args.part == "all":
            s.apply(x, prec=prec)
        else:
            s.operator(x, parts[args.part], prec=prec)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.part, "M": wl.M, "near_pairs": s.near_pairs, "fmm_levels": s.fmm_levels}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true", help="small case for ncu (see run_profile)")
    ap.add_argument("--mode", choices=["matvec", "solve", "grad", "3d"], default="matvec")
    ap.add_argument("--full-fp64", action="store_true", help="solve mode: run the FP64 solve too")
    ap.add_argument("--part", choices=["near", "far", "refl", "sapply", "all"], default="near")
    ap.add_argument("--M", type=int, default=None, help="particles: --profile (default 2500), --mode solve "
                    "(default 10000), --mode grad (default 2000, the inverse-scattering workload)")
    ap.add_argument("--nrhs", type=int, default=64, help="--mode solve: right-hand sides")
    ap.add_argument("--restart", type=int, default=50, help="--mode solve/grad: GMRES restart length (block "
                    "iterations with block GMRES)")
    ap.add_argument("--per-column", action="store_true", help="--mode solve: one Krylov space per column "
                    "instead of block GMRES")
    ap.add_argument("--max-iters", type=int, default=2000, help="--mode solve/grad: GMRES iteration cap")
    ap.add_argument("--tol", type=float, default=1e-8, help="--mode grad: solve tolerance")
    ap.add_argument("--inner-tol", type=float, default=0.0, help="--mode solve: inner GMRES tolerance (0: default)")
    ap.add_argument("--skip-fp64", action="store_true", help="--mode solve: mixed form only")
    ap.add_argument("--no-solve", action="store_true", help="--mode 3d: mat-vec timings only")
    ap.add_argument("--far-diag", action="store_true", help="--mode solve: FP32-vs-FP64 far-field discrepancy")
    ap.add_argument("--iter-sweep", type=str, default="", help="--mode solve: comma-separated iteration caps; "
                    "reports the mixed solve's FP64 residual after each cap (a fresh handle per cap)")
    ap.add_argument("--grad-prec", choices=["mixed", "fp64", "both"], default="mixed")
    ap.add_argument("--leaf-target", type=int, default=10, help="FMM particles per leaf box")
    ap.add_argument("--precond-group", type=int, default=0, help="--mode solve/grad: particles per block of the "
                    "group-block Jacobi preconditioner (0: none)")
    ap.add_argument("--store-near", type=int, default=96, help="device GB budget for the stored near-pair "
                    "operator tiles (0: generated in every application; the 10^4-particle workload stores 48 GB)")
    ap.add_argument("--no-tensor-cores", dest="tensor_cores", action="store_false",
                    help="FP32 near field and spectral maps on the CUDA cores instead of tcgen05")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
    elif args.mode == "solve":
        run_solve(args)
    elif args.mode == "grad":
        run_grad(args)
    elif args.mode == "3d":
        run_3d(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
