"""Benchmark of the matrix-free ghost-penalty apply y = G x on GB300.

Workload: 3D ball of radius 0.7 (seeded centre offset) in a 64^3 Cartesian mesh
on [-1,1]^3, FE_Q(3) on Gauss-Lobatto points, gamma = 0.5 for every order;
x ~ U[-1,1] on the active DoFs.  One step = one y = G x over all ghost faces.

Metric: GDoF/s = active DoFs / apply time (the paper's throughput convention,
Sec. 3.1), whole job over all ranks.  The inputs (about 12 MB) fit in L2, so
a 512 MB buffer is written between timed steps to flush it.

Arms
  default            the CUDA path through the C ABI: FP64-accuracy headline (float-float
                     arithmetic on FP64 data), native FP64 and FP32 beside it
  --impl reference   the CPU FP64 oracle timed on the host cores (bounded sample)

Multi-GPU: one independent replica per rank (the single-problem apply does not
shard); value = DoFs of all ranks / max over ranks of the device time.
"""
from __future__ import annotations

import argparse
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

METRIC = "ghost-penalty GDoF/s & %HBM roofline, FP64 vs FP32/batched at stated error"
WORKLOAD = "ghost-penalty y=Gx, 3D ball r=0.7 in 64^3 cells on [-1,1]^3, FE_Q(3) Gauss-Lobatto, gamma=0.5"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 / FP32 FMA issue rates of a GB300 SM (flop per clock, FMA = 2) at the 2070 MHz maximum SM clock
FP64_FLOP_PER_CLK_SM = 4
FP32_FLOP_PER_CLK_SM = 256
N_SM = 152
SM_MAX_MHZ = 2070.0
# FP32 instructions per float-float multiply-add term of a compensated dot product: the exact
# product (4) plus the two-sum into the running sum (6) plus the error accumulation (2)
FF_OPS_PER_FMA = 12.0


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


KERNEL_SOURCES = ["paper_2503_00246_gb300/csrc/gp_kernels.cuh", "paper_2503_00246_gb300/csrc/gp_arith.cuh",
                  "paper_2503_00246_gb300/csrc/gp_launch.h", "paper_2503_00246_gb300/csrc/gp_plan.cpp"]


def _traffic(tag):
    """DRAM bytes per face-kernel launch from the committed ncu summary, or None when the
    kernel sources changed since those counters were taken."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    try:
        txt = open(os.path.join(ROOT, "profiles", "face_kernel_ball64_k3.md")).read()
    except OSError:
        return None
    m = re.search(r"kernel_sources_sha256_16 = (\w+)", txt)
    t = re.search(r"traffic_bytes_per_launch\[" + re.escape(tag) + r"\] = (\d+)", txt)
    if not m or not t or m.group(1) != h.hexdigest()[:16]:
        return None
    return int(t.group(1))


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [s.strip() for s in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm --

def _flops_face(d, k, nf):
    """Flops the face kernel executes (a multiply-add counts 2, a multiply or add 1; an
    n-term dot product 2n - 1), per normal line: the even-odd split (2k adds), the k
    jump dot products (k + 1 terms for odd orders, k for even ones), (d-1) tangential
    passes of k (k+1)-term dot products, k scalings, and the expansion (per node b <= k
    one odd-order and, for b < k, one even-order partial sum, plus 2 adds)."""
    L = (k + 1) ** (d - 1)
    n_odd, n_even = (k + 1) // 2, k // 2            # orders j = 1, 3, ... and j = 2, 4, ...
    contraction = 2 * k + n_odd * (2 * (k + 1) - 1) + n_even * (2 * k - 1)
    tangential = (d - 1) * k * (2 * (k + 1) - 1)
    expansion = (k + 1) * (2 * n_odd - 1)
    if k > 1:
        expansion += k * ((2 * n_even - 1) + 2)
    per_line = contraction + tangential + k + expansion
    return float(nf) * L * per_line


def _flops_paper(d, k, nf):
    return 2.0 * nf * ((k + 1) ** (d - 1) * (2 * k + 1) ** 2 + (d - 1) * (k + 1) ** d * (2 * k + 1))


WORKLOADS = {
    "ball64_k3": lambda W: W.ball_3d(),
    "disc32_k2": lambda W: W.disc_2d(),
    "gyroid128_k4": lambda W: W.gyroid_3d(),
    **{f"ball96_k{k}": (lambda W, k=k: W.ball_3d_sweep(k)) for k in range(1, 9)},
}


def run_profile(args):
    """A few untimed applies of one workload and precision: the command ncu captures."""
    import torch

    from paper_2503_00246_gb300 import build as B
    B.build()
    from paper_2503_00246_gb300 import gp, workloads as W
    pr = WORKLOADS[args.workload](W)
    prec = {"fp64": gp.GP_FP64, "fp32": gp.GP_FP32, "ff": gp.GP_FP64_FF, "both": gp.GP_FP64_FF}[args.precision]
    ctx = gp.setup_problem(pr, precision=prec, device=0)
    tdt = torch.float32 if prec == gp.GP_FP32 else torch.float64
    x = torch.tensor(W.x_vectors(pr, ctx.n_active)[0], dtype=tdt, device="cuda")
    y = torch.empty_like(x)
    tiles = gp.gp_autotune(ctx, args.tune_reps)[0] if args.tune_reps > 0 else gp.gp_get_tiles(ctx)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")     # ncu --nvtx --nvtx-include "timed/" skips the tuning
    for _ in range(args.reps):
        gp.gp_apply(ctx, x, y)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"workload": args.workload, "precision": args.precision, "n_active": ctx.n_active,
                      "n_faces": ctx.n_faces, "n_touched": ctx.n_touched, "applies": args.reps,
                      "tiles": tiles}))


def run_batched(gp, W, torch, dev, prec, steps, warmup, tune_reps=0):
    """The batched workload: 64 independent 3D ball problems, n ~ U{16..96}, k ~ U{2..6},
    4 right-hand sides each, replayed as one CUDA graph per apply.  Inputs (> 7 GB) exceed L2.
    With tune_reps > 0 the tile shape of every degree is tuned on that degree's largest
    problem and used by the whole group."""
    probs = W.batched_3d()
    nrhs = 4
    ctxs = [gp.setup_problem(p, precision=prec, device=dev.index or 0) for p in probs]
    tuned = {}
    if tune_reps > 0:
        by_k = {}
        for p, c in zip(probs, ctxs):
            by_k.setdefault(p.degree, []).append(c)
        for k in sorted(by_k):
            big = max(by_k[k], key=lambda c: c.n_faces)
            t, _ = gp.gp_autotune(big, tune_reps)
            for c in by_k[k]:
                gp.gp_set_tiles(c, t)
            tuned[str(k)] = t
    batch = gp.gp_batch_create(ctxs, nrhs)
    tdt = torch.float32 if prec == gp.GP_FP32 else torch.float64
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.BASE_SEED + 5000)
    xs = [torch.rand(nrhs * c.n_active, generator=gen, dtype=tdt, device=dev) * 2 - 1 for c in ctxs]
    ys = [torch.empty_like(x) for x in xs]
    for _ in range(warmup):
        gp.gp_batch_apply(batch, xs, ys)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        gp.gp_batch_apply(batch, xs, ys)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / steps
    units = nrhs * sum(c.n_active for c in ctxs)
    ngroups, scratch = gp.gp_batch_info(batch)
    out = {"value": units / (t * 1e-3) / 1e9, "unit": "GDoF/s", "ms_per_apply": t,
           "problems": len(probs), "rhs": nrhs, "dof_vectors_per_apply": units,
           "ghost_faces": sum(c.n_faces for c in ctxs), "kernel_groups": ngroups,
           "graph_launches_per_apply": 1, "kernels_per_apply": 2 * ngroups,
           "scratch_bytes": scratch, "tiles_per_degree": tuned or None}
    batch.close()
    for c in ctxs:
        c.close()
    del xs, ys
    torch.cuda.empty_cache()
    return out


def run_sweep(args):
    """The degree sweep: 96^3 cells on [-1,1]^3, ball of radius 0.7, k = 1..8, y = G x in the
    three arithmetic forms (tile shapes tuned first), L2 flushed between timed applies.
    Reports GDoF/s, ghost faces/s, the face kernel's executed and the paper's flop rates
    against each form's ALU peak, the apply's algorithmic HBM bytes/s, and the relative error
    against the FP64 oracle (full oracle apply for k <= --sweep-check-kmax)."""
    import torch

    from paper_2503_00246_gb300 import build as B
    B.build()
    from paper_2503_00246_gb300 import gp, workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks, peak_src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    fp64_peak = N_SM * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    fp32_peak = N_SM * FP32_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    peak = {gp.GP_FP64: fp64_peak, gp.GP_FP32: fp32_peak, gp.GP_FP64_FF: fp32_peak / FF_OPS_PER_FMA}
    tags = {gp.GP_FP64_FF: "ff64", gp.GP_FP64: "fp64", gp.GP_FP32: "fp32"}
    names = args.sweep_workloads.split(",") if args.sweep_workloads else \
        [f"ball96_k{int(v)}" for v in args.sweep_k.split(",")]
    out = {"workload": "96^3 cells on [-1,1]^3, ball r = 0.7 (seeded centre offset), gamma = 0.5 for every order"
                       if not args.sweep_workloads else "see the keys",
           "peaks_tflops": {tags[p]: peak[p] for p in peak}, "hbm_gbs": hbm, "hbm_source": peak_src, "k": {}}
    stream = torch.cuda.current_stream()
    for name in names:
        pr = WORKLOADS[name](W)
        k = pr.degree
        rec = {}
        ref = ref32 = None
        for prec in (gp.GP_FP64_FF, gp.GP_FP64, gp.GP_FP32):
            ctx = gp.setup_problem(pr, precision=prec, device=0)
            tiles = gp.gp_autotune(ctx, args.tune_reps)[0] if args.tune_reps > 0 else gp.gp_get_tiles(ctx)
            tdt = torch.float32 if prec == gp.GP_FP32 else torch.float64
            x_np = W.x_vectors(pr, ctx.n_active)[0]
            x = torch.tensor(x_np, dtype=tdt, device=dev)
            y = torch.empty_like(x)
            for _ in range(3):
                gp.gp_apply(ctx, x, y)
            nsteps = args.sweep_steps
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
            torch.cuda.synchronize()
            for i in range(nsteps):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                gp.gp_apply(ctx, x, y)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            gp.gp_profile_enable(ctx, True)        # per-kernel split, in separate traced steps
            for i in range(nsteps):
                flush.fill_(float(i))
                gp.gp_apply(ctx, x, y)
            torch.cuda.synchronize()
            ms_face, ms_lift, calls = gp.gp_profile_read(ctx)
            gp.gp_profile_enable(ctx, False)
            t = sum(a.elapsed_time(b) for a, b in ev) / nsteps * 1e-3
            tf = ms_face / calls * 1e-3
            nf = ctx.n_faces
            w = 4 if prec == gp.GP_FP32 else 8
            fl_exec, fl_paper = _flops_face(pr.dim, k, nf), _flops_paper(pr.dim, k, nf)
            r = {"gdofs": ctx.n_active / t / 1e9, "ms": t * 1e3, "face_ms": tf * 1e3, "lift_ms": ms_lift / calls,
                 "gfaces_per_s": nf / t / 1e9,
                 "face_tflops_executed": fl_exec / tf / 1e12, "face_frac_of_peak": fl_exec / tf / 1e12 / peak[prec],
                 "paper_flops_tflops": fl_paper / t / 1e12,
                 "apply_hbm_gbs": w * (ctx.n_touched + ctx.n_active) / t / 1e9,
                 "apply_hbm_frac": w * (ctx.n_touched + ctx.n_active) / t / 1e9 / hbm,
                 "tiles": tiles, "rel_err_vs_oracle": None}
            if k <= args.sweep_check_kmax:
                if ref is None:
                    from oracle.ghost_penalty import Oracle
                    o = Oracle(pr)
                    ref = o.apply(x_np)
                    ref32 = o.apply(x_np.astype(np.float32).astype(np.float64))
                rr = ref32 if prec == gp.GP_FP32 else ref
                r["rel_err_vs_oracle"] = float(np.linalg.norm(y.double().cpu().numpy() - rr) / np.linalg.norm(rr))
            rec[tags[prec]] = r
            rec["n_active"], rec["n_faces"], rec["n_touched"] = ctx.n_active, nf, ctx.n_touched
            ctx.close()
            del x, y
            torch.cuda.empty_cache()
        out["k"][str(k) if not args.sweep_workloads else name] = rec
        print(json.dumps({"workload": name, **rec}), file=sys.stderr, flush=True)
    print(json.dumps(out), flush=True)


def run_micro(args):
    """Per-face and per-cell cost with the data in cache, the GPU counterpart of the paper's
    single-cell benchmark (Sec. 3.1: the ghost-penalty evaluation on one face against the
    sum-factorised interior-cell Laplace, per k, in 2D and 3D).  Every cell of a box is
    inside and every interior face penalised; the box is sized to about four waves of
    face-kernel threads (1.2M normal lines), and the applies repeat over the same data
    without an L2 flush.  Reports ns per face (face kernel alone and whole y = G x),
    ns per cell of the Laplace cell kernel (mass weight 0, stiffness 1), in each arithmetic."""
    import torch

    from paper_2503_00246_gb300 import build as B
    B.build()
    from paper_2503_00246_gb300 import gp, workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    ks = [int(v) for v in args.sweep_k.split(",")]
    reps = args.micro_reps
    out = {"what": "ns per face / per cell, data hot in L2, all cells inside, all interior faces penalised",
           "d": {}}

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps * 1e-3

    for d in (2, 3):
        out["d"][str(d)] = {}
        for k in ks:
            L = (k + 1) ** (d - 1)      # face-kernel threads per face: about 4 waves of the GPU
            n = max(4, int(round((1.2e6 / (d * L)) ** (1.0 / d))))
            pr = W.box_problem(d, n, k, all_faces=True)
            rec = {"n": n, "cells": n ** d}
            lo = gp.setup_problem(pr, precision=gp.GP_FP32, device=0)
            for prec in (gp.GP_FP64_FF, gp.GP_FP64, gp.GP_FP32):
                ctx = lo if prec == gp.GP_FP32 else gp.setup_problem(pr, precision=prec, device=0)
                if args.tune_reps > 0:
                    gp.gp_autotune(ctx, args.tune_reps)
                tdt = torch.float32 if prec == gp.GP_FP32 else torch.float64
                x = torch.rand(ctx.n_active, dtype=tdt, device=dev)
                y = torch.empty_like(x)
                gp.gp_profile_enable(ctx, True)
                t_apply = timed(lambda: gp.gp_apply(ctx, x, y))
                ms_face, ms_lift, calls = gp.gp_profile_read(ctx)
                gp.gp_profile_enable(ctx, False)
                nf = ctx.n_faces
                r = {"ns_per_face_apply": t_apply / nf * 1e9, "ns_per_face_kernel": ms_face / calls * 1e6 / nf}
                if prec != gp.GP_FP32:
                    sysm = gp.gp_system_create(ctx, lo)
                    r["ns_per_cell_laplace"] = timed(lambda: gp.gp_system_cells(sysm, 0, x, y, 0.0, 1.0)) / n ** d * 1e9
                    if prec == gp.GP_FP64:
                        x32 = torch.rand(lo.n_active, dtype=torch.float32, device=dev)
                        y32 = torch.empty_like(x32)
                        rec["fp32_ns_per_cell_laplace"] = timed(
                            lambda: gp.gp_system_cells(sysm, 1, x32, y32, 0.0, 1.0)) / n ** d * 1e9
                    sysm.close()
                rec[{gp.GP_FP64_FF: "ff64", gp.GP_FP64: "fp64", gp.GP_FP32: "fp32"}[prec]] = r
                rec["faces"] = nf
                if ctx is not lo:
                    ctx.close()
            rec["fp32"]["ns_per_cell_laplace"] = rec.pop("fp32_ns_per_cell_laplace")
            lo.close()
            out["d"][str(d)][str(k)] = rec
            print(json.dumps({"d": d, "k": k, **rec}), file=sys.stderr, flush=True)
            torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def run_cg(args):
    """The solver study: gyroid (iso 0.3) on [-pi,pi]^3, n^3 cells, k = 4, model system
    (M_active + K_active + G) u = b, b ~ U[-1,1], per-order weights gamma / (j!)^2: FP32-inner
    defect correction and FP64 PCG, both to relative residual 1e-10 (Jacobi), float-float as
    the FP64-accuracy operator.  The full 128^3 mesh needs ~1e5 iterations; --cg-n picks n."""
    import torch

    from paper_2503_00246_gb300 import build as B
    B.build()
    from paper_2503_00246_gb300 import gp, workloads as W
    t0 = time.perf_counter()
    pr = W.gyroid_3d(k=4, n=args.cg_n)
    pr.weights = W.paper_weights(0.5, 4)
    hi = gp.setup_problem(pr, precision=gp.GP_FP64_FF, device=0)
    lo = gp.setup_problem(pr, precision=gp.GP_FP32, device=0)
    sysm = gp.gp_system_create(hi, lo)
    b = torch.tensor(W.rhs_vector(pr, hi.n_active), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(b)
    setup = time.perf_counter() - t0
    out = {"workload": f"{args.cg_n}^3 gyroid sin x cos y + sin y cos z + sin z cos x = 0.3 on [-pi,pi]^3, "
                       "k=4, c_j = 0.5/(j!)^2, (M_active + K_active + G) u = b, b ~ U[-1,1]",
           "n_active_dofs": hi.n_active, "ghost_faces": hi.n_faces, "setup_s": setup}
    for name, mode in (("defect_correction_fp32_inner", 0), ("pcg_fp64", 1)):
        torch.cuda.nvtx.range_push(name)        # ncu --nvtx --nvtx-include "<name>/" picks one solver
        st = gp.gp_system_solve(sysm, b, u, rtol=1e-10, inner_rtol=args.inner_rtol, mode=mode,
                                max_outer=args.max_outer, max_inner=args.max_inner)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        out[name] = st
    print(json.dumps(out), flush=True)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2503_00246_gb300 import build as B
    B.build()
    from paper_2503_00246_gb300 import gp, workloads as W

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pr = W.ball_3d()
    forms = {}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    peaks, peak_src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    fp64_peak = N_SM * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12   # TFLOP/s
    fp32_peak = N_SM * FP32_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    ff_peak = fp32_peak / FF_OPS_PER_FMA
    clocks = Clocks(local)

    results = {}
    names = {"fp64": gp.GP_FP64, "fp32": gp.GP_FP32, "ff": gp.GP_FP64_FF}
    precs = ([gp.GP_FP64_FF, gp.GP_FP64, gp.GP_FP32] if args.precision == "both" else [names[args.precision]])
    for prec in precs:
        ctx = gp.setup_problem(pr, precision=prec, device=local)
        tiles = None
        if args.tune_reps > 0:          # tile shape picked on this GPU, before any timing
            default = gp.gp_get_tiles(ctx)
            chosen, (tf, tl) = gp.gp_autotune(ctx, args.tune_reps)
            tiles = {"default": default, "chosen": chosen, "face_ms": tf, "lift_ms": tl}
        w = 4 if prec == gp.GP_FP32 else 8
        tdt = torch.float32 if prec == gp.GP_FP32 else torch.float64
        x_np = W.x_vectors(pr, ctx.n_active)[0]
        x = torch.tensor(x_np, dtype=tdt, device=dev)
        y = torch.empty_like(x)
        for _ in range(args.warmup):
            gp.gp_apply(ctx, x, y)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if prec == precs[0]:
            clocks.start()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))                 # evict x, y and the tables from L2
            ev[i][0].record(stream)
            gp.gp_apply(ctx, x, y)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
        if ws > 1:
            dist.barrier()
        ck = clocks.stop() if prec == precs[0] else None
        # per-kernel split: the same flushed steps with the library's event tracing, which puts
        # an event between the face and lift kernels (and so gives up their overlap)
        gp.gp_profile_enable(ctx, True)
        for i in range(min(args.steps, 500)):
            flush.fill_(float(i))
            gp.gp_apply(ctx, x, y)
        torch.cuda.synchronize()
        ms_jump, ms_lift, calls = gp.gp_profile_read(ctx)
        gp.gp_profile_enable(ctx, False)
        t_step = sum(a.elapsed_time(b) for a, b in ev) / args.steps   # ms
        t_max = t_step
        if ws > 1:
            tt = torch.tensor([t_step], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t_max = float(tt.item())
        d, k, nf = pr.dim, pr.degree, ctx.n_faces
        jump_ms = ms_jump / calls
        lift_ms = ms_lift / calls
        # end to end through the C ABI with pinned host buffers (copies inside the timed region)
        xh = torch.tensor(x_np, dtype=tdt).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        for _ in range(max(3, args.warmup // 4)):
            gp.gp_apply_host(ctx, xh, yh, stream)
        ne = max(10, args.steps // 10)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ne):
            gp.gp_apply_host(ctx, xh, yh, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t_e2e = e0.elapsed_time(e1) / ne
        # accuracy of this very output against the oracle (outside every timed region)
        err = None
        if args.check:
            from oracle.ghost_penalty import Oracle
            o = Oracle(pr)
            ref = o.apply(x_np if prec != gp.GP_FP32 else x_np.astype(np.float32).astype(np.float64))
            err = float(np.linalg.norm(y.double().cpu().numpy() - ref) / np.linalg.norm(ref))
        flop_face = _flops_face(d, k, nf)
        kname = {gp.GP_FP64: "double", gp.GP_FP32: "float", gp.GP_FP64_FF: "ff64"}[prec]
        roof = {"bound": "alu", "kernel": f"face_kernel<3,3,{kname}>",
                "achieved": flop_face / (jump_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                "peak": {gp.GP_FP64: fp64_peak, gp.GP_FP32: fp32_peak, gp.GP_FP64_FF: ff_peak}[prec],
                "peak_source": {gp.GP_FP64: "derived: 152 SM x 2 FP64 FMA/clk x 2070 MHz x 2 flop",
                                gp.GP_FP32: "derived: 152 SM x 128 FP32 FMA/clk x 2070 MHz x 2 flop",
                                gp.GP_FP64_FF: "derived: FP32 peak / 12 FP32 ops per compensated float-float multiply-add"}[prec]}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["traffic"] = _traffic({gp.GP_FP64: "f64", gp.GP_FP32: "f32", gp.GP_FP64_FF: "ff64"}[prec])
        alg_bytes = w * (ctx.n_touched + ctx.n_active)
        results[prec] = {
            "value": ws * ctx.n_active / (t_max * 1e-3) / 1e9,
            "ghost_faces_per_s": ws * ctx.n_faces / (t_max * 1e-3),
            "ms_per_step": t_max,
            "wall_ms_per_step": wall * 1e3 / args.steps,
            "kernel_ms": {"jump": jump_ms, "lift": lift_ms},
            "apply_hbm_gbs": alg_bytes / (t_step * 1e-3) / 1e9,
            "apply_hbm_frac": alg_bytes / (t_step * 1e-3) / 1e9 / hbm,
            "lift_hbm_gbs": w * ctx.n_active / (lift_ms * 1e-3) / 1e9,
            "roofline": roof,
            "e2e_ms": t_e2e,
            "e2e_value": ws * ctx.n_active / (t_e2e * 1e-3) / 1e9,
            "h2d": w * ctx.n_active, "d2h": w * ctx.n_active,
            "rel_err_vs_oracle": err,
            "clocks": ck,
            "n_active": ctx.n_active, "n_faces": nf, "n_touched": ctx.n_touched,
            "paper_flops_per_step": _flops_paper(d, k, nf),
            "paper_flop_rate": {"tflops": _flops_paper(d, k, nf) / (jump_ms * 1e-3) / 1e12,
                                "flops_per_face": _flops_paper(d, k, 1),
                                "count": "the paper's per-face count 2[(k+1)^(d-1) (2k+1)^2 + (d-1) (k+1)^d (2k+1)] "
                                         "over the face kernel's time"},
            "tiles": tiles,
        }
        ctx.close()

    order = [p for p in (gp.GP_FP64_FF, gp.GP_FP64, gp.GP_FP32) if p in results]
    head = order[0]
    r = results[head]
    dtypes = {gp.GP_FP64: "f64", gp.GP_FP32: "f32", gp.GP_FP64_FF: "ff64 (float-float arithmetic on f64 data)"}
    line = {
        "metric": METRIC,
        "value": r["value"],
        "unit": "GDoF/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": dtypes[head],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_cells": 64 ** 3, "degree": 3, "n_active_dofs": r["n_active"],
                   "ghost_faces": r["n_faces"], "touched_dofs": r["n_touched"],
                   "l2": "512 MB buffer written between timed steps (inputs < L2)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": r["roofline"],
        "e2e": {"value": r["e2e_value"], "unit": "GDoF/s", "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": 2 * args.steps,
        "clocks": r["clocks"],
        "apply_hbm": {"achieved": r["apply_hbm_gbs"], "peak": hbm, "unit": "GB/s", "frac": r["apply_hbm_frac"],
                      "peak_source": peak_src},
        "kernel_ms": r["kernel_ms"],
        "ghost_faces_per_s": r["ghost_faces_per_s"],
        "paper_flop_rate": r["paper_flop_rate"],
        "tiles": r["tiles"],
        "rel_err_vs_oracle": r["rel_err_vs_oracle"],
    }
    tags = {gp.GP_FP64: "fp64", gp.GP_FP32: "fp32", gp.GP_FP64_FF: "ff64"}
    for p in order[1:]:
        f = results[p]
        line[tags[p]] = {k2: f[k2] for k2 in ("value", "ms_per_step", "kernel_ms", "roofline", "apply_hbm_gbs",
                                              "apply_hbm_frac", "rel_err_vs_oracle", "e2e_value", "tiles",
                                              "ghost_faces_per_s", "paper_flop_rate")}
    if not args.no_batched:
        line["batched"] = {tags[p]: run_batched(gp, W, torch, dev, p, args.batched_steps, 2, args.tune_reps)
                           for p in (gp.GP_FP64_FF, gp.GP_FP64, gp.GP_FP32)}
        line["batched"]["workload"] = ("64 independent 3D balls on [-1,1]^3, n ~ U{16..96}, k ~ U{2..6}, "
                                       "r ~ U[0.4,0.8], 4 right-hand sides, one CUDA graph per apply")
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        line["cpu_paper_like"] = cpu_kronecker(args.cpu_seconds / 2)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- CPU arm --

def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(seconds: float):
    """The oracle, as it stands, on the host cores: full applies for about `seconds`."""
    from oracle.ghost_penalty import Oracle
    from paper_2503_00246_gb300 import workloads as W
    pr = W.ball_3d()
    o = Oracle(pr)
    x = W.x_vectors(pr, o.n_active)[0]
    for a in range(pr.dim):
        o.patch_index(a)
        o.A(a)
    o.apply(x)
    reps, t0 = 0, time.perf_counter()
    while True:
        o.apply(x)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds and reps >= 3:
            break
    t = el / reps
    return {"value": o.n_active / t / 1e9, "unit": "GDoF/s", "cores": _cores(), "kind": "oracle",
            "sample": f"{reps} full applies of the 64^3 k=3 workload ({o.n_faces} faces, explicit "
                      f"{(2 * 3 + 1) * 16}x{(2 * 3 + 1) * 16} face matrices, numpy FP64), {el:.1f} s"}


def cpu_kronecker(seconds: float):
    """The paper-like CPU baseline: the factorised (Kronecker) face operator of the paper
    in C with OpenMP over faces, FP64 (oracle/kron_cpu.c), full applies for about `seconds`."""
    from oracle.cpu_kronecker import KroneckerOpenMP
    from oracle.ghost_penalty import Oracle
    from paper_2503_00246_gb300 import workloads as W
    pr = W.ball_3d()
    o = Oracle(pr)
    kc = KroneckerOpenMP(pr, o)
    x = W.x_vectors(pr, o.n_active)[0]
    kc.apply(x)
    reps, t0 = 0, time.perf_counter()
    while True:
        kc.apply(x)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds and reps >= 3:
            break
    t = el / reps
    return {"value": o.n_active / t / 1e9, "unit": "GDoF/s", "cores": kc.nthreads,
            "kind": "paper-like CPU (Kronecker form of the face operator, C + OpenMP over faces, FP64)",
            "sample": f"{reps} full applies of the 64^3 k=3 workload, {el:.1f} s"}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    from oracle.ghost_penalty import Oracle
    from paper_2503_00246_gb300 import workloads as W
    pr = W.ball_3d()
    o = Oracle(pr)
    x = W.x_vectors(pr, o.n_active)[0]
    for a in range(pr.dim):
        o.patch_index(a)
        o.A(a)
    t0 = time.perf_counter()
    o.apply(x)
    t_full = time.perf_counter() - t0
    # each step is a bounded sample: a fixed fraction of the faces, so the whole run takes ~60 s
    budget = 60.0
    frac = min(1.0, budget / max(1, args.steps + args.warmup) / t_full)
    sub = {}
    for a in range(pr.dim):
        nfa = o.faces[a].shape[0]
        sub[a] = o.patch_index(a)[: max(1, int(math.ceil(frac * nfa)))]
    nsub = sum(v.shape[0] for v in sub.values())
    frac_eff = nsub / o.n_faces

    def step():
        y = np.zeros(o.n_active)
        for a, idx in sub.items():
            yf = x[idx] @ o.A(a).T
            y += np.bincount(idx.ravel(), weights=yf.ravel(), minlength=o.n_active)
        return y

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    t = (time.perf_counter() - t0) / args.steps
    value = frac_eff * o.n_active / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_fraction_of_faces": frac_eff},
            "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": _cores(), "kind": "oracle",
                             "sample": f"{nsub} of {o.n_faces} faces per step (explicit face matrices, numpy FP64); "
                                       f"DoF throughput scaled by that fraction"},
            "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gp", choices=["gp", "reference"])
    ap.add_argument("--precision", default="both", choices=["fp64", "fp32", "ff", "both"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", dest="check", action="store_false")
    ap.add_argument("--mode", default="bench", choices=["bench", "profile", "cg", "sweep", "micro"])
    ap.add_argument("--micro-reps", type=int, default=200)
    ap.add_argument("--sweep-k", default="1,2,3,4,5,6,7,8")
    ap.add_argument("--sweep-workloads", default="", help="comma-separated workload names instead of --sweep-k")
    ap.add_argument("--sweep-steps", type=int, default=50)
    ap.add_argument("--sweep-check-kmax", type=int, default=5)
    ap.add_argument("--inner-rtol", type=float, default=1e-4)
    ap.add_argument("--max-inner", type=int, default=200000)
    ap.add_argument("--max-outer", type=int, default=50)
    ap.add_argument("--cg-n", type=int, default=32)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=10)
    ap.add_argument("--workload", default="ball64_k3", choices=sorted(WORKLOADS))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tune-reps", type=int, default=5,
                    help="timed launches per candidate tile shape before the run (0: default shapes)")
    args = ap.parse_args()
    if args.mode == "profile":
        run_profile(args)
    elif args.mode == "sweep":
        run_sweep(args)
    elif args.mode == "micro":
        run_micro(args)
    elif args.mode == "cg":
        run_cg(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
