"""Benchmark of the matrix-free ghost-penalty apply y = G x on GB300.

Workload (the headline): gyroid sin x cos y + sin y cos z + sin z cos x = 0.3 on
[-pi,pi]^3, 128^3 Cartesian cells, FE_Q(4) on Gauss-Lobatto points, gamma = 0.5 for
every order (58.8M active DoFs, 335,664 ghost faces); x ~ U[-1,1] on the active DoFs.
One step = one y = G x over all ghost faces, native FP64.  The FP32 and float-float
forms run beside it on the same workload, each with its error against the FP64
oracle on sampled rows.  Also in the line: the degree sweep k = 1..8 on the 96^3
ball (bounded), and the batched workload (64 problems x 4 right-hand sides).

Metric: GDoF/s = active DoFs / apply time (the paper's throughput convention,
Sec. 3.1), whole job over all ranks.  x and y of the headline (470 MB each in
FP64) exceed the L2, and a 512 MB buffer is written between timed steps anyway.

Arms
  default            the CUDA path through the C ABI
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
WORKLOAD = ("ghost-penalty y=Gx, 3D gyroid sin x cos y + sin y cos z + sin z cos x = 0.3 in 128^3 cells on "
            "[-pi,pi]^3, FE_Q(4) Gauss-Lobatto, gamma=0.5, x ~ U[-1,1]")
# kernel launches of one gp_apply (face kernel, lift kernel)
KERNELS_PER_APPLY = 2


def config_dict(ws=1):
    """The config object of both arms' JSON lines (identical keys and values)."""
    return {"workload": WORKLOAD, "n_cells": 128 ** 3, "degree": 4, "n_active_dofs": 58763303,
            "ghost_faces": 335664, "touched_dofs": 10956390,
            "l2": "inputs larger than L2 (x, y 470 MB each in FP64); a 512 MB buffer is also written "
                  "between timed steps",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}
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
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(key):
    """DRAM bytes (read + write) per launch of kernel `key` from the committed ncu counters
    (profiles/traffic.json), or None when they are absent or the kernel sources changed
    since they were taken."""
    try:
        with open(TRAFFIC_FILE) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    if t.get("kernel_sources_sha256_16") != kernel_sources_hash():
        return None
    v = t.get("traffic_bytes_per_launch", {}).get(key)
    return int(v) if v is not None else None


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

def _flops_face(d, k, nf, prec="fp64", per_output=False):
    """Flops the face kernel executes (a multiply-add counts 2, a multiply or add 1; an
    n-term dot product 2n - 1), per normal line: the even-odd split (2k adds), the k
    jump dot products (k + 1 terms for odd orders, k for even ones), the tangential
    masses, the scaling by s_j (FP32 only: FP64 and float-float fold s_j into the jump
    vectors), and the expansion (per node b <= k one odd-order and, for b < k, one
    even-order partial sum, plus 2 adds).  Tangential masses: M^ applied to whole lines of
    N = k+1 values through its even / odd halves (2 floor(N/2) folds, ceil(N/2) dot
    products of ceil(N/2) terms, floor(N/2) of floor(N/2) terms, 2 floor(N/2) merges per N
    outputs), k N such lines per pass and face in 3D (k in 2D).  prec = "fp64" with
    per_output=True gives the earlier one-output-per-thread count ((d-1) passes of k
    (k+1)-term dot products per line)."""
    L = (k + 1) ** (d - 1)
    n_odd, n_even = (k + 1) // 2, k // 2            # orders j = 1, 3, ... and j = 2, 4, ...
    contraction = 2 * k + n_odd * (2 * (k + 1) - 1) + n_even * (2 * k - 1)
    if per_output:
        tangential_face = L * (d - 1) * k * (2 * (k + 1) - 1)
    else:
        N = k + 1
        H, NE = N // 2, (N + 1) // 2
        task = 2 * H + NE * (2 * NE - 1) + H * (2 * H - 1) + 2 * H
        tangential_face = (d - 1) * k * N * task if d == 3 else k * task
    scaling = k if prec == "fp32" else 0
    expansion = (k + 1) * (2 * n_odd - 1)
    if k > 1:
        expansion += k * ((2 * n_even - 1) + 2)
    return float(nf) * (L * (contraction + scaling + expansion) + tangential_face)


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
    prec = {"fp64": gp.GP_FP64, "fp32": gp.GP_FP32, "ff": gp.GP_FP64_FF, "all": gp.GP_FP64_FF}[args.precision]
    path = {"auto": gp.GP_PATH_AUTO, "face_lift": gp.GP_PATH_FACE_LIFT, "brick": gp.GP_PATH_BRICK}[args.path]
    ctx = gp.setup_problem(pr, precision=prec, device=0, path=path)
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
                      "tiles": tiles, "kernel_path": gp.gp_kernel_path(ctx)}))


def run_batched(gp, W, torch, dev, prec, steps, warmup, tune_reps=0):
    """The batched workload: 64 independent 3D ball problems, n ~ U{16..96}, k ~ U{2..6},
    4 right-hand sides each, replayed as one CUDA graph per apply (one face launch and one
    lift launch per degree, each over all problems and right-hand sides of that degree).
    Inputs (> 7 GB) exceed L2."""
    probs = W.batched_3d()
    nrhs = 4
    ctxs = [gp.setup_problem(p, precision=prec, device=dev.index or 0, path=gp.GP_PATH_FACE_LIFT) for p in probs]
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
           "scratch_bytes": scratch}
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
            fl_exec = _flops_face(pr.dim, k, nf, tags[prec].replace("ff64", "ff"))
            fl_paper = _flops_paper(pr.dim, k, nf)
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
    (M_active + K_active + G) u = b, b ~ U[-1,1], per-order weights gamma / (j!)^2, all to
    relative residual 1e-10 with Jacobi: defect correction (FP32 inner CG, outer residuals with
    the float-float FP64-accuracy operator), FP64 PCG with the native FP64 operator, and FP64
    PCG with the float-float operator.  The full 128^3 mesh needs ~1e5 iterations; --cg-n picks n."""
    import torch

    from paper_2503_00246_gb300 import build as B
    B.build()
    from paper_2503_00246_gb300 import gp, workloads as W
    t0 = time.perf_counter()
    pr = W.gyroid_3d(k=4, n=args.cg_n)
    pr.weights = W.paper_weights(0.5, 4)
    ff = gp.setup_problem(pr, precision=gp.GP_FP64_FF, device=0)
    f64 = gp.setup_problem(pr, precision=gp.GP_FP64, device=0)
    lo = gp.setup_problem(pr, precision=gp.GP_FP32, device=0)
    sys_ff = gp.gp_system_create(ff, lo)
    sys_64 = gp.gp_system_create(f64, None)
    b = torch.tensor(W.rhs_vector(pr, ff.n_active), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(b)
    setup = time.perf_counter() - t0
    out = {"workload": f"{args.cg_n}^3 gyroid sin x cos y + sin y cos z + sin z cos x = 0.3 on [-pi,pi]^3, "
                       "k=4, c_j = 0.5/(j!)^2, (M_active + K_active + G) u = b, b ~ U[-1,1]",
           "n_active_dofs": ff.n_active, "ghost_faces": ff.n_faces, "setup_s": setup}
    runs = (("defect_correction_fp32_inner", sys_ff, 0), ("pcg_fp64_native", sys_64, 1), ("pcg_fp64", sys_ff, 1))
    for name, sysm, mode in runs:
        if args.cg_only and name not in args.cg_only.split(","):
            continue
        torch.cuda.nvtx.range_push(name)        # ncu --nvtx --nvtx-include "<name>/" picks one solver
        st = gp.gp_system_solve(sysm, b, u, rtol=1e-10, inner_rtol=args.inner_rtol, mode=mode,
                                max_outer=args.max_outer, max_inner=args.max_inner)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        out[name] = st
        print(json.dumps({name: st}), file=sys.stderr, flush=True)
    out["operators"] = {"defect_correction_fp32_inner": "FP32 inner CG; outer residual with the float-float operator",
                        "pcg_fp64_native": "FP64 PCG, native FP64 operator (FP64 pipe)",
                        "pcg_fp64": "FP64 PCG, float-float FP64-accuracy operator"}
    print(json.dumps(out), flush=True)


def _sampled_error(o, x_np, y_dev, prec, nrows, seed=12):
    """max |y - y_ref| / max |y_ref| on sampled rows (random rows plus the patches of random
    faces of every axis), with the oracle's apply_rows: the check at sizes where a full oracle
    apply is too slow."""
    rng = np.random.default_rng(seed)
    touched = [o.patch_index(a)[rng.integers(0, o.faces[a].shape[0], 40)].ravel()
               for a in range(o.pr.dim) if o.faces[a].shape[0] > 0]
    rows = np.unique(np.concatenate([rng.integers(0, o.n_active, nrows)] + touched))
    xin = x_np if prec != 1 else x_np.astype(np.float32).astype(np.float64)
    ref = o.apply_rows(xin, rows)
    y = y_dev[rows].double().cpu().numpy()
    return float(np.abs(y - ref).max() / np.abs(ref).max())


def measure_form(gp, W, torch, pr, prec, dev, args, flush, o=None, e2e=True, tune=True, steps=None):
    """One arithmetic form of y = G x on one workload: device time per apply (CUDA events on
    the launching stream around each apply, L2 flushed between applies), the per-kernel split
    (separate traced applies), end to end through gp_apply_host, and the error against the
    oracle on sampled rows (when o is given)."""
    stream = torch.cuda.current_stream()
    steps = args.steps if steps is None else steps
    path = {"auto": gp.GP_PATH_AUTO, "face_lift": gp.GP_PATH_FACE_LIFT, "brick": gp.GP_PATH_BRICK}[args.path]
    ctx = gp.setup_problem(pr, precision=prec, device=dev.index or 0, path=path, slabs=args.slabs)
    kp = gp.gp_kernel_path(ctx)
    tiles = None
    if tune and args.tune_reps > 0:          # tile shape picked on this GPU, before any timing
        chosen, (tf, tl) = gp.gp_autotune(ctx, args.tune_reps)
        tiles = {"chosen": chosen, "face_ms": tf, "lift_ms": tl}
    tdt = torch.float32 if prec == gp.GP_FP32 else torch.float64
    x_np = W.x_vectors(pr, ctx.n_active)[0]
    x = torch.tensor(x_np, dtype=tdt, device=dev)
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        gp.gp_apply(ctx, x, y)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    t0 = time.perf_counter()
    for i in range(steps):
        flush.fill_(float(i))                 # evict x, y and the tables from L2
        ev[i][0].record(stream)
        gp.gp_apply(ctx, x, y)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    t_step = sum(a.elapsed_time(b) for a, b in ev) / steps   # ms
    # per-kernel split: the same flushed applies with the library's event tracing (an event
    # between the two kernels gives up their overlap)
    gp.gp_profile_enable(ctx, True)
    for i in range(min(steps, 200)):
        flush.fill_(float(i))
        gp.gp_apply(ctx, x, y)
    torch.cuda.synchronize()
    ms_face, ms_lift, calls = gp.gp_profile_read(ctx)
    gp.gp_profile_enable(ctx, False)
    err = _sampled_error(o, x_np, y, prec, args.check_rows) if (o is not None and args.check) else None
    rec = {"ctx_sizes": (ctx.n_active, ctx.n_faces, ctx.n_touched), "t_step": t_step, "kernel_path": kp,
           "wall_ms_per_step": wall * 1e3 / steps, "face_ms": ms_face / calls, "lift_ms": ms_lift / calls,
           "tiles": tiles, "rel_err_vs_oracle": err}
    if e2e:
        # end to end through the C ABI with pinned host buffers (the transfers inside the timed
        # region: x gathered from the host on the touched DoFs, y copied back whole)
        xh = torch.tensor(x_np, dtype=tdt).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        for _ in range(2):
            gp.gp_apply_host(ctx, xh, yh, stream)
        ne = max(3, min(10, steps))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ne):
            gp.gp_apply_host(ctx, xh, yh, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        rec["t_e2e"] = e0.elapsed_time(e1) / ne
        rec["h2d"], rec["d2h"] = gp.gp_apply_host_bytes(ctx)
        del xh, yh
    ctx.close()
    del x, y
    torch.cuda.empty_cache()
    return rec


def form_summary(rec, pr, prec, gp, hbm, peak_src, ws=1):
    """GDoF/s, ghost faces/s, the apply's algorithmic HBM fraction and the face kernel's
    roofline (ALU: executed flops over its traced time) of one measured form."""
    n_active, nf, n_touched = rec["ctx_sizes"]
    d, k = pr.dim, pr.degree
    w = 4 if prec == gp.GP_FP32 else 8
    t = rec["t_step"]
    fp64_peak = N_SM * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12   # TFLOP/s
    fp32_peak = N_SM * FP32_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    peak = {gp.GP_FP64: fp64_peak, gp.GP_FP32: fp32_peak, gp.GP_FP64_FF: fp32_peak / FF_OPS_PER_FMA}[prec]
    kname = {gp.GP_FP64: "double", gp.GP_FP32: "float", gp.GP_FP64_FF: "ff64"}[prec]
    flop_face = _flops_face(d, k, nf, {gp.GP_FP64: "fp64", gp.GP_FP32: "fp32", gp.GP_FP64_FF: "ff"}[prec])
    brick = rec["kernel_path"]["path"] == gp.GP_PATH_BRICK
    kernels = ("brick_kernel", "plane_fixup_kernel") if brick else ("face_kernel", "lift_kernel")
    roof = {"bound": "alu", "kernel": f"{kernels[0]}<{d},{k},{kname}>",
            "achieved": flop_face / (rec["face_ms"] * 1e-3) / 1e12 if rec["face_ms"] > 0 else None,
            "unit": "TFLOP/s", "peak": peak,
            "peak_source": {gp.GP_FP64: "derived: 152 SM x 2 FP64 FMA/clk x 2070 MHz x 2 flop",
                            gp.GP_FP32: "derived: 152 SM x 128 FP32 FMA/clk x 2070 MHz x 2 flop",
                            gp.GP_FP64_FF: "derived: FP32 peak / 12 FP32 ops per compensated float-float "
                                           "multiply-add"}[prec]}
    roof["frac"] = roof["achieved"] / peak if roof["achieved"] else None
    roof["traffic"] = _traffic(f"face_kernel_{kname}_d{d}k{k}")
    alg = w * (n_touched + n_active)
    out = {"value": ws * n_active / (t * 1e-3) / 1e9, "unit": "GDoF/s", "ms_per_step": t,
           "wall_ms_per_step": rec["wall_ms_per_step"],
           "ghost_faces_per_s": ws * nf / (t * 1e-3),
           "kernel_ms": {kernels[0]: rec["face_ms"], kernels[1]: rec["lift_ms"]},
           "kernel_path": rec["kernel_path"],
           "apply_hbm": {"achieved": alg / (t * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg / (t * 1e-3) / 1e9 / hbm, "peak_source": peak_src,
                         "algorithmic_bytes": alg,
                         "bytes": f"{w} B x (touched DoFs {n_touched} read + active DoFs {n_active} written)"},
           "roofline": roof,
           "paper_flop_rate": {"tflops": _flops_paper(d, k, nf) / (t * 1e-3) / 1e12,
                               "count": "2[(k+1)^(d-1) (2k+1)^2 + (d-1) (k+1)^d (2k+1)] per face over the apply time"},
           "rel_err_vs_oracle": rec["rel_err_vs_oracle"], "tiles": rec["tiles"],
           "n_active": n_active, "n_faces": nf, "n_touched": n_touched}
    if "t_e2e" in rec:
        out["e2e"] = {"value": ws * n_active / (rec["t_e2e"] * 1e-3) / 1e9, "unit": "GDoF/s",
                      "h2d_bytes_per_step": rec["h2d"], "d2h_bytes_per_step": rec["d2h"]}
    return out


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
    pr = W.gyroid_3d()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks, peak_src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    clocks = Clocks(local)
    o = None
    if args.check:
        from oracle.ghost_penalty import Oracle
        o = Oracle(pr)

    names = {"fp64": gp.GP_FP64, "fp32": gp.GP_FP32, "ff": gp.GP_FP64_FF}
    precs = [gp.GP_FP64, gp.GP_FP32, gp.GP_FP64_FF] if args.precision == "all" else [names[args.precision]]
    head = precs[0]
    recs = {}
    for prec in precs:
        if ws > 1:
            dist.barrier()
        if prec == head:
            clocks.start()
        recs[prec] = measure_form(gp, W, torch, pr, prec, dev, args, flush, o=o)
        if prec == head:
            ck = clocks.stop()
        if ws > 1:
            tt = torch.tensor([recs[prec]["t_step"]], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            recs[prec]["t_step"] = float(tt.item())
    forms = {p: form_summary(recs[p], pr, p, gp, hbm, peak_src, ws) for p in precs}
    r = forms[head]
    tags = {gp.GP_FP64: "fp64", gp.GP_FP32: "fp32", gp.GP_FP64_FF: "ff64"}
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
        "config": config_dict(ws),
        "roofline": r["roofline"],
        "e2e": r["e2e"],
        "gpu_launches": KERNELS_PER_APPLY * args.steps,
        "clocks": ck,
        "apply_hbm": r["apply_hbm"],
        "kernel_ms": r["kernel_ms"],
        "ghost_faces_per_s": r["ghost_faces_per_s"],
        "paper_flop_rate": r["paper_flop_rate"],
        "rel_err_vs_oracle": r["rel_err_vs_oracle"],
        "tiles": r["tiles"],
        "forms": {tags[p]: {k2: forms[p][k2] for k2 in ("value", "ms_per_step", "kernel_ms", "apply_hbm", "roofline",
                                                      "rel_err_vs_oracle", "e2e", "ghost_faces_per_s", "tiles",
                                                      "kernel_path")}
                  for p in precs},
        "error_check": f"max |y - y_ref| / max |y_ref| over ~{args.check_rows} sampled rows plus the patches of "
                       "sampled faces, FP64 oracle (explicit face matrices); FP32 against the oracle applied to x "
                       "rounded to FP32; targets 1e-12 (FP64, float-float) and 1e-5 (FP32)",
    }
    if not args.no_sweep:
        line["sweep_96"] = run_sweep_record(gp, W, torch, dev, args, flush, hbm, peak_src)
    if not args.no_batched:
        line["batched"] = {tags[p]: run_batched(gp, W, torch, dev, p, args.batched_steps, 2, args.tune_reps)
                           for p in (gp.GP_FP64, gp.GP_FP32, gp.GP_FP64_FF)}
        line["batched"]["workload"] = ("64 independent 3D balls on [-1,1]^3, n ~ U{16..96}, k ~ U{2..6}, "
                                       "r ~ U[0.4,0.8], 4 right-hand sides, one CUDA graph per apply")
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, o)
        line["cpu_paper_like"] = cpu_kronecker(args.cpu_seconds / 2)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_sweep_record(gp, W, torch, dev, args, flush, hbm, peak_src):
    """The degree sweep at its stated size, bounded: 96^3 ball, k = 1..8, each form timed over
    a few flushed applies (tiles tuned first), with sampled-row errors for k <= --sweep-check-kmax."""
    from oracle.ghost_penalty import Oracle
    out = {"workload": "96^3 cells on [-1,1]^3, ball r = 0.7 (seeded centre offset), gamma = 0.5, x ~ U[-1,1]",
           "steps_per_form": args.sweep_steps, "k": {}}
    tags = {gp.GP_FP64: "fp64", gp.GP_FP32: "fp32", gp.GP_FP64_FF: "ff64"}
    for k in range(1, 9):
        pr = W.ball_3d_sweep(k)
        o = Oracle(pr) if (args.check and k <= args.sweep_check_kmax) else None
        rec = {}
        for prec in (gp.GP_FP64, gp.GP_FP32, gp.GP_FP64_FF):
            m = measure_form(gp, W, torch, pr, prec, dev, args, flush, o=o, e2e=False, steps=args.sweep_steps)
            f = form_summary(m, pr, prec, gp, hbm, peak_src)
            rec[tags[prec]] = {"gdofs": f["value"], "ms": f["ms_per_step"], "apply_hbm_frac": f["apply_hbm"]["frac"],
                               "face_alu_frac": f["roofline"]["frac"], "rel_err_vs_oracle": f["rel_err_vs_oracle"]}
            rec["n_active"], rec["n_faces"] = f["n_active"], f["n_faces"]
        out["k"][str(k)] = rec
        print(json.dumps({"sweep_k": k, **rec}), file=sys.stderr, flush=True)
    return out


# ---------------------------------------------------------------- CPU arm --

def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_sample(o, frac):
    """The first ceil(frac * n_a) faces of every axis, and one oracle step over them: the
    explicit face matrices applied to the gathered patches, scattered with bincount."""
    sub = {}
    for a in range(o.pr.dim):
        nfa = o.faces[a].shape[0]
        if nfa:
            sub[a] = o.patch_index(a)[: max(1, int(math.ceil(frac * nfa)))]
    nsub = sum(v.shape[0] for v in sub.values())

    def step(x):
        y = np.zeros(o.n_active)
        for a, idx in sub.items():
            yf = x[idx] @ o.A(a).T
            y += np.bincount(idx.ravel(), weights=yf.ravel(), minlength=o.n_active)
        return y
    return step, nsub


def _headline_oracle(o=None):
    from oracle.ghost_penalty import Oracle
    from paper_2503_00246_gb300 import workloads as W
    pr = W.gyroid_3d()
    if o is None:
        o = Oracle(pr)
    x = W.x_vectors(pr, o.n_active)[0]
    for a in range(pr.dim):
        o.patch_index(a)
        o.A(a)
    return o, x


def cpu_baseline(seconds: float, o=None):
    """The oracle, as it stands, on the host cores: full applies of the headline workload
    for about `seconds` (at least one)."""
    o, x = _headline_oracle(o)
    o.apply(x)
    reps, t0 = 0, time.perf_counter()
    while True:
        o.apply(x)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds and reps >= 1:
            break
    t = el / reps
    P = 9 * 25
    return {"value": o.n_active / t / 1e9, "unit": "GDoF/s", "cores": _cores(), "kind": "oracle",
            "sample": f"{reps} full applies of the 128^3 gyroid k=4 workload ({o.n_faces} faces, explicit "
                      f"{P}x{P} face matrices, numpy FP64), {el:.1f} s"}


def cpu_kronecker(seconds: float, o=None):
    """The paper-like CPU baseline: the factorised (Kronecker) face operator of the paper
    in C with OpenMP over faces, FP64 (baselines/kron_cpu.c), full applies of the headline
    workload for about `seconds` (at least one)."""
    from baselines.cpu_kronecker import KroneckerOpenMP
    o, x = _headline_oracle(o)
    kc = KroneckerOpenMP(o.pr, o)
    kc.apply(x)
    reps, t0 = 0, time.perf_counter()
    while True:
        kc.apply(x)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds and reps >= 1:
            break
    t = el / reps
    return {"value": o.n_active / t / 1e9, "unit": "GDoF/s", "cores": kc.nthreads,
            "kind": "paper-like CPU (Kronecker form of the face operator, C + OpenMP over faces, FP64)",
            "sample": f"{reps} full applies of the 128^3 gyroid k=4 workload, {el:.1f} s"}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    o, x = _headline_oracle()
    t0 = time.perf_counter()
    o.apply(x)
    t_full = time.perf_counter() - t0
    # each step is a bounded sample: a fixed fraction of the faces, so the whole run takes ~60 s
    budget = 60.0
    frac = min(1.0, budget / max(1, args.steps + args.warmup) / t_full)
    step, nsub = _oracle_sample(o, frac)
    frac_eff = nsub / o.n_faces
    for _ in range(args.warmup):
        step(x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(x)
    t = (time.perf_counter() - t0) / args.steps
    value = frac_eff * o.n_active / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(ws),
            "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": _cores(), "kind": "oracle",
                             "sample": f"{nsub} of {o.n_faces} faces per step (explicit face matrices, numpy FP64); "
                                       f"DoF throughput scaled by that fraction"},
            "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gp", choices=["gp", "reference"])
    ap.add_argument("--precision", default="all", choices=["fp64", "fp32", "ff", "all"])
    ap.add_argument("--check-rows", type=int, default=2000, help="sampled rows of the oracle error check")
    ap.add_argument("--no-sweep", action="store_true", help="leave out the bounded 96^3 degree sweep")
    ap.add_argument("--slabs", type=int, default=0,
                    help="face + lift launch pipeline: 0 or 1 one launch pair, n about n slabs")
    ap.add_argument("--path", default="auto", choices=["auto", "face_lift", "brick"],
                    help="kernel path of the single-problem applies (gp_opts.kernel_path)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", dest="check", action="store_false")
    ap.add_argument("--mode", default="bench", choices=["bench", "profile", "cg", "sweep", "micro"])
    ap.add_argument("--micro-reps", type=int, default=200)
    ap.add_argument("--sweep-k", default="1,2,3,4,5,6,7,8")
    ap.add_argument("--sweep-workloads", default="", help="comma-separated workload names instead of --sweep-k")
    ap.add_argument("--sweep-steps", type=int, default=10)
    ap.add_argument("--sweep-check-kmax", type=int, default=4)
    ap.add_argument("--inner-rtol", type=float, default=1e-4)
    ap.add_argument("--max-inner", type=int, default=200000)
    ap.add_argument("--max-outer", type=int, default=50)
    ap.add_argument("--cg-n", type=int, default=32)
    ap.add_argument("--cg-only", default="", help="comma-separated solver names of --mode cg to run")
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
