#!/usr/bin/env python3
"""Benchmark: ADMM iterations/s of the separable low-rank Hankel reconstruction.

Workload (N=1): 12-coil 256x256 complex64 k-space (seeded ellipse phantom,
Gaussian coil maps, noise 1e-3), 1D random mask R=4 + 24 ACS lines, SHLR with
window 16 -> 512 lifted 241x192 matrices per iteration.  A "step" is one ADMM
iteration (X-update, all 512 SVTs, multiplier update, adjoints).  The batched
form (one launch per step kind, iteration captured as a CUDA graph) is the
headline; the plain per-matrix form is reported beside it.

Multi-GPU (torchrun, one process per GPU): each rank reconstructs its own
instance (weak scaling, no collective on the data path); value = iterations
of all ranks / max-over-ranks time.

`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "iters/s at 12-coil 256² k-space, batched vs plain, rel err ≤1e-4 vs FP64"
WORKLOAD = "shlr_12c_256"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi clocks / throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
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
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- GPU arm
def kernel_launches_per_iteration(plan, model2d, exec_mode, svd="eig", reduction=0):
    """Kernels libselr launches per ADMM iteration (mirrors admm_stage and svd_apply in
    selr.cu): adjoint, FFTs of the adjoints, DC + reduction, hybrid FFTs, lift, and the
    SVT kernels: either the warp-per-matrix SVT (s <= 8, len <= 64) or Gram, tridiagonal
    reduction, eigenvectors, the three apply kernels (streaming for r <= 32 and
    32 < r <= 64 pairs, general above) and the FP64 re-solve of flagged matrices (eig),
    Jacobi and apply (jacobi).  Batched, one
    SVT launch sequence covers each run of consecutive lift families of the same SVT
    size class (svt_class in selr.cu); plain, one per matrix.  With the two-stage reduction in
    force (reduction 2) a sequence whose orders all lie in 48 .. 192 launches both of its
    kernels in place of the one-stage reduction."""
    fams = [plan.lift_shape(a) for a in (("row", "col") if model2d else ("pe", "param"))]
    fft_a = 2 if model2d else 1

    def svt_class(r, c):
        s, l = min(r, c), max(r, c)
        if s <= 8 and l <= 64:
            return 0
        if svd == "jacobi":
            return 1
        for i, bound in enumerate((32, 64, 128, 192, 208, 256), 1):
            if s <= bound:
                return i
        return 7

    def two_stage(shapes):
        return svd == "eig" and reduction == 2 and all(48 <= min(r, c) <= 192 for r, c in shapes)

    def svt_kernels(r, c):
        return 1 if svt_class(r, c) == 0 else ((8 if two_stage([(r, c)]) else 7) if svd == "eig" else 2)

    if exec_mode == "batched":
        runs = []                                   # (class, shapes) of consecutive families
        for _, r, c in fams:
            k = svt_class(r, c)
            if runs and runs[-1][0] == k:
                runs[-1][1].append((r, c))
            else:
                runs.append((k, [(r, c)]))
        per = 1 + fft_a + 2 + fft_a + 1 + sum(
            1 if k == 0 else ((8 if two_stage(sh) else 7) if svd == "eig" else 2) for k, sh in runs)
    else:
        nmat = sum(nm for nm, _, _ in fams)
        per = nmat + fft_a + 2 + fft_a + sum(nm * (1 + svt_kernels(r, c)) for nm, r, c in fams)
    desc = getattr(plan, "desc", None)
    if desc is not None and desc.model in ("SHLR_S", "SHLR_SV"):
        # the SPIRiT X-update (spirit.cu) replaces the pointwise divide: copy, one operator
        # application (4 FFTs, pixel kernel, combine), init, then per CG iteration one
        # application, the update and (but the last) the direction update, and the finish
        per += 7 + 8 * desc.cg_iters
    return per + (0 if model2d else 1)


def calibration_launches(plan):
    """Kernels of the SPIRiT calibration that opens every SHLR-S / SHLR-SV solve: Gram of
    the ACS rows, one Cholesky launch per 4 target coils, placement, 2 FFTs, finish."""
    if plan.desc.model not in ("SHLR_S", "SHLR_SV"):
        return 0
    return 5 + (plan.desc.J + 3) // 4


def gram_for(args, model2d):
    """Gram precision the plans start from (before autotuning): --gram if given, else
    3xtf32 (FP32-level accuracy on every model)."""
    return args.gram or "3xtf32"


def instance_workload(wl, rank):
    """Rank r reconstructs its own seeded instance of the same workload (weak scaling)."""
    return wl.with_(seed=wl.seed + 1000 * rank) if rank else wl


def max_over_ranks(ms, world, device="cuda"):
    """Slowest rank's time (all ranks call this; no-op for one rank)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, steps, ms):
    """Iterations of all ranks per second of the slowest rank."""
    return world * steps / (ms / 1000.0)


def flops_svd_per_matrix(l, s):
    """Textbook flops of one SVD (Gram + full Hermitian eigensolve): 8 l s^2 + 36 s^3."""
    return 8.0 * l * s * s + 36.0 * s ** 3


# Flops of the eigensolver SVT as this method does it, per l x s matrix with r
# singular values above t (real flops; a complex multiply-add is 8):
#   Gram G = B^H B, lower triangle with diagonal         4 l s (s + 1)
#   Householder tridiagonalisation of the Hermitian G      (16/3) s^3
#   multisection of each of the r eigenvalues:  12 rounds x 32 Sturm counts of s steps,
#     4 flops a step (a subtraction, a division, a comparison folded into a multiply-add)
#                                                          1536 s r
#   inverse iteration (LU of the shifted tridiagonal and two solves, three passes)  90 s r
#   back-transformation of r vectors through s - 1 reflectors          8 s^2 r
#   apply Z = (B V) diag(h) V^H and the multiplier update            16 l s r
def method_flops(l, s, r):
    return {"gram": 4.0 * l * s * (s + 1),
            "tridiag": 16.0 / 3.0 * s ** 3,
            "eigvec": (1536.0 + 90.0) * s * r + 8.0 * s * s * r,
            "apply": 16.0 * l * s * r}


def step_bytes(plan, model2d):
    """Algorithmic HBM bytes of one ADMM iteration: the persistent multipliers D of
    every lifted matrix read and written once, plus the k-space sized passes (adjoint
    output, the DC's reads of Y, mask, both adjoints and K and its write, the FFTs of
    the adjoints and of K to the two hybrid arrays): about 16 complex k-space arrays."""
    fams = ("row", "col") if model2d else ("pe", "param")
    lift = sum(n * r * c for n, r, c in (plan.lift_shape(a) for a in fams))
    return 2 * 8 * lift + 16 * 8 * plan.nK


def measured_peaks(api):
    """FP32 FMA (scalar FFMA and packed FFMA2) from libselr's probe and TF32 tensor
    throughput from a cuBLAS FP32 GEMM with TF32 allowed (8192^3, best of 5)."""
    import torch
    out = {}
    try:
        f1, _ = api.selr_probe_fp32_peak(False, 4096)
        f2, _ = api.selr_probe_fp32_peak(True, 4096)
        out.update(fp32_ffma_tflops=f1, fp32_ffma2_tflops=f2, fp32_tflops=max(f1, f2))
    except Exception as e:                      # reported, not fatal
        out["fp32_error"] = str(e)
    try:
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = True
        n = 8192
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        c = a @ b
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out["tf32_tflops"] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
        torch.backends.cuda.matmul.allow_tf32 = prev
        del a, b, c
        torch.cuda.empty_cache()
    except Exception as e:
        out["tf32_error"] = str(e)
    return out


def run_gpu(args, rank, world):
    import torch
    from paper_2107_11650_gb300 import api, build

    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
        build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    wl = synth.get_config(args.config)
    inp = synth.make_inputs(instance_workload(wl, rank))
    Yh = torch.from_numpy(inp["Y"].astype(np.complex64))
    mh = torch.from_numpy(inp["mask"].astype(np.uint8))
    Y = Yh.cuda()
    mask = mh.cuda()
    X = torch.empty_like(Y)
    stream = torch.cuda.Stream()
    results = {}
    model2d = wl.model in ("SHLR", "SHLR_V", "SHLR_S", "SHLR_SV")
    modes = ["batched", "plain"] if args.exec == "both" else [args.exec]
    for mode in modes:
        plan = api.Plan(api.Desc.from_workload(wl, exec=mode, max_iter=max(args.warmup, 1), svd=args.svd,
                                               gram=gram_for(args, model2d)))
        if args.reduction:
            plan.set_reduction(args.reduction)
        nmat = sum(plan.lift_shape(a)[0] for a in (("row", "col") if model2d else ("pe", "param")))
        with torch.cuda.stream(stream):
            api.selr_solve(plan, Y, mask, X, stream=stream)           # W warm-up iterations
        st = api.selr_sync_status(plan, stream)
        if mode == "batched" and args.ev_chunk:
            plan.set_tuning(plan.desc.gram, args.ev_chunk)
            results["tuning"] = plan.tuning()
        elif mode == "batched" and not args.no_autotune:
            with torch.cuda.stream(stream):
                results["tuning"] = plan.autotune(Y, mask, allow_tf32=args.allow_tf32, stream=stream)
        steps = args.steps if mode == "batched" else max(1, min(args.steps, args.plain_steps))
        plan.set_iterations(steps)
        with torch.cuda.stream(stream):
            api.selr_solve(plan, Y, mask, X, stream=stream)           # capture the K-iteration graph
        stream.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(dev) if (mode == "batched" and rank == 0) else None
        if clk:
            clk.start()
            time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            api.selr_solve(plan, Y, mask, X, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), world)
        clocks = clk.stop() if clk else None
        st2 = api.selr_sync_status(plan, stream)
        if mode == "batched" and args.svd == "eig":
            results["rank_sums"] = api.selr_plan_rank_sums(plan, stream)   # ranks over the timed iterations
        # stage split, outside the timed region: the same K iterations with one graph per
        # stage and events between the stages (the stage boundaries cut the programmatic
        # launch chain of the eigensolver, so these stage times add up to more than ms)
        plan.profile(True)
        with torch.cuda.stream(stream):
            api.selr_solve(plan, Y, mask, X, stream=stream)           # capture the stage graphs
            api.selr_solve(plan, Y, mask, X, stream=stream)
        stream.synchronize()
        prof = plan.profile_read()
        plan.profile(False)
        st3 = api.selr_sync_status(plan, stream)
        results[mode] = dict(ms=ms, steps=steps, status=max(st, st2, st3), nmat=nmat, clocks=clocks, stages=prof,
                             launches=steps * kernel_launches_per_iteration(plan, model2d, mode, args.svd,
                                                                            plan.tuning()["reduction"]) + 6
                             + calibration_launches(plan))
        if mode == "batched":
            results["plan"] = plan
        else:
            plan.close()
    plan = results["plan"]
    jac = work_model(plan, model2d, args.svd, results.get("rank_sums"), results["batched"]["stages"])
    e2e = time_e2e(plan, Yh, mh, stream, reps=2)
    e2e_ms = max_over_ranks(1000.0 * plan.desc.max_iter / e2e["value"], world)
    e2e["value"] = whole_job_value(world, plan.desc.max_iter, e2e_ms)
    results["accuracy"] = accuracy_vs_oracle(plan, wl, Y, mask, stream) if rank == 0 else None
    return results, jac, e2e, wl


def work_model(plan, model2d, svd, rank_sums, stages):
    """Per-iteration algorithmic work of the batched step: flops by kind (the method's
    own count, method_flops, with each family's mean rank over the timed iterations),
    the SVD stage's flops per launch, and its measured duration (stage-profiled run)."""
    fams = ("row", "col") if model2d else ("pe", "param")
    tot = {"gram": 0.0, "tridiag": 0.0, "eigvec": 0.0, "apply": 0.0, "small_svt": 0.0}
    ranks = {}
    eig_shapes = []
    m0 = 0
    for ax in fams:
        nm_, r_, c_ = plan.lift_shape(ax)
        l, s = max(r_, c_), min(r_, c_)
        if s <= 8 and l <= 64:                 # warp-per-matrix Jacobi family: textbook count
            tot["small_svt"] += nm_ * 2.0 * flops_svd_per_matrix(l, s)
        elif svd == "jacobi":
            tot["small_svt"] += nm_ * 2.0 * flops_svd_per_matrix(l, s)
        else:
            rbar = 0.0
            if rank_sums is not None:
                sums, it = rank_sums
                rbar = float(sums[m0:m0 + nm_].sum()) / max(it * nm_, 1)
            ranks[ax] = rbar
            eig_shapes.append((nm_, s))
            for k, v in method_flops(l, s, rbar).items():
                tot[k] += nm_ * v
        m0 += nm_
    st_ = stages
    ms_svd = st_["svd"][0] / max(st_["svd"][1], 1)
    return dict(ms=ms_svd, flops=tot["tridiag"] + tot["eigvec"], stage="svd", flops_by_kind=tot, mean_rank=ranks,
                bytes=step_bytes(plan, model2d), eig_shapes=eig_shapes)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per matrix of k_tridiag + k_eigvec,
# by order s, from one full-size ncu capture of each kernel on the 12-coil 256x256 workload
# (k_tridiag 75.94 + 18.22 MB, k_eigvec 77.59 + 0.06 MB per launch of 512 matrices): the packed
# Gram read once, the Householder vectors written once and read once.  Orders without a
# capture report no traffic.
NCU_SVD_BYTES_PER_MATRIX = {192: (75.94e6 + 18.22e6 + 77.59e6 + 0.06e6) / 512}


def svd_traffic(eig_shapes):
    if not eig_shapes or any(s not in NCU_SVD_BYTES_PER_MATRIX for _, s in eig_shapes):
        return None
    return sum(nm * NCU_SVD_BYTES_PER_MATRIX[s] for nm, s in eig_shapes)


def accuracy_vs_oracle(plan, wl, Y, mask, stream):
    """Relative error of the reconstruction after the stored number of iterations
    against FP64 oracle values at seeded sample positions (tests/golden, written by
    an oracle-only script); None if no values are stored for the workload."""
    import torch
    from paper_2107_11650_gb300 import api
    path = os.path.join(ROOT, "tests", "golden", f"{wl.name}_30it.npz")
    if not os.path.exists(path):
        return None
    g = np.load(path)
    plan.set_iterations(int(g["n_iter"]))
    X = torch.empty_like(Y)
    with torch.cuda.stream(stream):
        api.selr_solve(plan, Y, mask, X, stream=stream)
    st = api.selr_sync_status(plan, stream)
    xs = X.cpu().numpy().ravel()[g["idx"]].astype(np.complex128)
    err = float(np.linalg.norm(xs - g["values"]) / np.linalg.norm(g["values"]))
    return {"rel_err_vs_fp64": err, "iterations": int(g["n_iter"]), "status": st,
            "reference": f"FP64 oracle values at {len(g['idx'])} seeded positions, tests/golden/{wl.name}_30it.npz"}


def time_e2e(plan, Yh, mh, stream, reps):
    import torch
    from paper_2107_11650_gb300 import api
    Yp = Yh.pin_memory()
    mp = mh.pin_memory()
    Xp = torch.empty_like(Yp).pin_memory()
    Yd = torch.empty(Yp.shape, dtype=Yp.dtype, device="cuda")
    md = torch.empty(mp.shape, dtype=mp.dtype, device="cuda")
    Xd = torch.empty_like(Yd)
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            Yd.copy_(Yp, non_blocking=True)
            md.copy_(mp, non_blocking=True)
            api.selr_solve(plan, Yd, md, Xd, stream=stream)
            Xp.copy_(Xd, non_blocking=True)
        stream.synchronize()
        times.append(time.perf_counter() - t0)
    t = min(times)
    it = plan.desc.max_iter
    return dict(value=it / t, h2d=(Yp.numel() * 8 + mp.numel()) / it, d2h=Xp.numel() * 8 / it)


# ------------------------------------------------------------- CPU oracle
_ORACLE_CACHE = {}


def oracle_sample(wl, n_svt=64):
    """One bounded oracle step on the workload's initial state: the X-update
    (Eq. 15 / S7) and the lifts of every matrix, timed in full, then the SVT and
    multiplier update (Eqs. 13-17 / S5-S9) of about n_svt of the lifted matrices
    (every k-th matrix of each family, so the sample spans the whole array),
    timed on their own.  Returns (estimated seconds of one full
    iteration = full part + SVT part x matrices / sampled matrices, wall seconds
    of the step, sampled share of the SVTs)."""
    from oracle import admm as oadmm
    from oracle.svt import svt
    if wl.name not in _ORACLE_CACHE:
        _ORACLE_CACHE[wl.name] = synth.make_inputs(wl)
    inp = _ORACLE_CACHE[wl.name]
    b = wl.beta
    if wl.model in ("SHLR", "SHLR_V", "SHLR_S", "SHLR_SV"):
        s = oadmm.Shlr2D(inp["Y"], inp["mask"], wl)
        st = s.init_state()
        t0 = time.perf_counter()
        K = s.x_update(st["Zr"], st["Zc"], st["Dr"], st["Dc"])
        LXr, LXc = s.lifts(K)
        t1 = time.perf_counter()
        nt = LXr.shape[0] + LXc.shape[0]
        step = max(1, nt // max(n_svt, 1))
        ir, ic = np.arange(0, LXr.shape[0], step), np.arange(step // 2, LXc.shape[0], step)
        Zr = svt(LXr[ir] + st["Dr"][ir] / b, 1.0 / b)
        Zc = svt(LXc[ic] + st["Dc"][ic] / b, 1.0 / b)
        _ = (st["Dr"][ir] + wl.tau * (LXr[ir] - Zr), st["Dc"][ic] + wl.tau * (LXc[ic] - Zc))
        t2 = time.perf_counter()
        share = (len(ir) + len(ic)) / nt
    else:
        s = oadmm.ShlrParam(inp["Y"], inp["mask"], wl)
        st = s.init_state()
        t0 = time.perf_counter()
        K = s.x_update(st["Zpe"], st["Zp"], st["Dpe"], st["Dp"])
        LXpe, LXp = s.lifts(K)
        t1 = time.perf_counter()
        step = max(1, LXpe.shape[0] // max(n_svt, 1))
        ipe, ipp = np.arange(0, LXpe.shape[0], step), np.arange(0, LXp.shape[0], step)
        share = len(ipe) / LXpe.shape[0]
        Z1 = svt(LXpe[ipe] + st["Dpe"][ipe] / b, 1.0 / b)
        Z2 = svt(LXp[ipp] + st["Dp"][ipp] / b, wl.lam2 / b)
        _ = (st["Dpe"][ipe] + wl.tau * (LXpe[ipe] - Z1), st["Dp"][ipp] + wl.tau * (LXp[ipp] - Z2))
        t2 = time.perf_counter()
    return (t1 - t0) + (t2 - t1) / share, t2 - t0, share


def cpu_baseline(wl, iters=2):
    """The oracle timed over `iters` full ADMM iterations of the workload (the first
    iterations of Algorithm S1 / S2 from the initial state); cores = CPU time / wall
    time of the run (the threads the BLAS and FFT actually kept busy)."""
    from oracle import admm as oadmm
    if wl.name not in _ORACLE_CACHE:
        _ORACLE_CACHE[wl.name] = synth.make_inputs(wl)
    inp = _ORACLE_CACHE[wl.name]
    two_d = wl.model in ("SHLR", "SHLR_V", "SHLR_S", "SHLR_SV")
    s = oadmm.Shlr2D(inp["Y"], inp["mask"], wl) if two_d else oadmm.ShlrParam(inp["Y"], inp["mask"], wl)
    st = s.init_state()
    act = None if two_d else np.ones(wl.M, bool)
    c0, t0 = time.process_time(), time.perf_counter()
    for _ in range(iters):
        st, _ = s.step(st) if two_d else s.step(st, act)
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    return {"value": iters / wall, "unit": "iters/s", "cores": round(cpu / wall, 1), "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"FP64 NumPy oracle on {wl.name}: {iters} full ADMM iterations timed ({wall:.1f} s)"}


def run_reference_unrolled(args):
    """Oracle arm of the unrolled batch: FP64 forward + reverse pass of the
    smallest instance (8 coils, 128x128), scaled to the whole batch by the
    SVT work ratio sum_i nmat_i l_i s_i^2 / (nmat_0 l_0 s_0^2)."""
    from oracle.unrolled import unrolled_2d_vjp
    wls = synth.unrolled_batch()
    n_iter = wls[0].n_iter

    def work(w):
        tot = 0
        for nv, nmat in ((w.N, w.M), (w.M, w.N)):
            l, s = max(nv - w.window + 1, w.J * w.window), min(nv - w.window + 1, w.J * w.window)
            tot += nmat * l * s * s
        return tot

    w0 = min(wls, key=work)
    inp = synth.make_inputs(w0)
    rng = np.random.default_rng(77)
    Xb = rng.standard_normal(inp["Y"].shape) + 1j * rng.standard_normal(inp["Y"].shape)
    ts = np.full(n_iter, 1.0 / w0.beta)
    taus = np.full(n_iter, w0.tau)
    scale = sum(work(w) for w in wls) / work(w0)
    vals = []
    for _ in range(max(args.steps, 1)):
        t0 = time.perf_counter()
        unrolled_2d_vjp(inp["Y"], inp["mask"], w0, ts, taus, Xb)
        dt = time.perf_counter() - t0
        vals.append(len(wls) * n_iter / (dt * scale))
    v = float(np.median(vals))
    line = {"metric": "instance-iterations/s, forward + backward, 16 uneven unrolled SHLR instances",
            "value": v, "unit": "instance-iters/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * len(wls) * n_iter / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "unrolled_16_uneven", "unrolled_iterations": n_iter},
            "cpu_baseline": {"value": v, "unit": "instance-iters/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"FP64 forward + reverse pass of the {w0.J}-coil {w0.M}x{w0.N} instance, "
                                       f"scaled by the SVT work ratio {scale:.1f} of the batch"},
            "e2e": {"value": v, "unit": "instance-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return line


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores (rank 0 only).  A step is the bounded
    sample of oracle_sample: value = 1 / (median estimated seconds of one full
    iteration); ms_per_step = the measured wall time of a step."""
    if world > 1 and rank != 0:
        return None
    if args.config == "unrolled_16_uneven":
        return run_reference_unrolled(args)
    wl = synth.get_config(args.config)
    for _ in range(args.warmup):
        oracle_sample(wl, n_svt=8)
    est, walls = [], []
    c0, t0 = time.process_time(), time.perf_counter()
    for _ in range(args.steps):
        e, w, share = oracle_sample(wl, n_svt=64)
        est.append(e)
        walls.append(w)
    wall = time.perf_counter() - t0
    cores = (time.process_time() - c0) / wall
    v = 1.0 / float(np.median(est))
    sample = (f"per step: X-update and lifts of one ADMM iteration timed in full, SVT + multiplier update of "
              f"{share:.4f} of the lifted matrices timed and scaled by 1/{share:.4f}")
    line = {"metric": METRIC, "value": v, "unit": "iters/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean(walls)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wl.name, "coils": wl.J, "size": [wl.M, wl.N], "window": wl.window,
                       "model": wl.model, "mask": f"{wl.mask} R={wl.R} acs={wl.n_acs}"},
            "iteration_s_estimated": float(np.median(est)),
            "cpu_baseline": {"value": v, "unit": "iters/s", "cores": round(cores, 1), "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line))
    return line


def run_unrolled(args, rank, world):
    """Uneven batch of 16 unrolled SHLR reconstructions (10 iterations, shared
    learnable t_k, tau_k): a step is one forward + hand-written backward pass of
    the whole batch; value = instance-iterations per second."""
    import torch
    from paper_2107_11650_gb300 import api, build
    from paper_2107_11650_gb300.unrolled import UnrolledBatch

    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
        build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    wls = synth.unrolled_batch()
    n_iter = wls[0].n_iter
    inputs = [synth.make_inputs(instance_workload(w, rank)) for w in wls]
    Yh = [torch.from_numpy(i["Y"].astype(np.complex64)) for i in inputs]
    Ys = [y.cuda() for y in Yh]
    masks = [torch.from_numpy(i["mask"].astype(np.uint8)).cuda() for i in inputs]
    rng = np.random.default_rng(77 + rank)
    Xbs = [torch.from_numpy((rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape)).astype(np.complex64))
           .cuda() for y in Yh]
    net = UnrolledBatch([api.Desc.from_workload(w) for w in wls], masks, n_iter)

    def step(Ys_):
        net.zero_grad(set_to_none=True)
        Xs = net([y.requires_grad_(False) for y in Ys_])
        loss = sum((xb.conj() * x).real.sum() for xb, x in zip(Xbs, Xs))
        loss.backward()
        return loss

    for _ in range(max(args.warmup, 1)):
        step(Ys)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    with torch.no_grad():
        for _ in range(args.steps):
            net(Ys)
    e1.record()
    e1.synchronize()
    fwd_ms = max_over_ranks(e0.elapsed_time(e1), world) / args.steps
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dev) if rank == 0 else None
    if clk:
        clk.start()
        time.sleep(0.3)
    e0.record()
    for _ in range(args.steps):
        step(Ys)
    e1.record()
    e1.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    clocks = clk.stop() if clk else None
    # end to end: k-space from pinned host memory, loss and parameter gradients back to the host
    Yp = [y.pin_memory() for y in Yh]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Yd = [y.cuda(non_blocking=True) for y in Yp]
        loss = step(Yd)
        out = torch.cat([loss.reshape(1), net.ts.grad, net.taus.grad]).cpu()
    e2e_ms = max_over_ranks(1000.0 * (time.perf_counter() - t0), world)
    units = len(wls) * n_iter
    status = max(api.selr_sync_status(e.plan) for e in net.engines)
    if rank != 0:
        return None
    line = {
        "status": status,
        "metric": "instance-iterations/s, forward + backward, 16 uneven unrolled SHLR instances",
        "value": whole_job_value(world, args.steps * units, ms), "unit": "instance-iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "unrolled_16_uneven", "instances": [f"{w.J}c {w.M}x{w.N}" for w in wls],
                   "window": wls[0].window, "unrolled_iterations": n_iter,
                   "l2": "per-step checkpoints and lifted arrays (GBs) exceed L2; no flush"},
        "forward_ms_per_step": fwd_ms, "backward_over_forward": (ms / args.steps - fwd_ms) / fwd_ms,
        "roofline": None,
        "e2e": {"value": whole_job_value(world, args.steps * units, e2e_ms), "unit": "instance-iters/s",
                "h2d_bytes_per_step": sum(y.numel() * 8 for y in Yh), "d2h_bytes_per_step": 4 * (1 + 2 * n_iter)},
        "clocks": clocks,
    }
    print(json.dumps(line))
    return line


def run_batch(args, rank, world):
    """16 SHLR instances of uneven size (M = N in 128..320, 8..32 coils, window 6) in
    one batched plan: a step is one ADMM iteration of every instance; value =
    instance-iterations per second.  Beside it: the same instances solved by 16
    single-instance plans one after the other."""
    import torch
    from paper_2107_11650_gb300 import api, build

    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
        build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    wls = synth.unrolled_batch()
    inputs = [synth.make_inputs(instance_workload(w, rank)) for w in wls]
    descs = [api.Desc.from_workload(w, max_iter=max(args.warmup, 1), gram=gram_for(args, True)) for w in wls]
    plan = api.BatchPlan(descs)
    Yh = [torch.from_numpy(i["Y"].astype(np.complex64)) for i in inputs]
    Yp = plan.pack([y.cuda() for y in Yh], torch.complex64)
    mp = plan.pack([torch.from_numpy(i["mask"]).cuda() for i in inputs], torch.uint8, mask=True)
    Xp = torch.empty_like(Yp)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        api.selr_solve_batch(plan, Yp, mp, Xp, stream=stream)
    plan.set_iterations(args.steps)
    with torch.cuda.stream(stream):
        api.selr_solve_batch(plan, Yp, mp, Xp, stream=stream)       # capture the graph
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = ClockSampler(dev) if rank == 0 else None
    if clk:
        clk.start()
        time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        api.selr_solve_batch(plan, Yp, mp, Xp, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    clocks = clk.stop() if clk else None
    st = api.selr_sync_status(plan, stream)
    # the same work through 16 single-instance plans, one after the other
    singles = [api.Plan(api.Desc.from_workload(w, max_iter=args.steps, gram=gram_for(args, True))) for w in wls]
    Ys = [plan.unpack(Yp, i).contiguous() for i in range(len(wls))]
    Ms = [torch.from_numpy(i["mask"]).cuda() for i in inputs]
    Xs = [torch.empty_like(y) for y in Ys]
    for sp, y, m, x in zip(singles, Ys, Ms, Xs):
        with torch.cuda.stream(stream):
            api.selr_solve(sp, y, m, x, stream=stream)              # capture
    stream.synchronize()
    e0.record(stream)
    for sp, y, m, x in zip(singles, Ys, Ms, Xs):
        with torch.cuda.stream(stream):
            api.selr_solve(sp, y, m, x, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms_single = max_over_ranks(e0.elapsed_time(e1), world)
    # torch.max propagates NaN (a Python max over floats would not)
    diff = float(torch.stack([(plan.unpack(Xp, i) - Xs[i]).abs().max() / Xs[i].abs().max()
                              for i in range(len(wls))]).max())
    st = max(st, max(api.selr_sync_status(sp, stream) for sp in singles))
    units = len(wls) * args.steps
    if rank != 0:
        return None
    line = {
        "metric": "instance-iterations/s, 16 uneven SHLR instances in one batched plan",
        "value": whole_job_value(world, units, ms), "unit": "instance-iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch_16_uneven", "instances": [f"{w.J}c {w.M}x{w.N}" for w in wls],
                   "window": wls[0].window, "gram": gram_for(args, True),
                   "l2": "lifted state of the batch (GBs) exceeds L2; no flush"},
        "separate_plans": {"value": whole_job_value(world, units, ms_single), "ms_per_step": ms_single / args.steps,
                           "max_rel_diff_vs_batch": diff},
        "roofline": None, "clocks": clocks, "status": st,
    }
    print(json.dumps(line))
    return line


def run_quality(args):
    """Reconstruction quality on the synthetic stand-ins, computed with the library's own
    metric kernels (SSOS, RLNE, MSSIM, T2 fit): the model ablation on one data set and
    mask (SHLR, SHLR-S, SHLR-V, SHLR-SV), the sampling patterns, an ACS-line sweep at a
    fixed sampling rate and the T2 map of the parameter model, each against the
    zero-filled reconstruction.  One JSON line per experiment; not a throughput line."""
    import torch
    from paper_2107_11650_gb300 import api
    from paper_2107_11650_gb300.build import build
    build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    n_iter = 30

    def solve(wl, Y, mask):
        plan = api.Plan(api.Desc.from_workload(wl, max_iter=n_iter, gram="3xtf32"))
        X = torch.empty_like(Y)
        with torch.cuda.stream(stream):
            api.selr_solve(plan, Y, mask, X, stream=stream)           # first call captures the graph
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            api.selr_solve(plan, Y, mask, X, stream=stream)
        e1.record(stream)
        e1.synchronize()
        st = api.selr_sync_status(plan, stream)
        return plan, X, n_iter * 1000.0 / e0.elapsed_time(e1), st

    def zero_filled(plan, Y, two_d):
        with torch.cuda.stream(stream):
            Z = Y.clone()
            if two_d:
                api.selr_transform(plan, 0, True, Z, Z, stream=stream)
            api.selr_transform(plan, 1, True, Z, Z, stream=stream)
        return Z

    def scores(ref_img, X):
        with torch.cuda.stream(stream):
            rec = api.selr_ssos(X, stream=stream)
            rl = api.selr_rlne(ref_img, rec, stream=stream)
            ms, _ = api.selr_mssim(ref_img, rec, stream=stream)
        stream.synchronize()
        return float(rl.item()), float(ms.item())

    def case(wl, Y=None, mask=None, truth=None):
        if Y is None:
            inp = synth.make_inputs(wl)
            Y, mask, truth = inp["Y"], inp["mask"], inp["truth"]
        Yd = torch.from_numpy(Y.astype(np.complex64)).cuda()
        md = torch.from_numpy(mask.astype(np.uint8)).cuda()
        with torch.cuda.stream(stream):
            ref = api.selr_ssos(torch.from_numpy(truth.astype(np.complex64)).cuda(), stream=stream)
        plan, X, its, st = solve(wl, Yd, md)
        rl, ms = scores(ref, X)
        zr, zm = scores(ref, zero_filled(plan, Yd, True))
        plan.close()
        return {"model": wl.model, "rlne": rl, "mssim": ms, "zero_filled_rlne": zr, "zero_filled_mssim": zm,
                "iters_per_s": its, "status": st, "sampling": float(mask.mean())}

    base = synth.get_config("shlr_12c_256")
    lam1 = {"SHLR_S": 1e3, "SHLR_SV": 1e2}
    rows = []
    for model in ("SHLR", "SHLR_S", "SHLR_V", "SHLR_SV"):
        r = case(base.with_(model=model, lam1=lam1.get(model, base.lam1)))
        if model in lam1:
            r["lambda1"] = lam1[model]
        rows.append(r)
    print(json.dumps({"quality": "model_ablation", "workload": "12-coil 256x256, 1D random R=4 + 24 ACS lines",
                      "iterations": n_iter, "rows": rows}))

    rows = []
    for name in ("shlr_12c_256_uniform6", "shlr_12c_256_uniform6_pf34", "shlr_12c_256_gauss_pf34",
                 "shlrv_12c_256", "shlrv_12c_256_poisson_pf45"):
        wl = synth.get_config(name)
        r = case(wl)
        r["workload"] = name
        r["mask"] = f"{wl.mask} R={wl.R} acs={wl.n_acs}" + (f" pf={wl.pf}" if wl.pf < 1.0 else "")
        rows.append(r)
    print(json.dumps({"quality": "sampling_patterns", "iterations": n_iter, "rows": rows}))

    sw = synth.ACS_SWEEP
    x = synth.multicoil_image(base.J, base.M, base.N, base.seed)
    rows = []
    for n_acs, mask in synth.acs_sweep_masks(base.M, base.N, sw["rate"], sw["acs_lines"], base.seed + 101).items():
        Y = synth.acquire_2d(x, mask, base.sigma_n, base.seed)
        sc = 1.0 / np.abs(Y).max()
        for model in ("SHLR", "SHLR_SV"):
            wl = base.with_(model=model, n_acs=n_acs, mask="gauss1d", lam1=lam1.get(model, base.lam1))
            r = case(wl, Y * sc, mask, x * sc)
            r["acs_lines"] = n_acs
            rows.append(r)
    print(json.dumps({"quality": "acs_sweep", "rate": sw["rate"], "iterations": n_iter, "rows": rows}))

    wl = synth.get_config("shlrvp_8c_192_8e")
    inp = synth.make_inputs(wl)
    te = [wl.te_ms * (l + 1) for l in range(wl.L)]
    _, t2_true, m0 = synth.t2_series(wl.J, wl.M, wl.N, wl.L, te, wl.seed)
    Yd = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    md = torch.from_numpy(inp["mask"].astype(np.uint8)).cuda()
    plan, X, its, st = solve(wl, Yd, md)
    support = m0 > 0.1 * m0.max()

    def t2_rlne(Ximg):
        with torch.cuda.stream(stream):
            S = api.selr_ssos(Ximg, stream=stream)
            T2, _ = api.selr_t2_fit(S, te, stream=stream)
        stream.synchronize()
        t2 = T2.cpu().numpy()
        ok = support & np.isfinite(t2)
        fit_frac = float(ok.sum() / support.sum())
        err = float(np.linalg.norm((t2 - t2_true)[ok]) / np.linalg.norm(t2_true[ok]))
        return err, fit_frac

    with torch.cuda.stream(stream):
        ref = api.selr_ssos(torch.from_numpy(inp["truth"].astype(np.complex64)).cuda(), stream=stream)
        rec = api.selr_ssos(X, stream=stream)
        rl = api.selr_rlne(ref, rec, stream=stream)
        Z = zero_filled(plan, Yd, False)
        zr = api.selr_rlne(ref, api.selr_ssos(Z, stream=stream), stream=stream)
    stream.synchronize()
    (t2e, t2f), (zt2e, zt2f) = t2_rlne(X), t2_rlne(Z)
    print(json.dumps({"quality": "t2_map", "workload": "shlrvp_8c_192_8e", "model": wl.model, "iterations": n_iter,
                      "t2_rlne": t2e, "t2_fitted_fraction": t2f, "zero_filled_t2_rlne": zt2e,
                      "zero_filled_t2_fitted_fraction": zt2f, "series_rlne": float(rl.item()),
                      "zero_filled_series_rlne": float(zr.item()), "iters_per_s": its, "status": st,
                      "support": "pixels with M0 > 0.1 max M0 and a fitted T2 in range",
                      "t2_fit_range_ms": [1.0, 1000.0]}))
    plan.close()


def run_iteration_log(args):
    """--steps iterations of --config, one JSON line per iteration (paper_2107_11650_gb300.iterlog)."""
    import torch
    from paper_2107_11650_gb300 import api, iterlog
    from paper_2107_11650_gb300.build import build
    build()
    torch.cuda.set_device(0)
    wl = synth.get_config(args.config)
    inp = synth.make_inputs(wl)
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    mask = torch.from_numpy(inp["mask"].astype(np.uint8)).cuda()
    model2d = wl.model in ("SHLR", "SHLR_V", "SHLR_S", "SHLR_SV")
    plan = api.Plan(api.Desc.from_workload(wl, svd=args.svd, gram=gram_for(args, model2d)))
    X = torch.empty_like(Y)
    stream = torch.cuda.Stream()
    recs = iterlog.run_logged(plan, Y, mask, X, args.steps, args.iteration_log, stream=stream)
    print(json.dumps({"iteration_log": args.iteration_log, "workload": wl.name, "iterations": len(recs),
                      "last": recs[-1]}))
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--exec", default="both", choices=["both", "batched", "plain"])
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--svd", default="eig", choices=["eig", "jacobi"])
    ap.add_argument("--gram", default=None, choices=["fp32", "tf32", "3xtf32", "bf16x3", "bf16x6"],
                    help="Gram precision before autotuning (default: 3xtf32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--reduction", type=int, default=0, choices=[0, 1, 2],
                    help="Householder reduction: 0 by order, 1 one-stage, 2 two-stage where the order allows")
    ap.add_argument("--ev-chunk", type=int, default=0, choices=[0, 8, 16],
                    help="eigenvectors per k_eigvec pass (replaces the autotuner; 0: autotune)")
    ap.add_argument("--allow-tf32", action="store_true")
    ap.add_argument("--quality", action="store_true",
                    help="reconstruction-quality experiments (RLNE / MSSIM / T2) instead of the throughput line")
    ap.add_argument("--iteration-log", default=None, metavar="PATH",
                    help="write a per-iteration JSONL log of --steps iterations of --config to PATH "
                         "instead of the throughput line")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl" if args.impl == "ours" else "gloo")

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.quality:
        if rank == 0:
            run_quality(args)
        return
    if args.iteration_log:
        if rank == 0:
            run_iteration_log(args)
        return
    if args.config == "unrolled_16_uneven":
        run_unrolled(args, rank, world)
        return
    if args.config == "batch_16_uneven":
        run_batch(args, rank, world)
        return

    results, jac, e2e, wl = run_gpu(args, rank, world)
    if rank != 0:
        return
    b = results["batched"]
    value = whole_job_value(world, b["steps"], b["ms"])
    from paper_2107_11650_gb300 import api
    peaks = _peaks()
    mp = measured_peaks(api)
    smax = peaks.get("sm_max_mhz", 2070.0)
    if "fp32_tflops" in mp:
        fp32_peak, fp32_src = mp["fp32_tflops"], ("measured: selr_probe_fp32_peak, FP32 FMA chains on every SM "
                                                  f"(FFMA {mp['fp32_ffma_tflops']:.1f}, FFMA2 "
                                                  f"{mp['fp32_ffma2_tflops']:.1f} TFLOP/s; the larger)")
    else:
        fp32_peak, fp32_src = 152 * 128 * 2 * smax * 1e6 / 1e12, "derived: 152 SMs x 128 lanes x 2 x max SM clock"
    tf32_peak = mp.get("tf32_tflops")
    achieved = jac["flops"] / (jac["ms"] / 1000.0) / 1e12
    gram = (results.get("tuning") or {}).get("gram", gram_for(args, wl.model in ("SHLR", "SHLR_V", "SHLR_S", "SHLR_SV")))
    fk = jac["flops_by_kind"]
    bf16 = peaks.get("bf16_tflops")
    p_tc = {"fp32": fp32_peak, "tf32": tf32_peak, "3xtf32": (tf32_peak / 3.0) if tf32_peak else None,
            "bf16x3": (bf16 / 3.0) if bf16 else None, "bf16x6": (bf16 / 6.0) if bf16 else None}.get(gram)
    hbm = peaks.get("hbm_gbs", 6800.3)
    t_star = None
    if p_tc:
        t_star = 1e3 * (fk["gram"] / (p_tc * 1e12)
                        + (fk["tridiag"] + fk["eigvec"] + fk["apply"] + fk["small_svt"]) / (fp32_peak * 1e12)
                        + jac["bytes"] / (hbm * 1e9))
    t_meas = b["ms"] / b["steps"]
    two_stage = results["plan"].tuning()["reduction"] == 2 if args.svd == "eig" else False
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": b["steps"],
        "warmup": args.warmup, "ms_per_step": b["ms"] / b["steps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "coils": wl.J, "size": [wl.M, wl.N], "window": wl.window,
                   "model": wl.model, "mask": f"{wl.mask} R={wl.R} acs={wl.n_acs}",
                   "matrices_per_step": b["nmat"], "exec": "batched (graph-captured)", "svd": args.svd,
                   "gram": (results.get("tuning") or {}).get("gram", gram_for(args, wl.model in ("SHLR", "SHLR_V", "SHLR_S", "SHLR_SV"))),
                   "l2": "per-step state (D, E, work copies: 760 MB) exceeds L2; no flush"},
        "plain": ({"value": whole_job_value(world, results["plain"]["steps"], results["plain"]["ms"]),
                   "ms_per_step": results["plain"]["ms"] / results["plain"]["steps"],
                   "steps": results["plain"]["steps"]} if "plain" in results else None),
        "roofline": {"bound": "alu",
                     "kernel": ("k_jacobi (one-sided Jacobi SVD)" if args.svd == "jacobi" else
                                "k_sb1 + k_sb2 + k_eigvec (two-stage Householder reduction, multisection, "
                                "inverse iteration and back-transformation of the pairs above t^2)" if two_stage else
                                "k_tridiag + k_eigvec (Householder tridiagonalisation, multisection, inverse "
                                "iteration and back-transformation of the pairs above t^2)"),
                     "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": svd_traffic(jac.get("eig_shapes")) if args.svd == "eig" and not two_stage else None,
                     "traffic_unit": "bytes per launch (ncu capture of the same kernels, scaled per matrix)",
                     "peak_source": fp32_src,
                     "flops_per_launch": jac["flops"], "launch_ms": jac["ms"],
                     "flop_model": "(16/3) s^3 + (8 s^2 + 1626 s) r per matrix, r = mean rank over the timed "
                                   "iterations", "mean_rank": jac["mean_rank"]},
        "step_bound": {"T_star_ms": t_star, "T_ms": t_meas, "frac": (t_star / t_meas) if t_star else None,
                       "formula": "F_gram / P_gram + F_fp32 / P_fp32 + bytes / BW_hbm",
                       "flops": fk, "bytes": jac["bytes"], "gram": gram,
                       "peaks": {"fp32_tflops": fp32_peak, "tf32_tflops": tf32_peak,
                                 "gram_tflops": p_tc, "hbm_gbs": hbm,
                                 "hbm_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback"}},
        "e2e": {"value": e2e["value"], "unit": "iters/s", "h2d_bytes_per_step": e2e["h2d"],
                "d2h_bytes_per_step": e2e["d2h"]},
        "stages_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in b["stages"].items()},
        "gpu_launches": b["launches"],
        "clocks": b["clocks"],
        "status": b["status"],
        "accuracy": results.get("accuracy"),
        "tuning": results.get("tuning"),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
