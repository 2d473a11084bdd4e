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
def kernel_launches_per_iteration(plan, model2d, exec_mode, svd="eig"):
    """Kernels libselr launches per ADMM iteration (mirrors admm_stage and svd_apply in
    selr.cu): adjoint, FFTs of the adjoints, DC + reduction, hybrid FFTs, lift, and the
    SVT kernels: either the warp-per-matrix SVT (s <= 8, len <= 64) or Gram, tridiagonal
    reduction, eigenvectors and the three apply kernels (streaming for r <= 32 and
    32 < r <= 64 pairs, general above) (eig), Jacobi and apply (jacobi).  Batched, one
    SVT launch sequence covers each run of consecutive lift families of the same SVT
    size class (svt_class in selr.cu); plain, one per matrix."""
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

    def svt_kernels(r, c):
        return 1 if svt_class(r, c) == 0 else (6 if svd == "eig" else 2)

    if exec_mode == "batched":
        classes = [svt_class(r, c) for _, r, c in fams]
        runs = [k for i, k in enumerate(classes) if i == 0 or k != classes[i - 1]]
        per = 1 + fft_a + 2 + fft_a + 1 + sum(1 if k == 0 else (6 if svd == "eig" else 2) for k in runs)
    else:
        nmat = sum(nm for nm, _, _ in fams)
        per = nmat + fft_a + 2 + fft_a + sum(nm * (1 + svt_kernels(r, c)) for nm, r, c in fams)
    return per + (0 if model2d else 1)


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
    """Algorithmic flops of one SVD (Gram + Hermitian eigensolve convention): 8 l s^2 + 36 s^3."""
    return 8.0 * l * s * s + 36.0 * s ** 3


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
    model2d = wl.model in ("SHLR", "SHLR_V")
    modes = ["batched", "plain"] if args.exec == "both" else [args.exec]
    for mode in modes:
        plan = api.Plan(api.Desc.from_workload(wl, exec=mode, max_iter=max(args.warmup, 1), svd=args.svd,
                                               gram=gram_for(args, model2d)))
        nmat = sum(plan.lift_shape(a)[0] for a in (("row", "col") if model2d else ("pe", "param")))
        with torch.cuda.stream(stream):
            api.selr_solve(plan, Y, mask, X, stream=stream)           # W warm-up iterations
        st = api.selr_sync_status(plan, stream)
        if mode == "batched" and not args.no_autotune:
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
                             launches=steps * kernel_launches_per_iteration(plan, model2d, mode, args.svd) + 6)
        if mode == "batched":
            results["plan"] = plan
        else:
            plan.close()
    plan = results["plan"]
    st_ = results["batched"]["stages"]
    # algorithmic flops per launch of each SVT stage, summed over both lift families:
    # 8 l s^2 (Gram), 36 s^3 (Hermitian eigensolve), 8 l s^2 (apply)
    algo = {"gram": 0.0, "svd": 0.0, "apply": 0.0}
    for ax in (("row", "col") if model2d else ("pe", "param")):
        nm_, r_, c_ = plan.lift_shape(ax)
        l, s = max(r_, c_), min(r_, c_)
        algo["gram"] += nm_ * 8.0 * l * s * s
        algo["apply"] += nm_ * 8.0 * l * s * s
        algo["svd"] += nm_ * (flops_svd_per_matrix(l, s) if args.svd == "jacobi" else 36.0 * s ** 3)
    dom = max(algo, key=lambda k: st_[k][0])
    ms_dom = st_[dom][0] / max(st_[dom][1], 1)
    jac = dict(ms=ms_dom, flops=algo[dom], stage=dom)
    e2e = time_e2e(plan, Yh, mh, stream, reps=2)
    e2e_ms = max_over_ranks(1000.0 * plan.desc.max_iter / e2e["value"], world)
    e2e["value"] = whole_job_value(world, plan.desc.max_iter, e2e_ms)
    results["accuracy"] = accuracy_vs_oracle(plan, wl, Y, mask, stream) if rank == 0 else None
    return results, jac, e2e, wl


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


def oracle_sample(wl, frac_mats=64):
    """One bounded oracle step: the full X-update plus the SVTs of a sample of
    the lifted matrices (the SVT is where the oracle's time goes).  2D models:
    `frac_mats` row lifts; parameter models: the same fraction of the PE and
    of the parameter lifts.  Returns (seconds, fraction of one iteration's
    SVT work done)."""
    from oracle import admm as oadmm
    from oracle.svt import svt
    if wl.name not in _ORACLE_CACHE:
        _ORACLE_CACHE[wl.name] = synth.make_inputs(wl)
    inp = _ORACLE_CACHE[wl.name]
    b = wl.beta
    if wl.model in ("SHLR", "SHLR_V"):
        s = oadmm.Shlr2D(inp["Y"], inp["mask"], wl)
        st = s.init_state()
        t0 = time.perf_counter()
        K = s.x_update(st["Zr"], st["Zc"], st["Dr"], st["Dc"])
        LXr, LXc = s.lifts(K)
        Z = svt(LXr[:frac_mats] + st["Dr"][:frac_mats] / b, 1.0 / b)
        _ = st["Dr"][:frac_mats] + wl.tau * (LXr[:frac_mats] - Z)
        dt = time.perf_counter() - t0
        return dt, frac_mats / (LXr.shape[0] + LXc.shape[0])
    s = oadmm.ShlrParam(inp["Y"], inp["mask"], wl)
    st = s.init_state()
    t0 = time.perf_counter()
    K = s.x_update(st["Zpe"], st["Zp"], st["Dpe"], st["Dp"])
    LXpe, LXp = s.lifts(K)
    npe = max(1, LXpe.shape[0] * frac_mats // 512)
    npp = max(1, LXp.shape[0] * frac_mats // 512)
    Z1 = svt(LXpe[:npe] + st["Dpe"][:npe] / b, 1.0 / b)
    Z2 = svt(LXp[:npp] + st["Dp"][:npp] / b, wl.lam2 / b)
    _ = (st["Dpe"][:npe] + wl.tau * (LXpe[:npe] - Z1), st["Dp"][:npp] + wl.tau * (LXp[:npp] - Z2))
    dt = time.perf_counter() - t0
    return dt, npe / LXpe.shape[0]


def cpu_baseline(wl, steps=1):
    vals = []
    for _ in range(steps):
        dt, frac = oracle_sample(wl)
        vals.append(frac / dt)             # iterations/s (scaled by the SVT fraction)
    return {"value": float(np.median(vals)), "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 NumPy oracle on {wl.name}: full X-update + SVTs of 1/8 of the lifted matrices of one "
                      "ADMM iteration, scaled to a full iteration by that fraction"}


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
    if world > 1 and rank != 0:
        return None
    if args.config == "unrolled_16_uneven":
        return run_reference_unrolled(args)
    wl = synth.get_config(args.config)
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle_sample(wl, frac_mats=8)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dt, frac = oracle_sample(wl, frac_mats=16)
        vals.append(frac / dt)
    wall = time.perf_counter() - t0
    v = float(np.median(vals))
    line = {"metric": METRIC, "value": v, "unit": "iters/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wl.name, "coils": wl.J, "size": [wl.M, wl.N], "window": wl.window,
                       "model": wl.model, "mask": f"{wl.mask} R={wl.R} acs={wl.n_acs}"},
            "cpu_baseline": {"value": v, "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "per step: full X-update + SVTs of 16 of 512 lifted matrices, "
                                       "scaled to one iteration by the SVT share"},
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
    ap.add_argument("--gram", default=None, choices=["fp32", "tf32", "3xtf32"],
                    help="Gram precision before autotuning (default: 3xtf32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--allow-tf32", action="store_true")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl" if args.impl == "ours" else "gloo")

    if args.impl == "reference":
        run_reference(args, rank, world)
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
    peaks = _peaks()
    smax = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * smax * 1e6 / 1e12          # TFLOP/s, FP32 FMA pipe at max SM clock
    achieved = jac["flops"] / (jac["ms"] / 1000.0) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": b["steps"],
        "warmup": args.warmup, "ms_per_step": b["ms"] / b["steps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "coils": wl.J, "size": [wl.M, wl.N], "window": wl.window,
                   "model": wl.model, "mask": f"{wl.mask} R={wl.R} acs={wl.n_acs}",
                   "matrices_per_step": b["nmat"], "exec": "batched (graph-captured)", "svd": args.svd,
                   "gram": (results.get("tuning") or {}).get("gram", gram_for(args, wl.model in ("SHLR", "SHLR_V"))),
                   "l2": "per-step state (D, E, work copies: 760 MB) exceeds L2; no flush"},
        "plain": ({"value": whole_job_value(world, results["plain"]["steps"], results["plain"]["ms"]),
                   "ms_per_step": results["plain"]["ms"] / results["plain"]["steps"],
                   "steps": results["plain"]["steps"]} if "plain" in results else None),
        "roofline": {"bound": "alu", "kernel": {"gram": "k_gram (Gram matrices of all 512 lifts)",
                                                "svd": ("k_jacobi (one-sided Jacobi SVD)" if args.svd == "jacobi" else
                                                        "k_tridiag + k_eigvec (Householder tridiagonal eigensolver, eigenpairs above t^2)"),
                                                "apply": "k_apply_stream (Z and multiplier update)"}[jac["stage"]],
                     "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": None, "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock",
                     "launch_ms": jac["ms"]},
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
