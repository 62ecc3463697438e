#!/usr/bin/env python
"""Benchmark of the DIA kernel fit on GB300.

One step = one full fit of a reference/target pair through the C ABI
(dia_fit): initialisation, Adam then L-BFGS (each iteration one fused
forward/loss/backward pass, a float64 reduction and a float64 optimiser step,
replayed from a CUDA graph), the sigma-clipped refits and the difference
image.  Default workload: a 4096 x 4096 crowded field (60,000 stars), 25 x 25
kernel, 2% masked pixels, Cauchy loss with 3 clip-and-refit passes.

value  = loss+gradient evaluations per second over the whole job (all ranks);
         pair fits per second is reported beside it (fits_per_s).
e2e    = the same metric with the images in pinned HOST memory: the library
         stages them to the device and returns theta, K, B0 and the difference
         image to the host inside the timed region.
roofline: the fused evaluation kernel, FP32 FMA pipe (4 m^2 flops per unmasked
         valid pixel, forward + weight gradient) against 152 SMs x 128 lanes x
         2 flops x the maximum SM clock.
cpu_baseline / --impl reference: the FP64 CPU oracle (plain C loops, OpenMP)
         on a bounded crop of the same pair, scaled to the full pixel count.

Multi-GPU (torchrun): each rank fits its own independent pair (seed + rank),
no collective on the data path; the barrier and max-over-ranks timing follow
the launch contract ("scaling": "weak").
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
sys.path.insert(0, ROOT)

from paper_2104_13715_gb300 import shard, synth  # noqa: E402

METRIC = ("pair fits/s and loss+grad evals/s (4096², m=25) vs plain FP32; "
          "err vs FP64 oracle")
DEFAULT_WORKLOAD = "ccd4096_m25_cauchy_clip3"
L2_BYTES = 129 * 2 ** 20


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

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
        if self._t:
            self._t.join(timeout=2)
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
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_source_sha():
    """Hash of the fused kernel's source and of its m = 25 tile variants."""
    h = hashlib.sha256()
    for f in ("dia_eval.cuh", "dia_eval_m25.cu"):
        with open(os.path.join(ROOT, "paper_2104_13715_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_record(name="fused_eval_m25_4096"):
    """DRAM bytes per launch of the fused kernel from the committed ncu record
    (profiles/<name>.json, written from the same capture as the summary
    beside it), if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", name + ".json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_sha256_16") != kernel_source_sha():
        return None
    v = rec.get("dram_bytes_per_launch")
    return float(v) if isinstance(v, (int, float)) else None


def _loss_kw(d):
    return {k: v for k, v in d["loss"].items()
            if k in ("rho", "noise", "sigma0", "gain", "excess", "huber_c", "var", "var_floor")}


def _oracle_spec(d):
    import oracle
    keys = ("rho", "noise", "sigma0", "gain", "excess", "huber_c", "var", "var_floor")
    lk = dict(d["loss"])
    if lk.get("noise", "fixed") == "fixed":
        lk.pop("sigma0", None)
        lk.pop("gain", None)
    return oracle.LossSpec(**{k: lk[k] for k in keys if k in lk})


def _crop(d, side):
    """Top-left side x side crop of a pair (same recipe, fewer pixels)."""
    out = dict(d)
    for k in ("R", "I", "mask", "var"):
        if d.get(k) is not None:
            out[k] = np.ascontiguousarray(d[k][:side, :side])
    return out


def cpu_model():
    """Host CPU model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def _theta_boxcar(d):
    m = d["m"]
    th = np.full(m * m + 1, 1.0 / (m * m))
    th[-1] = float(np.median(d["I"]))
    return th


def oracle_evals(d, n, nthreads=0):
    """Run n FP64 oracle loss+gradient evaluations of the whole pair at the
    box-car start; returns the seconds taken."""
    import oracle
    m = d["m"]
    spec = _oracle_spec(d)
    th = _theta_boxcar(d)
    t0 = time.perf_counter()
    for _ in range(n):
        oracle.loss_grad(d["R"], d["I"], m, th, spec, mask=d.get("mask"), var=d.get("var"),
                         nthreads=nthreads)
    return time.perf_counter() - t0


def oracle_rate(d, budget_s=15.0, max_evals=50):
    """FP64 oracle loss+gradient evaluations per second on the whole pair
    (all host cores), as many as fit in budget_s (at least one), plus a
    single-thread figure from one evaluation of a 1024^2 crop scaled by valid
    pixel count.  Returns (rate, cores, sample, extra)."""
    cores = os.cpu_count() or 1
    n, dt = 0, 0.0
    while n < max_evals and (n == 0 or dt < budget_s):
        dt += oracle_evals(d, 1, nthreads=cores)
        n += 1
    h = d["m"] // 2
    px_f = (d["R"].shape[0] - 2 * h) * (d["R"].shape[1] - 2 * h)
    c = _crop(d, min(1024, d["R"].shape[0]))
    px_c = (c["R"].shape[0] - 2 * h) * (c["R"].shape[1] - 2 * h)
    t1 = oracle_evals(c, 1, nthreads=1)
    extra = {"cpu_model": cpu_model(),
             "single_thread_evals_per_s": px_c / px_f / t1,
             "single_thread_sample": f"one evaluation of a {c['R'].shape[0]}x{c['R'].shape[1]} "
                                     f"crop ({px_c} valid px) on one thread in {t1:.2f} s, "
                                     f"scaled by valid pixel count"}
    sample = (f"{n} FP64 loss+gradient evaluations of the oracle on the whole "
              f"{d['R'].shape[0]}x{d['R'].shape[1]} pair ({px_f} valid px) at the box-car "
              f"start in {dt:.1f} s on {cores} threads")
    return n / dt, cores, sample, extra


# ------------------------------------------------------------------ arms
def run_reference(args, rank, world):
    """The FP64 oracle as it stands, on the same pair: one whole-pair
    loss+gradient evaluation per step on all host cores."""
    if rank != 0:
        return
    d = synth.workload(args.workload, seed=args.seed)
    cores = os.cpu_count() or 1
    oracle_evals(d, args.warmup, nthreads=cores)
    dt = oracle_evals(d, args.steps, nthreads=cores)
    value = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args, d),
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": f"one FP64 loss+gradient evaluation of the whole "
                                   f"{d['R'].shape[0]}x{d['R'].shape[1]} pair per step, "
                                   f"{cores} threads", "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(args, d):
    H, W = d["R"].shape
    m = d["m"]
    by = sum(d[k].nbytes for k in ("R", "I", "mask", "var") if d.get(k) is not None)
    return {"workload": args.workload, "H": H, "W": W, "m": m, "loss": d["loss"].get("rho"),
            "variance": d["loss"].get("noise"), "clip_passes": d["loss"].get("clip_passes", 0),
            "masked_frac": None if d.get("mask") is None else float(1 - d["mask"].mean()),
            "seeds": [args.seed + r for r in range(_env_int("WORLD_SIZE", 1))],
            "l2": f"inputs larger than L2 ({by / 2**20:.0f} MiB > {L2_BYTES / 2**20:.0f} MiB)",
            "init": "box-car K, B0 = median(I) (Sec. 2.9)",
            "optimizer": "Adam -> L-BFGS (Gauss-Newton preconditioned, library defaults)"}


def oracle_check(nat, d, R, I, m, spec, opts, mask, var, ws, stream, out_plain, th_init):
    """K, B0 and difference-image errors of the fit against the FP64 oracle's
    optimum theta*: theta* = theta_gpu + one Newton step with the oracle's
    exact FP64 Hessian, on the mask the fit itself returned (its clip
    decisions, taken in float32, are the fit's; the oracle optimises on that
    mask).  Also the oracle's max|dL/dtheta| at theta_gpu and at theta*,
    relative to the box-car start."""
    import oracle
    out = nat.fit(R, I, m, spec, opts, mask=mask, var=var, ws=ws, stream=stream,
                  want_diff=True, want_mask=opts.clip_passes > 0)
    th = out["theta"].cpu().numpy()
    fmask = out["mask"].cpu().numpy() if opts.clip_passes > 0 else d.get("mask")
    spec_o = _oracle_spec(d)
    kw = dict(mask=fmask, var=d.get("var"))
    t0 = time.perf_counter()
    ref = oracle.newton(d["R"], d["I"], m, th, spec_o, max_iter=1, **kw)
    t_newton = time.perf_counter() - t0
    _, g_fit = oracle.loss_grad(d["R"], d["I"], m, th, spec_o, **kw)
    _, g_ref = oracle.loss_grad(d["R"], d["I"], m, ref, spec_o, **kw)
    _, g_ini = oracle.loss_grad(d["R"], d["I"], m, th_init, spec_o, **kw)
    D_ref = oracle.diff_image(d["R"], d["I"], m, ref)
    D = out["diff"].cpu().numpy()
    h = m // 2
    sky = float(np.median(d["I"]))
    vv = d.get("var")
    sig_med = float(np.sqrt(np.median(vv[h:-h, h:-h]))) if vv is not None else float(
        np.sqrt(_loss_kw(d).get("var", 1.0)))
    sumK = abs(ref[:-1].sum())
    th_pl = out_plain["theta"].cpu().numpy()
    gi = np.max(np.abs(g_ini))
    return {"_ref": (ref, D_ref), "err_K": float(np.max(np.abs(th[:-1] - ref[:-1])) / sumK),
            "err_B0": float(abs(th[-1] - ref[-1]) / sky),
            "err_D": float(np.max(np.abs(D - D_ref)) / sig_med),
            "err_D_rel_maxI": float(np.max(np.abs(D - D_ref)) / np.max(np.abs(d["I"]))),
            "plain_K_err_rel_sumK": float(np.max(np.abs(th_pl[:-1] - ref[:-1])) / sumK),
            "oracle_grad_ratio": float(np.max(np.abs(g_fit)) / gi),
            "oracle_grad_ratio_polished": float(np.max(np.abs(g_ref)) / gi),
            "P": float(th[:-1].sum()), "B0": float(th[-1]),
            "tolerances": {"err_K": 1e-4, "err_B0": 1e-4},
            "what": "err_K = max|K - K*| / |sum K*|, err_B0 = |B0 - B0*| / median(I), "
                    "err_D = max|D - D*| / sigma_median, theta* = theta_gpu + one FP64 "
                    f"Newton step of the oracle on the fit's final mask ({t_newton:.0f} s on "
                    f"{os.cpu_count()} host cores)"}


def batch_subset(nat, dev, stream, n, seed):
    """The first n pairs of the batch workload fitted three ways: batched
    (one dia_fit_batch call, graph-captured), one at a time in the plain form
    (no graph) and one at a time with the graph; fits/s of each and the max
    K error (relative to sum K*) against the oracle's normal-equation solve."""
    import oracle
    import torch
    ds = synth.batch(n, seed=seed)
    items = [dict(R=torch.from_numpy(x["R"]).to(dev), I=torch.from_numpy(x["I"]).to(dev),
                  m=x["m"]) for x in ds]
    spec = nat.loss_spec(rho="gauss", noise="fixed", var=1.0)
    refs = [oracle.normal_solve(x["R"], x["I"], x["m"]) for x in ds]

    def kerr(thetas):
        return float(max(np.max(np.abs(t[:-1] - r[:-1])) / abs(r[:-1].sum())
                         for t, r in zip(thetas, refs)))

    res = {"pairs": n}
    opts = nat.default_opts(timeout_s=900.0)
    nat.fit_batch(items, spec, opts, stream=stream)   # warm-up (graph capture)
    for mode in ("batch", "single_plain", "single_graph"):
        o = nat.default_opts(use_graph=0 if mode == "single_plain" else 1, timeout_s=900.0)
        if mode != "batch":
            nat.fit(items[0]["R"], items[0]["I"], items[0]["m"], spec, o, want_diff=False,
                    stream=stream)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        if mode == "batch":
            thetas = [t.cpu().numpy() for t in nat.fit_batch(items, spec, opts,
                                                             stream=stream)["thetas"]]
        else:
            thetas = [nat.fit(it["R"], it["I"], it["m"], spec, o, want_diff=False,
                              stream=stream)["theta"] for it in items]
            torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        if mode != "batch":
            thetas = [t.cpu().numpy() for t in thetas]
        res[mode] = {"fits_per_s": n / dt, "K_err_rel_sumK": kerr(thetas)}
    res["batch_over_single_plain"] = res["batch"]["fits_per_s"] / res["single_plain"]["fits_per_s"]
    res["what"] = ("first pairs of the batch recipe (side 64-512, m 7-21, chi^2): batched vs "
                   "one at a time plain (no graph) and with the graph; host wall clock "
                   "around each; K error against the oracle's normal-equation solve")
    return res


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2104_13715_gb300 import native as nat

    dist = None
    if world > 1:
        import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    d = synth.workload(args.workload, seed=args.seed + rank)
    m = d["m"]
    H, W = d["R"].shape
    h = m // 2

    # CPU baseline first (rank 0, N=1 only), before the GPU is busy
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, sample, extra = oracle_rate(d, budget_s=args.ref_budget)
        cpu = {"value": r, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample,
               **extra}

    def up(a, dt):
        return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)

    R, I = up(d["R"], torch.float32), up(d["I"], torch.float32)
    mask, var = up(d.get("mask"), torch.uint8), up(d.get("var"), torch.float32)
    spec = nat.loss_spec(**_loss_kw(d))
    opts = nat.default_opts(clip_passes=int(d["loss"].get("clip_passes", 0)),
                            clip_kappa=float(d["loss"].get("kappa", 5.0)))
    clip = opts.clip_passes > 0
    ws = nat.workspace(H, W, m, clip=clip, device=dev)
    stream = torch.cuda.current_stream(dev)
    # tile shape of the fused kernel for this (m, image size): autotuned, cached
    from paper_2104_13715_gb300 import autotune
    tuned = autotune.tune(R, I, m, spec, mask=mask, var=var, stream=stream)

    def step():
        return nat.fit(R, I, m, spec, opts, mask=mask, var=var, ws=ws, stream=stream,
                       want_diff=True)

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local_rank) if local_rank == 0 else None
    if sampler:
        sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evals = 0
    launches = 0
    infos = []
    e0.record(stream)
    for _ in range(args.steps):
        out = step()
        evals += out["info"]["evals"]
        launches += out["info"]["kernel_launches"]
        infos.append(out["info"])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms, float(evals)], dtype=torch.float64, device=dev)
    if dist:
        tmax = t.clone()
        dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
        tsum = t.clone()
        dist.all_reduce(tsum[1:], op=dist.ReduceOp.SUM)
        ms_max, evals_all = float(tmax[0]), float(tsum[1])
    else:
        ms_max, evals_all = ms, float(evals)
    value = evals_all / (ms_max / 1000.0)
    fits_per_s = args.steps * world / (ms_max / 1000.0)

    # roofline of the fused evaluation kernel: its launches alone, each bracketed
    # by CUDA events on the stream, L2 overwritten before each (dia_time_eval)
    th0 = torch.full((m * m + 1,), 1.0 / (m * m), dtype=torch.float64, device=dev)
    th0[-1] = float(np.median(d["I"]))
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    nat.time_eval(R, I, m, th0, spec, mask=mask, var=var, reps=3, flush=flush, ws=ws,
                  stream=stream)
    t_eval = nat.time_eval(R, I, m, th0, spec, mask=mask, var=var, reps=args.kernel_evals,
                           flush=flush, ws=ws, stream=stream) / 1000.0
    del flush
    npx = int(d["mask"][h:H - h, h:W - h].sum()) if d.get("mask") is not None else (H - 2 * h) * (W - 2 * h)
    flops = 4.0 * m * m * npx
    peaks, src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tf = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = flops / t_eval / 1e12
    traffic = _traffic_record()
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
            "frac": achieved / peak_tf, "traffic": traffic,
            "kernel": "dia::eval_kernel (fused forward + loss + weight gradient), tile " +
                      json.dumps(nat.kernel_variant_desc(m)),
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz (max SM clock, "
                          f"{src} peaks file); FP32 FMA pipe",
            "algorithmic": f"4*m^2 flop x {npx} unmasked valid px = {flops / 1e9:.2f} GFLOP per launch",
            "eval_ms": t_eval * 1e3,
            "timing": f"dia_time_eval: mean of {args.kernel_evals} launches, each between CUDA "
                      f"events on the launching stream after reading {2 * L2_BYTES >> 20} MiB "
                      f"through L2 (L2 flushed, no dirty lines)"}

    # the same fit without the Adam phase (preconditioned L-BFGS from the start)
    o_off = nat.default_opts(clip_passes=opts.clip_passes, clip_kappa=opts.clip_kappa,
                             max_adam_iters=0)
    step_off = lambda: nat.fit(R, I, m, spec, o_off, mask=mask, var=var, ws=ws, stream=stream,
                               want_diff=True)
    step_off()
    torch.cuda.synchronize(dev)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_off, ev_off = max(1, min(args.steps, 3)), 0
    a0.record(stream)
    for _ in range(n_off):
        ev_off += step_off()["info"]["evals"]
    a1.record(stream)
    torch.cuda.synchronize(dev)
    ms_off = a0.elapsed_time(a1)
    adam_off = {"fits_per_s": n_off / (ms_off / 1e3), "evals_per_fit": ev_off / n_off,
                "what": "same fits with max_adam_iters = 0 (the library default keeps the "
                        "paper's Adam phase)"}

    # e2e: the same fits with the pair in pinned host memory (library stages it)
    e2e = None
    if not args.no_e2e:
        hR = torch.from_numpy(d["R"]).pin_memory()
        hI = torch.from_numpy(d["I"]).pin_memory()
        hM = torch.from_numpy(d["mask"]).pin_memory() if d.get("mask") is not None else None
        hV = torch.from_numpy(d["var"]).pin_memory() if d.get("var") is not None else None
        wsh = nat.workspace(H, W, m, clip=clip, host=True, device=dev)
        out = nat.fit(hR, hI, m, spec, opts, mask=hM, var=hV, ws=wsh, stream=stream)
        out = None
        out = nat.fit(hR, hI, m, spec, opts, mask=hM, var=hV, ws=wsh, stream=stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev2 = 0
        n2 = max(1, min(args.steps, 3))
        g0.record(stream)
        for _ in range(n2):
            # the previous result is released first, so that its pinned output
            # buffers return to PyTorch's host cache and are reused, as a caller
            # keeping one set of output buffers would
            out = None
            out = nat.fit(hR, hI, m, spec, opts, mask=hM, var=hV, ws=wsh, stream=stream)
            ev2 += out["info"]["evals"]
        g1.record(stream)
        torch.cuda.synchronize(dev)
        ms2 = g0.elapsed_time(g1)
        t2 = torch.tensor([ms2, float(ev2)], dtype=torch.float64, device=dev)
        if dist:
            a = t2.clone()
            dist.all_reduce(a[:1], op=dist.ReduceOp.MAX)
            b = t2.clone()
            dist.all_reduce(b[1:], op=dist.ReduceOp.SUM)
            ms2, ev2 = float(a[0]), float(b[1])
        h2d = sum(t.numel() * t.element_size() for t in (hR, hI, hM, hV) if t is not None)
        d2h = (m * m + 1) * 8 + m * m * 4 + 4 + (H - 2 * h) * (W - 2 * h) * 4
        e2e = {"value": ev2 / (ms2 / 1000.0), "unit": "evals/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "fits_per_s": n2 * world / (ms2 / 1000.0)}

    # the plain form: the same fit with every optimiser iteration launched one
    # by one (no CUDA graph), one pair at a time
    o_plain = nat.default_opts(clip_passes=opts.clip_passes, clip_kappa=opts.clip_kappa,
                               use_graph=0)
    nat.fit(R, I, m, spec, o_plain, mask=mask, var=var, ws=ws, stream=stream, want_diff=True)
    torch.cuda.synchronize(dev)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_pl, ev_pl = max(1, min(args.steps, 3)), 0
    p0.record(stream)
    for _ in range(n_pl):
        out_pl = nat.fit(R, I, m, spec, o_plain, mask=mask, var=var, ws=ws, stream=stream,
                         want_diff=True)
        ev_pl += out_pl["info"]["evals"]
    p1.record(stream)
    torch.cuda.synchronize(dev)
    ms_pl = p0.elapsed_time(p1)
    plain = {"value": ev_pl / (ms_pl / 1e3), "unit": "evals/s",
             "fits_per_s": n_pl / (ms_pl / 1e3), "evals_per_fit": ev_pl / n_pl,
             "what": "the same fit, optimiser iterations launched one by one (use_graph = 0)"}

    # error vs the FP64 oracle: one Newton step (exact FP64 Hessian) from the
    # fitted theta on the fit's own final mask gives the oracle's optimum
    # theta* to second order; K, B0 and D are compared with it (outside the
    # timed region)
    err = None
    if rank == 0 and not args.no_oracle_check:
        err = oracle_check(nat, d, R, I, m, spec, opts, mask, var, ws, stream, out_pl,
                           th0.cpu().numpy())
        plain["K_err_rel_sumK"] = err.pop("plain_K_err_rel_sumK", None)

    batch_sub = None
    if rank == 0 and world == 1 and args.subset > 0 and not args.no_batch_subset:
        batch_sub = batch_subset(nat, dev, stream, args.subset, args.seed)

    # the same fits with both contractions on the tensor cores (dia_set_eval_form),
    # last, so that a failure there cannot take the figures above with it
    tc_form, out_tc = None, None
    ref_pack = err.pop("_ref", None) if err else None
    if not args.no_tc_form and m <= 31 and "bg_degree" not in d["loss"]:
        try:
            nat.set_eval_form(nat.EVAL_TC)
            try:
                ws_tc = nat.workspace(H, W, m, clip=clip, device=dev)
                step_tc = lambda: nat.fit(R, I, m, spec, opts, mask=mask, var=var, ws=ws_tc,
                                          stream=stream, want_diff=True)
                step_tc()
                torch.cuda.synchronize(dev)
                q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                n_tc, ev_tc, l_tc = max(1, min(args.steps, 3)), 0, 0
                q0.record(stream)
                for _ in range(n_tc):
                    out_tc = step_tc()
                    ev_tc += out_tc["info"]["evals"]
                    l_tc += out_tc["info"]["kernel_launches"]
                q1.record(stream)
                torch.cuda.synchronize(dev)
                ms_tc = q0.elapsed_time(q1)
                flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
                t_tc = nat.time_eval(R, I, m, th0, spec, mask=mask, var=var,
                                     reps=args.kernel_evals, flush=flush, ws=ws_tc, stream=stream)
                del flush, ws_tc
            finally:
                nat.set_eval_form(nat.EVAL_FP32)
            tc_form = {"value": ev_tc / (ms_tc / 1e3), "unit": "evals/s",
                       "fits_per_s": n_tc / (ms_tc / 1e3), "evals_per_fit": ev_tc / n_tc,
                       "eval_ms": t_tc, "eval_ms_fp32": t_eval * 1e3,
                       "gpu_launches_per_fit": l_tc / n_tc, "status": out_tc["info"]["status"],
                       "what": "the same fits with dia_set_eval_form(DIA_EVAL_TC): forward pass "
                               "(split bf16) with the g map and loss sums in its epilogue, weight "
                               "gradient (split fp16) on the tensor cores; eval_ms from "
                               "dia_time_eval as for the roofline"}
            if ref_pack is not None:
                ref, D_ref = ref_pack
                th_tc = out_tc["theta"].cpu().numpy()
                sumK = abs(ref[:-1].sum())
                tc_form.update({
                    "K_err_rel_sumK": float(np.max(np.abs(th_tc[:-1] - ref[:-1])) / sumK),
                    "B0_err_rel_sky": float(abs(th_tc[-1] - ref[-1]) / float(np.median(d["I"]))),
                    "D_err_rel_maxI": float(np.max(np.abs(out_tc["diff"].cpu().numpy() - D_ref)) /
                                            np.max(np.abs(d["I"])))})
        except Exception as exc:   # reported in the line; the figures above stand
            tc_form = {"error": f"{type(exc).__name__}: {exc}"[:300]}

    if rank == 0:
        last = infos[-1] if infos else {}
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(args, d),
            "kernel_tile": {**nat.kernel_variant_desc(m), "variant": tuned.get("variant")},
            "fits_per_s": fits_per_s,
            "vs_plain": value / plain["value"], "plain": plain, "batch_subset": batch_sub,
            "tc_form": tc_form,
            "evals_per_fit": evals_all / (args.steps * world),
            "adam_off": adam_off,
            "fit_info": {k: last.get(k) for k in ("status", "adam_iters", "lbfgs_iters", "evals",
                                                  "clip_passes_done", "reason", "ndata",
                                                  "precond_used")},
            "gpu_launches": launches * world,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "oracle_check": err,
            "dtype_note": "float32 pixel arithmetic; float64 cross-CTA sums and optimiser",
        }
        print(json.dumps(line), flush=True)


BATCH_WORKLOAD = "batch512_m7to21_chi2"


def _batch_costs(ds):
    return [shard.pair_cost(d["R"].shape[0], d["R"].shape[1], d["m"]) for d in ds]


def run_batch(args, rank, world, local_rank):
    """Batched fits of 512 stamp pairs (side ~ U{64..512}, odd m ~ U{7..21},
    fixed-variance chi^2): pair fits/s of the batched graph-captured form,
    and, on a same-pairs subset, batched vs one pair at a time (plain
    non-graph form, and graph form).  Under torchrun the 512 pairs are split
    across ranks by cost (strong scaling); each rank fits its share in one
    batched call, with no collective on the data path."""
    import torch
    from paper_2104_13715_gb300 import native as nat
    dist = None
    if world > 1:
        import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ds_all = synth.batch(args.batch_pairs, seed=args.seed)
    mine = shard.partition_by_cost(_batch_costs(ds_all), world)[rank]
    ds = [ds_all[k] for k in mine]
    items = [dict(R=torch.from_numpy(d["R"]).to(dev), I=torch.from_numpy(d["I"]).to(dev),
                  m=d["m"]) for d in ds]
    spec = nat.loss_spec(rho="gauss", noise="fixed", var=1.0)
    opts = nat.default_opts(timeout_s=900.0)
    stream = torch.cuda.current_stream(dev)
    # work-item size per kernel-side group: autotuned on these pairs, cached
    from paper_2104_13715_gb300 import autotune
    tuned = autotune.tune_batch(items, spec, stream=stream)
    ws = None
    for _ in range(args.warmup):
        out = nat.fit_batch(items, spec, opts, ws=ws, stream=stream)
        ws = out["ws"]
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local_rank) if local_rank == 0 else None
    if sampler:
        sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    evals = 0
    launches = 0
    flops = 0.0
    for _ in range(args.steps):
        out = nat.fit_batch(items, spec, opts, ws=ws, stream=stream)
        evals += sum(f["evals"] for f in out["infos"])
        launches += out["infos"][0]["kernel_launches"]   # per call, the same in every info
        flops += sum(4.0 * d["m"] ** 2 * f["ndata"] * f["evals"] for d, f in zip(ds, out["infos"]))
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    ms_own = e0.elapsed_time(e1)
    ok_own = sum(f["status"] == 0 for f in out["infos"])
    ms, pairs_all = shard.reduce_max_sum(ms_own, args.steps * len(items), device=dev)
    _, evals_all = shard.reduce_max_sum(0.0, evals, device=dev)
    _, ok = shard.reduce_max_sum(0.0, ok_own, device=dev)
    _, launches_all = shard.reduce_max_sum(0.0, launches, device=dev)
    _, flops_all = shard.reduce_max_sum(0.0, flops, device=dev)
    fits_s = pairs_all / (ms / 1e3)
    # the same batch without the Adam phase
    o_off = nat.default_opts(timeout_s=900.0, max_adam_iters=0)
    nat.fit_batch(items, spec, o_off, ws=ws, stream=stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    out_off = nat.fit_batch(items, spec, o_off, ws=ws, stream=stream)
    torch.cuda.synchronize(dev)
    adam_off = {"fits_per_s_rank0": len(items) / (time.perf_counter() - t0),
                "evals_per_pair": float(np.mean([f["evals"] for f in out_off["infos"]])),
                "converged": int(sum(f["status"] == 0 for f in out_off["infos"])),
                "what": "same pairs with max_adam_iters = 0 (the library default keeps the "
                        "paper's Adam phase)"}
    # the batched evaluation kernels alone: one more (untimed) batched call
    # whose first evaluation of every pair is timed per kernel-side group
    nat.set_batch_eval_timing(5)
    try:
        nat.fit_batch(items, spec, o_off, ws=ws, stream=stream)
        torch.cuda.synchronize(dev)
        bt = nat.batch_eval_timing()
    finally:
        nat.set_batch_eval_timing(0)
    # same-pairs subset: batched vs one at a time (single GPU only)
    t = None
    if world == 1:
        sub = items[:args.subset]
        t = {}
        for mode in ("batch", "single_plain", "single_graph"):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            if mode == "batch":
                nat.fit_batch(sub, spec, opts, stream=stream)
            else:
                o = nat.default_opts(use_graph=1 if mode == "single_graph" else 0, timeout_s=900.0)
                for it in sub:
                    nat.fit(it["R"], it["I"], it["m"], spec, o, want_diff=False, stream=stream)
            torch.cuda.synchronize(dev)
            t[mode] = len(sub) / (time.perf_counter() - t0)
        t = {"pairs": len(sub), **t, "batch_over_single_plain": t["batch"] / t["single_plain"]}
    npx = sum((d["R"].shape[0] - 2 * (d["m"] // 2)) * (d["R"].shape[1] - 2 * (d["m"] // 2))
              for d in ds_all)
    peaks, src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tf = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = flops_all / world / (ms / 1e3) / 1e12
    ms_k, fl_k = sum(bt["ms"]), sum(bt["flop"])
    ach_k = fl_k / (ms_k / 1e3) / 1e12 if ms_k > 0 else 0.0
    kernel_roof = {
        "achieved": ach_k, "frac": ach_k / peak_tf, "ms_per_evaluation_of_all_pairs": ms_k,
        "groups": [{"sides": sd, "ms": ms_g, "tflops": f / (ms_g / 1e3) / 1e12 if ms_g > 0 else 0.0,
                    "frac": (f / (ms_g / 1e3) / 1e12 / peak_tf) if ms_g > 0 else 0.0}
                   for sd, ms_g, f in zip(("1-7", "9-15", "17-23", "25-31"), bt["ms"], bt["flop"])
                   if f > 0],
        "timing": "dia_set_batch_eval_timing(5): each kernel-side group's evaluation kernel "
                  "alone over all its work items at the box-car start, mean of 5 launches "
                  "between CUDA events (rank 0's pairs)"}
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
            "frac": achieved / peak_tf, "traffic": None, "eval_kernels_alone": kernel_roof,
            "kernel": "dia::eval_batch_kernel (fused evaluations of all pairs, graph nodes)",
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz ({src} peaks file)",
            "algorithmic": "sum over pairs and evaluations of 4*m^2 flop x unmasked valid px",
            "note": "per GPU, lower bound: divided by the whole timed region (optimiser steps, "
                    "preconditioner builds and host polling included); the evaluation "
                    "kernels run inside CUDA graphs and are not timed alone"}
    line = {"metric": METRIC, "value": fits_s, "unit": "pair fits/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "pairs": len(ds_all), "valid_px": npx,
                       "sides": [int(min(d["R"].shape[0] for d in ds_all)),
                                 int(max(d["R"].shape[0] for d in ds_all))],
                       "m": sorted({d["m"] for d in ds_all}), "loss": "gauss",
                       "variance": "fixed",
                       "sharding": "pairs split across ranks by cost, no collective",
                       "work_item_variants": {str(g): r["variant"] for g, r in tuned.items()}},
            "evals_per_s": evals_all / (ms / 1e3), "pairs_converged": int(ok),
            "gpu_launches": int(launches_all), "roofline": roof,
            "subset_fits_per_s": t, "adam_off": adam_off, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference_batch(args, rank, world):
    """The FP64 oracle on the batch workload: pairs fitted one after another
    by the normal-equation solve (the chi^2 optimum), a bounded sample per step."""
    if rank != 0:
        return
    import oracle
    ds = synth.batch(args.batch_pairs, seed=args.seed)
    rates, k, sample_pairs = [], 0, 0
    budget = max(args.ref_budget / max(args.steps + args.warmup, 1), 1.0)
    for i in range(args.warmup + args.steps):
        n, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < budget or n == 0:
            d = ds[k % len(ds)]
            oracle.normal_solve(d["R"], d["I"], d["m"])
            k += 1
            n += 1
        if i >= args.warmup:
            rates.append(n / (time.perf_counter() - t0))
            sample_pairs += n
    value = float(np.mean(rates))
    cores = os.cpu_count() or 1
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pair fits/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "pairs": len(ds)},
        "cpu_baseline": {"value": value, "unit": "pair fits/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample_pairs} pairs of the batch (in order) fitted by the "
                                   f"oracle's FP64 normal-equation solve, ~{budget:.0f} s per step"},
        "e2e": {"value": value, "unit": "pair fits/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_precision_study(args):
    """Precision study: the FP32 fused path with float64 cross-block
    accumulation against the pure-float32 accumulation form and the
    tensor-core evaluation form (split bf16 forward, split fp16 weight
    gradient, float64 across tiles), on the 2048^2
    high-dynamic-range field (m = 21, CCD negative log-likelihood).  For each
    form: fit, then K, B0 and difference-image errors against the FP64
    oracle's Newton optimum (polished from the float64 form's theta), and the
    gradient error at a fixed non-stationary theta."""
    import torch
    import oracle
    from paper_2104_13715_gb300 import native as nat
    name = "hdr2048_m21_nll"
    d = synth.workload(name, seed=args.seed, size=args.size)
    m = d["m"]
    dev = torch.device("cuda", 0)
    up = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    R, I = up(d["R"]), up(d["I"])
    spec = nat.loss_spec(**_loss_kw(d))
    ospec = _oracle_spec(d)
    th_start = np.full(m * m + 1, 1.0 / (m * m))
    th_start[-1] = float(np.median(d["I"]))
    rng = np.random.default_rng(1)
    th_start[:-1] *= 1.0 + 0.3 * rng.uniform(-1, 1, m * m)
    _, g_or = oracle.loss_grad(d["R"], d["I"], m, th_start, ospec)
    forms = {}
    for mode, form, label in ((nat.ACCUM_FP64, nat.EVAL_FP32, "fp32_pixels_fp64_accumulation"),
                              (nat.ACCUM_FP32, nat.EVAL_FP32, "pure_fp32_accumulation"),
                              (nat.ACCUM_FP64, nat.EVAL_TC, "tensor_core_split_precision")):
        nat.set_accumulation(mode)
        nat.set_eval_form(form)
        try:
            _, g = nat.loss_grad(R, I, m, torch.from_numpy(th_start), spec)
            out = nat.fit(R, I, m, spec, nat.default_opts())
        finally:
            nat.set_accumulation(nat.ACCUM_FP64)
            nat.set_eval_form(nat.EVAL_FP32)
        forms[label] = {"theta": out["theta"].cpu().numpy(), "diff": out["diff"].cpu().numpy(),
                        "info": out["info"],
                        "grad_err": float(np.max(np.abs(g.cpu().numpy() - g_or)) /
                                          np.max(np.abs(g_or)))}
    t0 = time.perf_counter()
    ref = oracle.newton(d["R"], d["I"], m, forms["fp32_pixels_fp64_accumulation"]["theta"], ospec)
    t_or = time.perf_counter() - t0
    D_ref = oracle.diff_image(d["R"], d["I"], m, ref)
    sky = float(np.median(d["I"]))
    res = {}
    for label, f in forms.items():
        th = f["theta"]
        res[label] = {
            "K_err_rel_sumK": float(np.max(np.abs(th[:-1] - ref[:-1])) / abs(ref[:-1].sum())),
            "B0_err_rel_sky": float(abs(th[-1] - ref[-1]) / sky),
            "diff_err_rel_maxI": float(np.max(np.abs(f["diff"] - D_ref)) / np.max(np.abs(d["I"]))),
            "grad_err_rel_at_start": f["grad_err"],
            "evals": f["info"]["evals"], "reason": f["info"]["reason"]}
    print(json.dumps({"precision_study": name, "H": d["R"].shape[0], "W": d["R"].shape[1],
                      "m": m, "loss": "gauss", "variance": "ccd", "results": res,
                      "oracle": f"FP64 Newton polish from the float64-accumulation fit, "
                                f"{t_or:.1f} s on {os.cpu_count()} host cores",
                      "tolerances": {"K": 1e-4, "B0": 1e-4, "grad": 1e-5}}), flush=True)


def run_s10_study(args):
    """The simulated-image accuracy study (Sec. 3.2-3.3) at N = args.s10_study
    simulations: pairs drawn by the paper's recipe, fitted in one batched call
    with the CCD negative log-likelihood and a 19x19 kernel, binned by SNR and
    sampling regime; per bin the medians and 16/84 % points of P, MSE, MFB and
    MFV beside the paper's PyTorchDIA values (and its B08 MFB)."""
    import torch
    from paper_2104_13715_gb300 import native as nat
    table = json.load(open(os.path.join(ROOT, "tests", "golden", "s10_table.json")))
    t0 = time.perf_counter()
    ds = [d for d in (synth.s10_pair(s) for s in range(args.s10_study)) if d["snr_regime"] > 0]
    t_gen = time.perf_counter() - t0
    dev = torch.device("cuda", 0)
    items = [dict(R=torch.from_numpy(d["R"]).to(dev), I=torch.from_numpy(d["I"]).to(dev),
                  m=d["m"]) for d in ds]
    spec = nat.loss_spec(rho="gauss", noise="ccd", sigma0=synth.S10_SIGMA0, gain=1.0,
                         var_floor=1e-6)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = nat.fit_batch(items, spec, nat.default_opts(), want_diff=True)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    bins = {}
    bad = 0
    for d, th, D, info in zip(ds, out["thetas"], out["diffs"], out["infos"]):
        if info["status"] != 0:
            bad += 1
            continue
        met = synth.s10_metrics(d, th.cpu().numpy(), D.cpu().numpy())
        bins.setdefault((d["snr_regime"], d["sampling"]), []).append(met)
    res = []
    for (snr, samp), mets in sorted(bins.items()):
        row = {"snr_regime": snr, "sampling": table["sampling_regimes"][samp], "n": len(mets)}
        for k, ok in (("P", "P"), ("MSE", "MSE_noisy"), ("MFB", "MFB"), ("MFV", "MFV")):
            v = np.array([x[ok] for x in mets])
            med, lo, hi = table[k][str(snr)][samp]
            row[k] = {"median": float(np.median(v)), "p16": float(np.percentile(v, 16)),
                      "p84": float(np.percentile(v, 84)), "paper_median": med,
                      "paper_p16": med - lo, "paper_p84": med + hi,
                      "z": float((np.median(v) - med) / (1.2533 * 0.5 * (lo + hi) / np.sqrt(len(v))))}
        row["MFB"]["paper_b08_median"] = table["MFB_B08"][str(snr)][samp][0]
        row["MSE"]["what"] = "ours: mean (I - M)^2 against the noisy target"
        row["MSE_vs_noiseless"] = float(np.median([x["MSE"] for x in mets]))
        res.append(row)
    print(json.dumps({"s10_study": {"n_drawn": args.s10_study, "n_in_regimes": len(ds),
                                    "fit_failures": bad, "bins": res,
                                    "fit": {"pairs": len(ds), "seconds": t_fit,
                                            "fits_per_s": len(ds) / t_fit},
                                    "generation_seconds": t_gen,
                                    "loss": "gauss NLL, CCD variance sigma0 = 5, G = 1",
                                    "z": "(median - paper median) / standard error of a median"}}),
          flush=True)


def run_tc_forward(args):
    """The forward pass alone, two ways: the difference image D = I - M of the
    workload at the box-car kernel through dia_diff_image (float32 CUDA cores)
    and dia_diff_image_tc (tcgen05 tensor cores, split bf16), W + K calls each,
    CUDA events around the K calls (each call includes its small prep kernel;
    the tensor-core call also reads back its status word)."""
    import torch
    from paper_2104_13715_gb300 import native as nat
    d = synth.workload(args.workload, seed=args.seed, size=args.size)
    m = d["m"]
    dev = torch.device("cuda", 0)
    R = torch.from_numpy(d["R"]).to(dev)
    I = torch.from_numpy(d["I"]).to(dev)
    th = torch.full((m * m + 1,), 1.0 / (m * m), dtype=torch.float64)
    th[-1] = float(np.median(d["I"]))
    ws = nat.workspace(R.shape[0], R.shape[1], m, device=dev)
    H, W = R.shape
    h = m // 2
    npx = (H - 2 * h) * (W - 2 * h)
    res = {}
    outs = {}
    for name, fn in (("fp32_cuda_cores", nat.diff_image), ("tensor_cores_split_bf16", nat.diff_image_tc)):
        for _ in range(args.warmup):
            outs[name] = fn(R, I, m, th, ws=ws)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            outs[name] = fn(R, I, m, th, ws=ws)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / max(args.steps, 1)
        res[name] = {"ms": ms, "tflops_useful": 2.0 * m * m * npx / ms / 1e9}
    diff = (outs["tensor_cores_split_bf16"] - outs["fp32_cuda_cores"]).abs().max().item()
    print(json.dumps({"tc_forward": args.workload, "H": H, "W": W, "m": m, "results": res,
                      "max_abs_diff_rel_maxI": diff / I.abs().max().item(),
                      "useful": "2 m^2 flop per valid pixel"}), flush=True)


def run_tc_eval(args):
    """One loss+gradient evaluation of the workload at the box-car start in
    two forms: dia_loss_grad (the fused float32 kernel) and dia_loss_grad_tc
    (both contractions on the tensor cores), W + K calls each, CUDA events
    around the K calls (each call includes its small launches; the
    tensor-core call also reads back its status word); gradient error of each
    against the other."""
    import torch
    from paper_2104_13715_gb300 import native as nat
    d = synth.workload(args.workload, seed=args.seed, size=args.size)
    m = d["m"]
    dev = torch.device("cuda", 0)

    def up(a, dt):
        return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)

    R, I = up(d["R"], torch.float32), up(d["I"], torch.float32)
    mask, var = up(d.get("mask"), torch.uint8), up(d.get("var"), torch.float32)
    spec = nat.loss_spec(**_loss_kw(d))
    th = torch.full((m * m + 1,), 1.0 / (m * m), dtype=torch.float64)
    th[-1] = float(np.median(d["I"]))
    res, grads = {}, {}
    for name, fn in (("fp32_fused", nat.loss_grad), ("tensor_cores", nat.loss_grad_tc)):
        for _ in range(args.warmup):
            L, g = fn(R, I, m, th, spec, mask=mask, var=var)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            L, g = fn(R, I, m, th, spec, mask=mask, var=var)
        e1.record()
        torch.cuda.synchronize(dev)
        grads[name] = g.cpu().numpy()
        res[name] = {"ms": e0.elapsed_time(e1) / max(args.steps, 1)}
    diff = float(np.max(np.abs(grads["tensor_cores"] - grads["fp32_fused"])) /
                 np.max(np.abs(grads["fp32_fused"])))
    print(json.dumps({"tc_eval": args.workload, "H": d["R"].shape[0], "W": d["R"].shape[1], "m": m,
                      "results": res, "grad_diff_rel": diff}), flush=True)


def run_tc_sweep(args):
    """Kernel sizes m = 7 .. 31 on a 4096^2 field (the Cauchy-loss workload's
    recipe with its mask and variance map, the kernel side varied): one
    loss+gradient evaluation in the fused float32 form and in the tensor-core
    form (dia_set_eval_form), each launch set timed alone with dia_time_eval
    after reading 2 x L2 through the cache, and the gradients' difference."""
    import torch
    from paper_2104_13715_gb300 import native as nat
    dev = torch.device("cuda", 0)
    base = synth.WORKLOADS["ccd4096_m25_cauchy_clip3"]
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    rows = []
    for m in (7, 11, 15, 19, 25, 31):
        spec_m = synth.PairSpec(**{**base.__dict__, "m": m})
        d = synth.make_pair(spec_m, args.seed)

        def up(a, dt):
            return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)

        R, I = up(d["R"], torch.float32), up(d["I"], torch.float32)
        mask, var = up(d.get("mask"), torch.uint8), up(d.get("var"), torch.float32)
        spec = nat.loss_spec(**_loss_kw(d))
        th = torch.full((m * m + 1,), 1.0 / (m * m), dtype=torch.float64, device=dev)
        th[-1] = float(np.median(d["I"]))
        res = {"m": m}
        grads = {}
        for form, name in ((nat.EVAL_FP32, "fp32"), (nat.EVAL_TC, "tc")):
            nat.set_eval_form(form)
            try:
                ws = nat.workspace(*d["R"].shape, m, device=dev)
                nat.time_eval(R, I, m, th, spec, mask=mask, var=var, reps=2, flush=flush, ws=ws)
                res[name + "_ms"] = nat.time_eval(R, I, m, th, spec, mask=mask, var=var,
                                                  reps=args.steps, flush=flush, ws=ws)
                grads[name] = nat.loss_grad(R, I, m, th, spec, mask=mask, var=var, ws=ws)[1].cpu().numpy()
                del ws
            finally:
                nat.set_eval_form(nat.EVAL_FP32)
        res["tc_speedup"] = res["fp32_ms"] / res["tc_ms"]
        res["grad_diff_rel"] = float(np.max(np.abs(grads["tc"] - grads["fp32"])) /
                                     np.max(np.abs(grads["fp32"])))
        rows.append(res)
        print(json.dumps(res), flush=True)
    print(json.dumps({"tc_sweep": "4096^2 Cauchy, mask, variance map", "rows": rows}), flush=True)


def run_kernel_only(args):
    """The fused loss+gradient kernel of the workload at the box-car start:
    its launches alone (dia_time_eval: CUDA events around each launch on the
    stream, L2 overwritten before each), and whole dia_loss_grad calls
    (preparation, kernel, reduction) back to back; the driver of the ncu
    captures of the fused kernel.  Reports algorithmic GB/s and TFLOP/s and
    their fractions of the measured HBM copy and of the FP32 pipe."""
    import torch
    from paper_2104_13715_gb300 import native as nat
    d = synth.workload(args.workload, seed=args.seed, size=args.size)
    m = d["m"]
    H, W = d["R"].shape
    dev = torch.device("cuda", 0)

    def up(a, dt):
        return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)

    R, I = up(d["R"], torch.float32), up(d["I"], torch.float32)
    mask, var = up(d.get("mask"), torch.uint8), up(d.get("var"), torch.float32)
    spec = nat.loss_spec(**_loss_kw(d))
    if args.variant is not None:
        nat.select_kernel_variant(m, args.variant)
    if args.tiled:
        nat.set_small_kernel(False)
    ws = nat.workspace(H, W, m, device=dev)
    th = torch.full((m * m + 1,), 1.0 / (m * m), dtype=torch.float64, device=dev)
    th[-1] = float(np.median(d["I"]))
    s = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    nat.time_eval(R, I, m, th, spec, mask=mask, var=var, reps=args.warmup, flush=flush, ws=ws,
                  stream=s)
    ms_k = nat.time_eval(R, I, m, th, spec, mask=mask, var=var, reps=args.steps, flush=flush,
                         ws=ws, stream=s)
    # the same launches back to back between one pair of events (inputs larger
    # than L2 stand in for the flush; no launch gaps in the figure)
    ms_b2b = nat.time_eval(R, I, m, th, spec, mask=mask, var=var, reps=args.steps, flush=None,
                           ws=ws, stream=s)
    for _ in range(args.warmup):
        nat.loss_grad(R, I, m, th, spec, mask=mask, var=var, ws=ws, stream=s)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        nat.loss_grad(R, I, m, th, spec, mask=mask, var=var, ws=ws, stream=s)
    e1.record(s)
    torch.cuda.synchronize(dev)
    ms_call = e0.elapsed_time(e1) / max(args.steps, 1)
    h = m // 2
    npx = int(d["mask"][h:H - h, h:W - h].sum()) if d.get("mask") is not None else (H - 2 * h) * (W - 2 * h)
    # bytes every evaluation must read: R and I, and the mask / variance map if
    # given (4 + 4 + 1 + 4 per pixel of the image)
    nbytes = H * W * (8 + (1 if d.get("mask") is not None else 0) + (4 if d.get("var") is not None else 0))
    flops = 4.0 * m * m * npx
    peaks, src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tf = sms * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    gbs = nbytes / ms_k / 1e6
    tfl = flops / ms_k / 1e9
    print(json.dumps({"kernel_only": args.workload, "H": H, "W": W, "m": m,
                      "form": "tiled" if (args.tiled or m > 5) else "streaming small-kernel",
                      "variant": nat.kernel_variant_desc(m), "ms_per_launch": ms_k,
                      "ms_per_call": ms_call,
                      "gbs_algorithmic": gbs, "hbm_frac": gbs / float(peaks["hbm_gbs"]),
                      "tflops_algorithmic": tfl, "fp32_frac": tfl / peak_tf,
                      "back_to_back": {"ms_per_launch": ms_b2b,
                                       "hbm_frac": nbytes / ms_b2b / 1e6 / float(peaks["hbm_gbs"]),
                                       "fp32_frac": flops / ms_b2b / 1e9 / peak_tf,
                                       "inputs_vs_l2": f"{nbytes / 2**20:.0f} MiB of inputs, "
                                                       f"{L2_BYTES / 2**20:.0f} MiB L2",
                                       "valid": nbytes > L2_BYTES},
                      "bytes_algorithmic": nbytes, "flops_algorithmic": flops,
                      "peaks": f"{peaks['hbm_gbs']} GB/s HBM copy, {peak_tf:.1f} TFLOP/s FP32 "
                               f"({src})"}), flush=True)


def run_m_sweep(args):
    """The kernel-size sweep of the paper's speed tests (Sec. 5.3, a 1000^2
    crop fitted with kernels of increasing size): a 1000^2 field (--size for
    another side; lg rho = 1.5 per 100^2 px, phi_R = 1, phi_K = 1.5, sky 100,
    the Sec. 5.2 recipe) fitted
    with the fixed-variance chi^2 for every odd m in 3..31.  Per m: the fused
    evaluation kernel alone (dia_time_eval, L2 flushed before each launch) in
    algorithmic TFLOP/s and GB/s against the FP32 pipe and the measured HBM
    copy, and one full fit (dia_fit, Adam then L-BFGS) in ms with its
    evaluation count."""
    import torch
    from paper_2104_13715_gb300 import native as nat
    dev = torch.device("cuda", 0)
    peaks, src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tf = sms * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    rows = []
    S = args.size or 1000   # the paper's 1000^2 crop; --size for a larger field
    for m in range(3, 32, 2):
        spec_p = synth.PairSpec(size=(S, S), n_stars=int(round(10 ** 1.5 * S * S / 1e4)), m=m,
                                fwhm_ref=2.0 * math.sqrt(2 * math.log(2.0)), kernel_sigma=1.5,
                                sky=100.0, flux_law="paper", read=5.0, gain=1.0)
        d = synth.make_pair(spec_p, args.seed + m)
        R = torch.from_numpy(d["R"]).to(dev)
        I = torch.from_numpy(d["I"]).to(dev)
        spec = nat.loss_spec(rho="gauss", noise="fixed", var=1.0)
        th = torch.full((m * m + 1,), 1.0 / (m * m), dtype=torch.float64, device=dev)
        th[-1] = float(np.median(d["I"]))
        ws = nat.workspace(S, S, m, device=dev)
        nat.time_eval(R, I, m, th, spec, reps=3, flush=flush, ws=ws)
        ms = nat.time_eval(R, I, m, th, spec, reps=args.steps, flush=flush, ws=ws)
        h = m // 2
        npx = (S - 2 * h) ** 2
        tfl = 4.0 * m * m * npx / ms / 1e9
        gbs = S * S * 8 / ms / 1e6
        nat.fit(R, I, m, spec, want_diff=False)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = nat.fit(R, I, m, spec, want_diff=False)
        torch.cuda.synchronize(dev)
        fit_ms = (time.perf_counter() - t0) * 1e3
        rows.append({"m": m, "eval_ms": ms, "tflops": tfl, "fp32_frac": tfl / peak_tf,
                     "gbs": gbs, "hbm_frac": gbs / float(peaks["hbm_gbs"]),
                     "form": "streaming small-kernel" if m <= 5 else "tiled",
                     "fit_ms": fit_ms, "fit_evals": out["info"]["evals"],
                     "fit_status": out["info"]["status"]})
    print(json.dumps({"m_sweep": f"{S}x{S} chi^2, Sec. 5.3 recipe", "rows": rows,
                      "peaks": f"{peaks['hbm_gbs']} GB/s HBM copy, {peak_tf:.1f} TFLOP/s FP32 "
                               f"({src})"}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(synth.WORKLOADS) + [BATCH_WORKLOAD])
    ap.add_argument("--batch-pairs", type=int, default=512)
    ap.add_argument("--subset", type=int, default=32, help="same-pairs subset (batch workload)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--kernel-evals", type=int, default=20)
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--no-batch-subset", action="store_true")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time the fused loss+gradient kernel alone (ncu driver)")
    ap.add_argument("--size", type=int, default=None, help="image side override (--kernel-only, --m-sweep)")
    ap.add_argument("--variant", type=int, default=None, help="tile variant (--kernel-only)")
    ap.add_argument("--tiled", action="store_true",
                    help="the tiled kernel even where the streaming small-kernel form applies "
                         "(--kernel-only)")
    ap.add_argument("--tc-forward", action="store_true",
                    help="time the forward pass on CUDA cores and on tensor cores")
    ap.add_argument("--no-tc-form", action="store_true",
                    help="skip the tensor-core evaluation form's fits in the default run")
    ap.add_argument("--tc-sweep", action="store_true",
                    help="float32 vs tensor-core evaluation over kernel sides 7..31 at 4096^2")
    ap.add_argument("--tc-eval", action="store_true",
                    help="time the loss+gradient evaluation on CUDA cores and on tensor cores")
    ap.add_argument("--s10-study", type=int, default=0,
                    help="run the simulated-image accuracy study with this many simulations")
    ap.add_argument("--precision-study", action="store_true",
                    help="float64 vs float32 accumulation on the 2048^2 HDR field")
    ap.add_argument("--m-sweep", action="store_true",
                    help="kernel-size sweep m = 3..31 on a 1000^2 field (Sec. 5.3)")
    args = ap.parse_args()
    if args.m_sweep:
        run_m_sweep(args)
        return
    if args.s10_study:
        run_s10_study(args)
        return
    if args.tc_forward:
        run_tc_forward(args)
        return
    if args.tc_eval:
        run_tc_eval(args)
        return
    if args.tc_sweep:
        run_tc_sweep(args)
        return
    if args.precision_study:
        run_precision_study(args)
        return
    if args.kernel_only:
        run_kernel_only(args)
        return
    rank, world, local_rank = shard.rank_env()
    if args.impl == "reference":
        if args.workload == BATCH_WORKLOAD:
            run_reference_batch(args, rank, world)
        else:
            run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        if args.workload == BATCH_WORKLOAD:
            run_batch(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()

if __name__ == "__main__":
    main()
