"""Throughput benchmark of the EP sweep (Mpixel-EP-sweeps/s).

Workloads (synthetic, seeded; the paper's images are not available):
  deconv512     512x512, rectangles + discs + Gaussian random field (length 32 px),
                9x9 uniform periodic blur, BSNR 40 dB, beta by EM every 5 sweeps
                from 1, 32 RBMC probes, FP32 sweeps.                      (default)
  denoise4096   4096x4096, 40 rectangles, sigma 0.1, beta 20, damping 0.5.
  batched256    256 problems of uneven sizes, noise levels and blur widths.
  cs128, cs128h compressive sensing 128x128, M = 4915 Gaussian rows or Hadamard
                patterns, sigma 0.01, EM every 5 sweeps.
  warmstart512, warmstart4096
                sweeps and seconds to the converged cold-start posterior, cold
                start against the learned warm start and a non-learned control.
A step is one EP sweep: the four prior-site updates, the likelihood-site update
and, where configured, the EM update of beta.  Inputs are resident on the GPU
when the timed region starts; L2 is flushed (256 MB write) before every timed
step and the flush is not timed.  The default run also benches denoise4096 and
cs128 for a few steps, each in a fresh process, and reports them under
"secondary".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload NAME] [--no-cpu-baseline] [--no-secondary]

With --gpus N > 1 (one process per GPU, launched by torch.distributed.run) every
rank solves its own independent problem ("replicas", weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "deconv512": dict(kind="deconv", h=512, w=512, kernel=("uniform", 9), bsnr_db=40.0, beta0=1.0,
                      em_every=5, S=32, seed=0),
    "denoise4096": dict(kind="denoise", h=4096, w=4096, sigma=0.1, beta0=20.0, em_every=0,
                        seed=0, n_rect=40),
    "batched256": dict(kind="batch", n=256, h=None, w=None, em_every=5, beta0=1.0, S=32, seed=0),
    "cs128": dict(kind="cs", h=128, w=128, ratio=0.3, sigma=0.01, beta0=1.0, em_every=5, seed=0),
    # the same size with M uniformly drawn 2-D Hadamard patterns in place of the Gaussian rows
    "cs128h": dict(kind="cs", op="hadamard", h=128, w=128, ratio=0.3, sigma=0.01, beta0=1.0,
                   em_every=5, seed=0),
    # learned warm start: seconds and sweeps to the posterior of converged plain EP
    "warmstart512": dict(kind="warmstart", h=512, w=512, seed=900003, em_every=0),
    # config 5 at its stated size (15 x 15 Gaussian blur, std 2 px, BSNR 30 dB)
    "warmstart4096": dict(kind="warmstart", h=4096, w=4096, seed=900004, em_every=0, ref_sweeps=120,
                          max_sweeps=120),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _bf16_sustained():
    """Dense BF16 tensor peak for a kernel timed inside a long step (TFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "measured (sustained)"
    except Exception:
        return 1700.0, "fallback (sustained)"


# ---- multi-rank host logic (one process per GPU, independent replicas)

def replica_seed(base: int, rank: int) -> int:
    """Seed of rank's own problem: every replica solves a different instance."""
    return base + 1000 * rank


def barrier(world: int):
    if world > 1:
        import torch
        torch.distributed.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The job's time: the largest of the ranks' times."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(pixels_per_rank: int, world: int, steps: int, ms_total: float) -> float:
    """Whole-job Mpixel-EP-sweeps/s: all ranks' pixel-sweeps over the job's time."""
    return pixels_per_rank * world * steps / (ms_total / 1e3) / 1e6


def _problem(cfg, rank=0):
    from paper_2110_01585_gb300 import synthetic as syn
    seed = replica_seed(cfg["seed"], rank)
    if cfg["kind"] == "deconv":
        k = syn.uniform_kernel(cfg["kernel"][1])
        return syn.deconv_problem(cfg["h"], cfg["w"], kernel=k, bsnr_db=cfg["bsnr_db"],
                                  beta0=cfg["beta0"], seed=seed)
    if cfg["kind"] == "cs" and cfg.get("op") == "hadamard":
        return syn.hadamard_cs_problem(cfg["h"], cfg["w"], ratio=cfg["ratio"], sigma=cfg["sigma"],
                                       beta0=cfg["beta0"], seed=seed)
    if cfg["kind"] == "cs":
        return syn.cs_problem(cfg["h"], cfg["w"], ratio=cfg["ratio"], sigma=cfg["sigma"],
                              beta0=cfg["beta0"], seed=seed)
    return syn.denoise_problem(cfg["h"], cfg["w"], sigma=cfg["sigma"], beta=cfg["beta0"],
                               seed=seed, n_rect=cfg.get("n_rect", 8))


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                parts = [x.strip() for x in out.split(",")]
                if len(parts) == 6:
                    self.samples.append(parts)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = sorted(float(s[0]) for s in self.samples)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[2 + i].strip().lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(self.samples[0][1]),
                "reasons": reasons, "samples": len(sm)}


def _kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2110_01585_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        path = os.path.join(csrc, f)
        if not os.path.isfile(path) or f.endswith(".pyc"):
            continue  # e.g. a __pycache__ left by running the generator script
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel_name):
    """DRAM bytes per unit from the committed ncu summary, if taken on this source."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
        e = d.get(kernel_name)
        if e and e.get("source_hash") == _kernel_source_hash():
            return e["dram_bytes_per_unit"]
    except Exception:
        pass
    return None


# The conjugate-gradient iteration of the deconvolution likelihood site moves at
# least 32 bytes per pixel per right-hand side: read p, x, r and Q p, write x, r
# and p (FP32 planes; the method's work, whatever the implementation stores).
CG_BYTES_PER_PIXEL_RHS = 32.0


def cg_iteration_roofline(trace, peak, peak_src):
    """Whole-iteration roofline of the CG: 32 B per active system-pixel of each
    iteration over the device time of the direction, update and preconditioner
    kernels.  Active system-pixels are the update kernel's units."""
    need = ("cg_direction", "cg_update", "cg_precond")
    if not all(k in trace and trace[k][1] for k in need):
        return None
    ms = sum(trace[k][0] for k in need)
    units = trace["cg_update"][2]
    achieved = units * CG_BYTES_PER_PIXEL_RHS / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    return {"bytes_per_pixel_rhs": CG_BYTES_PER_PIXEL_RHS, "system_pixel_iterations": units,
            "ms": round(ms, 3), "achieved": round(achieved, 1), "peak": peak,
            "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / peak, 4)}


def run_batch(args, rank, world):
    """256 uneven problems (denoising and deconvolution) advanced by ep_tv_batch_sweep."""
    import numpy as np
    import torch

    from paper_2110_01585_gb300 import EPTV, OP_CONV_PERIODIC, Batch
    from paper_2110_01585_gb300 import synthetic as syn

    cfg = WORKLOADS[args.workload]
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    n_prob = args.batch_n or cfg["n"]
    probs = syn.batched_problems(n_prob, seed=replica_seed(cfg["seed"], rank))
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    ctxs = []
    with torch.cuda.stream(stream):
        for p in probs:
            yt = torch.as_tensor(p.y.astype(np.float32), device=dev)
            if p.kind == "denoise":
                ctxs.append(EPTV(yt, p.xi, p.beta, stream=stream))
            else:
                ctxs.append(EPTV(yt, p.xi, p.beta, op=OP_CONV_PERIODIC, kernel=p.kernel,
                                 rbmc_samples=cfg["S"], cg_max_iter=100000, stream=stream))
    n_px = sum(p.n_pixels for p in probs)
    batch = Batch(ctxs)
    idx = [0]

    def step():
        idx[0] += 1
        batch.sweep(1, em_every=1 if idx[0] % cfg["em_every"] == 0 else 0)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)

    def timed(steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize()
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[i][0].record(stream)
            step()
            with torch.cuda.stream(stream):
                ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev)

    # timed untraced (deconvolution sites as graph replays); per-kernel times from
    # a traced repeat of the same number of steps
    cs = ClockSampler(dev.index)
    with cs:
        ms_local = timed(args.steps)
    barrier(world)
    for c in ctxs:
        c.trace(True)
    timed(args.steps)
    # pixels per rank differ between replicas: the job rate sums the ranks' work
    ms_total = max_over_ranks(ms_local, world, dev)
    n_px_job = n_px
    if world > 1:
        t = torch.tensor([float(n_px)], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t)
        n_px_job = int(t.item())
    trace = {}
    for c in ctxs:
        for k, v in c.trace_read().items():
            t = trace.setdefault(k, [0.0, 0, 0.0, v[3]])
            t[0] += v[0]
            t[1] += v[1]
            t[2] += v[2]
            t[3] = v[3] or t[3]
    status = max(c.status() for c in ctxs)
    batch.close()
    for c in ctxs:
        c.close()
    value = job_throughput(n_px_job, 1, args.steps, ms_total)
    # kernel classes overlap across worker streams: shares are of summed kernel time
    tot_k = sum(v[0] for v in trace.values()) or 1.0
    name, (kms, kl, units, bpu) = max(trace.items(), key=lambda kv: kv[1][0])
    peak, peak_src = _peaks()
    achieved = units * bpu / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": None, "note": "per-launch event times summed over concurrent streams",
                "share_of_kernel_time": round(kms / tot_k, 4)}
    return dict(value=value, ms_per_step=ms_total / args.steps, roofline=roofline,
                clocks=cs.summary(), launches=sum(v[1] for v in trace.values()),
                trace={k: tuple(v) for k, v in trace.items()},
                stats={"cg_iters": None, "n_fp64": None}, status=status, e2e=None, n_px=n_px)


def run_warmstart(args, rank, world):
    """Cold start against the packaged warm-start network on one held-out
    problem of the warm-start workload: sweeps and device seconds until the
    posterior is within the parity tolerances of converged cold-start EP."""
    import torch

    import paper_2110_01585_gb300 as pkg
    from paper_2110_01585_gb300 import synthetic as syn
    from paper_2110_01585_gb300.train_warmstart import control_constants, sweeps_to_match
    from paper_2110_01585_gb300.warmstart import WarmStartNet

    cfg = WORKLOADS[args.workload]
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    net, meta = WarmStartNet.load(os.path.join(os.path.dirname(pkg.__file__), "data",
                                               "warmstart_gauss15_128.npz"))
    beta, probes = float(meta["beta"]), int(meta["probes"])
    p = syn.warmstart_problem(cfg["h"], cfg["w"], seed=cfg["seed"] + rank, beta=beta)
    # the non-learned control: constant site log-precisions (medians of the
    # training targets of 8 labelled problems), posterior mean y
    consts = control_constants(beta, probes)
    ref_sweeps, max_sweeps = cfg.get("ref_sweeps", 250), cfg.get("max_sweeps", 150)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as sampler:
        r = sweeps_to_match(p, beta, probes, net=net, control=consts, ref_sweeps=ref_sweeps,
                            max_sweeps=max_sweeps)
    clocks = sampler.summary()
    n_px = cfg["h"] * cfg["w"]
    cold, warm, ctrl = r["cold"], r["warm"], r["control"]
    ok = cold["sweeps"] is not None and warm["sweeps"] is not None
    value = n_px * warm["sweeps"] / warm["seconds"] / 1e6 if ok else 0.0
    return {"value": value, "ms_per_step": (warm["seconds"] / warm["sweeps"] * 1e3) if ok else 0.0,
            "n_px": n_px, "clocks": clocks, "launches": None, "roofline": None, "e2e": None,
            "stats": {"cg_iters": None, "n_fp64": None}, "status": 0, "trace": {},
            "to_posterior": {"tolerance": f"1e-4 means, 1e-3 variances vs {ref_sweeps} cold sweeps",
                             "cold_sweeps": cold["sweeps"], "warm_sweeps": warm["sweeps"],
                             "control_sweeps": ctrl["sweeps"],
                             "cold_s": cold["seconds"], "warm_s": warm["seconds"],
                             "control_s": ctrl["seconds"],
                             "speedup_time": (cold["seconds"] / warm["seconds"]) if ok else None,
                             "speedup_over_control": (ctrl["seconds"] / warm["seconds"])
                             if (ok and ctrl["seconds"]) else None,
                             "control": "mean y, constant site log-precisions (medians of the "
                                        "training targets)",
                             "network": "6 x conv3x3, 32 channels, FP32, trained on 256 x 128^2",
                             "beta": beta, "rbmc_probes": probes}}


def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_2110_01585_gb300 import (EPTV, OP_CONV_PERIODIC, OP_DENSE, OP_HADAMARD, OP_IDENTITY,
                                        solve_host)

    cfg = WORKLOADS[args.workload]
    if cfg["kind"] == "batch":
        return run_batch(args, rank, world)
    if cfg["kind"] == "warmstart":
        return run_warmstart(args, rank, world)
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    prob = _problem(cfg, rank)
    n_px = prob.n_pixels
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    kw = {}
    if cfg["kind"] == "deconv":
        kw = dict(op=OP_CONV_PERIODIC, kernel=prob.kernel, rbmc_samples=cfg["S"])
    with torch.cuda.stream(stream):
        if cfg["kind"] == "cs" and cfg.get("op") == "hadamard":
            kw = dict(op=OP_HADAMARD, patterns=prob.patterns, height=cfg["h"], width=cfg["w"])
        elif cfg["kind"] == "cs":
            At = torch.as_tensor(prob.A.astype(np.float32), device=dev)
            kw = dict(op=OP_DENSE, dense=At, height=cfg["h"], width=cfg["w"])
        yt = torch.as_tensor(prob.y.astype(np.float32), device=dev)
        ep = EPTV(yt, prob.xi, prob.beta, stream=stream, **kw)
    em_every = cfg["em_every"]
    sweep_idx = [0]

    def step():
        ep.sweep(1)
        sweep_idx[0] += 1
        if em_every and sweep_idx[0] % em_every == 0:
            ep.em_beta(sync=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)

    def timed(steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize()
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[i][0].record(stream)
            step()
            with torch.cuda.stream(stream):
                ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev)

    # the measured steps run as the library runs them untraced (deconvolution:
    # one graph per likelihood-site update); the per-kernel times of the
    # roofline come from the same number of steps run again with every launch
    # bracketed by CUDA events (which runs the host-driven solver loop)
    cs = ClockSampler(dev.index)
    with cs:
        ms_local = timed(args.steps)
    barrier(world)
    graph_sweeps = ep.graph_sweeps()
    ep.trace(True)
    ms_traced = timed(args.steps)
    trace = ep.trace_read()
    ep.trace(False)
    st = ep.stats()
    status = ep.status()
    ms_total = max_over_ranks(ms_local, world, dev)
    ms_per_step = ms_total / args.steps
    value = job_throughput(n_px, world, args.steps, ms_total)
    launches = sum(v[1] for v in trace.values())
    dom = max(trace.items(), key=lambda kv: kv[1][0])
    name, (kms, kl, units, bpu) = dom
    peak, peak_src = _peaks()
    achieved = units * bpu / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    traffic = _ncu_traffic(name)
    traffic_per_launch = traffic * units / kl if (traffic is not None and kl) else None
    bound, unit = "hbm", "GB/s"
    if name == "cs_mma":
        # split-BF16 slice products on the tensor cores: per-unit figure 1 BF16 flop
        tpk, tsrc = _bf16_sustained()
        bound, unit, peak, peak_src = "tensor", "TFLOP/s", tpk, tsrc
        achieved = units * bpu / (kms / 1e3) / 1e12 if kms > 0 else 0.0
    if name == "cs_woodbury":
        # FP64 ALU: per-unit figure is FP64 flops; GB300 nominal FP64 1.25 TFLOP/s
        bound, unit, peak, peak_src = "alu", "GFLOP/s (FP64)", 1250.0, "nominal FP64, GB300"
    roofline = {"bound": bound, "kernel": name, "achieved": round(achieved, 1), "peak": peak,
                "peak_source": peak_src, "unit": unit, "frac": round(achieved / peak, 4),
                "traffic": traffic_per_launch,
                "algorithmic_bytes_per_unit": bpu,
                "algorithmic_bytes_per_launch": units * bpu / kl if kl else None,
                "avg_launch_us": kms / kl * 1e3 if kl else None,
                "share_of_step": round(kms / ms_traced, 4) if ms_traced else None,
                "timing": "CUDA events around every launch, in a traced repeat of the timed steps "
                          f"({ms_traced / args.steps:.3f} ms per step traced)"}
    cgi = cg_iteration_roofline(trace, peak, peak_src)
    if cgi is not None:
        roofline["cg_iteration"] = cgi
    ep.close()

    # end to end through the host-buffer API: copies in, all sweeps, posterior out
    e2e = None
    if rank == 0:
        y32 = prob.y.astype(np.float32)
        n_e2e = max(args.steps, em_every or 1)
        t0 = time.perf_counter()
        extra = {}
        if cfg["kind"] == "deconv":
            extra = dict(op=OP_CONV_PERIODIC, kernel=prob.kernel, rbmc_samples=cfg["S"])
        if cfg["kind"] == "cs":
            extra = dict(kw)  # the host call copies y; the operator is the same
        solve_host(y32, prob.xi, prob.beta, n_e2e, em_every=em_every, **extra)
        t1 = time.perf_counter()
        e2e = {"value": round(n_px * n_e2e / (t1 - t0) / 1e6, 3), "unit": "Mpixel-EP-sweeps/s",
               "h2d_bytes_per_step": 4 * y32.size / n_e2e, "d2h_bytes_per_step": 8 * n_px / n_e2e,
               "sweeps_per_call": n_e2e,
               "what": "ep_tv_solve_host: y host->device, init, sweeps with EM, posterior "
                       "mean/var device->host, wall clock"}
    return dict(value=value, ms_per_step=ms_per_step, roofline=roofline, clocks=cs.summary(),
                launches=launches, trace=trace, stats=st, status=status, e2e=e2e, n_px=n_px,
                graph_sweeps=graph_sweeps)


def run_oracle_sample(cfg, budget_s=20.0):
    """The FP64 oracle on a bounded sample of the workload: same generator,
    operator and parameters at a reduced size, sweeps until the time budget."""
    from oracle.ep import EPOracle
    from paper_2110_01585_gb300 import synthetic as syn
    if cfg["kind"] in ("deconv", "batch"):
        side = 64
        width = cfg["kernel"][1] if cfg["kind"] == "deconv" else 9
        bsnr = cfg.get("bsnr_db", 40.0)
        grf = cfg.get("grf", 32.0) * side / (cfg["h"] or 512)
        p = syn.deconv_problem(side, side, kernel=syn.uniform_kernel(width), bsnr_db=bsnr,
                               beta0=cfg["beta0"], seed=cfg["seed"], grf_length=grf)
        pr = syn.rbmc_probes(cfg["S"], side * side, side * side, seed=1)
        o = EPOracle("deconv", p.y, p.xi, p.beta, side, side, kernel=p.kernel, site0="rbmc_cg",
                     probes=pr)
        sample = f"{side}x{side} crop-size instance of the same generator/blur/BSNR, CG mode"
    elif cfg["kind"] == "warmstart":
        side = 64
        p = syn.warmstart_problem(side, side, seed=cfg["seed"], beta=18.157)
        pr = syn.rbmc_probes(8, side * side, side * side, seed=1)
        o = EPOracle("deconv", p.y, p.xi, p.beta, side, side, kernel=p.kernel, site0="rbmc_cg",
                     probes=pr)
        sample = f"{side}x{side} instance of the warm-start workload, CG mode"
    elif cfg["kind"] == "cs" and cfg.get("op") == "hadamard":
        from oracle import operators
        side = 64
        p = syn.hadamard_cs_problem(side, side, ratio=cfg["ratio"], sigma=cfg["sigma"],
                                    beta0=cfg["beta0"], seed=cfg["seed"])
        A = operators.hadamard_matrix(side, side, p.patterns)
        o = EPOracle("cs", p.y, p.xi, p.beta, side, side, A=A, site0="woodbury")
        sample = f"{side}x{side} instance (M = {A.shape[0]} Hadamard patterns) of the same generator"
    elif cfg["kind"] == "cs":
        side = 64
        p = syn.cs_problem(side, side, ratio=cfg["ratio"], sigma=cfg["sigma"], beta0=cfg["beta0"],
                           seed=cfg["seed"])
        o = EPOracle("cs", p.y, p.xi, p.beta, side, side, A=p.A, site0="woodbury")
        sample = f"{side}x{side} instance (M = {p.A.shape[0]}) of the same generator"
    else:
        side = 512
        p = syn.denoise_problem(side, side, sigma=cfg["sigma"], beta=cfg["beta0"], seed=cfg["seed"])
        o = EPOracle("denoise", p.y, p.xi, p.beta, side, side)
        sample = f"{side}x{side} instance of the same generator"
    t0 = time.perf_counter()
    n = 0
    while True:
        o.sweep()
        n += 1
        if cfg["em_every"] and n % cfg["em_every"] == 0:
            o.em_update()
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = 1
    if cfg["kind"] == "cs":
        # the dense Woodbury step runs in multithreaded BLAS
        try:
            from threadpoolctl import threadpool_info
            cores = max(i.get("num_threads", 1) for i in threadpool_info()) or 1
        except Exception:
            cores = os.cpu_count() or 1
    return {"value": round(side * side * n / dt / 1e6, 5), "unit": "Mpixel-EP-sweeps/s", "cores": cores,
            "kind": "oracle", "sample": f"{sample}, {n} sweeps in {dt:.1f} s"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="deconv512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the short denoise4096 and cs128 legs of the default run")
    ap.add_argument("--size", type=int, default=None,
                    help="side of a single-image workload's image (smaller cases for profiling)")
    ap.add_argument("--batch-n", type=int, default=None,
                    help="number of problems of the batched256 workload (default 256)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    cfg = WORKLOADS[args.workload]
    if args.size is not None and cfg["h"] is not None:
        cfg["h"] = cfg["w"] = int(args.size)
    config = {"workload": args.workload, "height": cfg["h"], "width": cfg["w"],
              "l2": "flushed before every timed step (256 MB write, untimed)"}
    if cfg["kind"] == "cs":
        config.update(m=int(0.3 * cfg["h"] * cfg["w"]), sigma=cfg["sigma"], beta0=cfg["beta0"],
                      em_every=cfg["em_every"], precision="Woodbury in FP64",
                      operator=("subsampled 2-D Hadamard (uniform patterns)"
                                if cfg.get("op") == "hadamard" else "dense Gaussian N(0, 1/M)"))
    elif cfg["kind"] == "batch":
        config.update(problems=cfg["n"], sides="log-uniform 64..1024, even",
                      sigma="U[0.02, 0.2]", blur_widths=[1, 5, 9, 15], em_every=cfg["em_every"],
                      rbmc_probes=cfg["S"])
    elif cfg["kind"] == "warmstart":
        config.update(kernel="gaussian 15x15 std 2 periodic", bsnr_db=30.0,
                      l2="not flushed (each sweep is timed alone)")
    elif cfg["kind"] == "deconv":
        config.update(kernel="uniform 9x9 periodic", bsnr_db=cfg["bsnr_db"], beta0=cfg["beta0"],
                      em_every=cfg["em_every"], rbmc_probes=cfg["S"])
    else:
        config.update(sigma=cfg["sigma"], beta=cfg["beta0"])
    config["parallelism"] = f"replicas{world}" if world > 1 else "single"

    if args.impl == "reference":
        if rank != 0:
            return
        steps = []
        for _ in range(args.steps):
            steps.append(run_oracle_sample(cfg, budget_s=max(2.0, 60.0 / max(args.steps + args.warmup, 1)))["value"])
        v = sum(steps) / len(steps)
        cpu = run_oracle_sample(cfg, budget_s=2.0)
        line = {"impl": "reference", "metric": "Mpixel-EP-sweeps/s", "value": v,
                "unit": "Mpixel-EP-sweeps/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": v, "unit": "Mpixel-EP-sweeps/s", "cores": cpu["cores"], "kind": "oracle",
                                 "sample": cpu["sample"]},
                "e2e": {"value": v, "unit": "Mpixel-EP-sweeps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline and cfg["kind"] not in ("batch", "warmstart"):
        cpu = run_oracle_sample(cfg, budget_s=20.0)
    line = {"metric": "Mpixel-EP-sweeps/s", "value": round(res["value"], 3), "unit": "Mpixel-EP-sweeps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(res["ms_per_step"], 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
            "roofline": res["roofline"], "cpu_baseline": cpu, "e2e": res["e2e"],
            "gpu_launches": res["launches"], "clocks": res["clocks"],
            "solver": {"cg_iters_last_sweep": res["stats"]["cg_iters"],
                       "fp64_edges": res["stats"]["n_fp64"], "status": res["status"],
                       "graph_sweeps": res.get("graph_sweeps")},
            "pixels_per_step": res["n_px"],
            "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in res["trace"].items() if v[1]}}
    if "to_posterior" in res:
        line["to_posterior"] = res["to_posterior"]
    if (world == 1 and args.workload == "deconv512" and args.size is None and not args.no_secondary):
        # the prior pass and the compressive-sensing site measured in the same run:
        # short legs of their own workloads, each in a fresh process (as when the
        # workload is benched on its own), reported beside the headline
        line["secondary"] = {}
        for wl, steps in (("denoise4096", 20), ("cs128", 5)):
            cmd = [sys.executable, os.path.abspath(__file__), "--workload", wl, "--steps", str(steps),
                   "--warmup", "3", "--no-cpu-baseline"]
            out = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
            try:
                r2 = json.loads(out.stdout.strip().splitlines()[-1])
            except (ValueError, IndexError):
                line["secondary"][wl] = {"error": (out.stderr or out.stdout)[-400:]}
                continue
            line["secondary"][wl] = {k: r2[k] for k in ("value", "unit", "steps", "warmup", "ms_per_step",
                                                          "roofline", "clocks", "e2e", "kernels",
                                                          "gpu_launches") if k in r2}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
