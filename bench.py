#!/usr/bin/env python
"""Benchmark: batched HMC posteriors per minute at fixed ESS on one GB300.

Workload (one "step" = one pass of the whole hot path over one batch):
4,096 galaxies x 4 chains, production SSP grid (107 ages x 12 metallicities x
5,994 wavelengths), 12 Gaussian bands 300-2400 nm with 3-12 observed per
galaxy, trajectory lengths U(8, 64), 500 warm-up + 500 sampling iterations,
per-chain dual-averaged step size, approximate photometry, one persistent
graph-captured launch.  Inputs are synthetic and seeded (sps_workloads);
observed magnitudes are the model at a seeded truth plus N(0, 0.05) noise.

value = sum_g min(1, ESS_g / 100) / (minutes per step), ESS_g the minimum over
the 12 parameters of the multi-chain ESS of galaxy g.

Also reported: the same sampler run as the plain lock-step forward-mode
baseline (posteriors/min at equal ESS), NUTS in the same kernel on the same
galaxies (100 + 100 iterations, its own ESS), the cost of the model
extensions (skew-normal prior, age-dependent MDF, tabulated filter curves), log-likelihood + gradient
evaluations per second on 100,000 (galaxy, chain) pairs (approximate FP32,
exact FP32, exact BF16), the
roofline of the dominant kernel, the clocks seen during the timed region,
an end-to-end number through the C ABI with host buffers, and the FP64
oracle timed on a bounded sample on the host cores.
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

import sps_workloads as W  # noqa: E402

ESS_TARGET = 100.0
# Dual-averaging target acceptance of the HMC legs.  With the workload's
# fixed trajectory lengths L ~ U(8, 64), a lower target lengthens each
# trajectory; measured on the full workload at 500 + 500 iterations,
# posteriors/min at fixed ESS: 0.6 -> 3,599, 0.65 -> 4,264, 0.7 -> 4,634-4,655,
# 0.72 -> 4,689, 0.75 -> 4,627, 0.8 (the library default) -> 4,286, 0.9 -> 3,179.
TARGET_ACCEPT = 0.7
METRIC = "posteriors/min at fixed ESS"
UNIT = "posteriors/min"

# DRAM traffic of one bench step's k_hmc_team launches on this workload (the
# whole waves of two-chain teams and the last wave's one-chain teams;
# dram__bytes_read.sum + dram__bytes_write.sum, mean of five steps of a reduced
# case with the same 4,096-galaxy working set at 50 + 50 iterations, scaled by
# gradient evaluations to 500 + 500; profiles/k_hmc_team_hmc4096gal_x4_launches.md),
# valid only while the kernel's sources hash to the recorded value; otherwise
# reported as null.
KERNEL_SOURCES = ("hmc_team.cu", "sps_device.cuh", "sps_eval.cuh", "sps_internal.h", "philox.cuh")
TRAFFIC = {"sha": "3c9f052df06e2568", "bytes": 217.10e9 + 11.23e9}


def _kernel_sha():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2506_19919_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
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
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("SPS_BENCH_GLOO") is None else "gloo")
    return ws, rank


def _reduce(x: float, ws: int, op: str) -> float:
    """All-reduce of one number over the ranks ("max" or "sum"); the identity
    for one rank.  CUDA tensors under NCCL, CPU tensors under gloo."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def _max_over_ranks(x: float, ws: int) -> float:
    return _reduce(x, ws, "max")


def job_value(post: float, ms_step: float, ws: int):
    """Whole-job posteriors/min: the posteriors of all ranks (each rank runs
    its own seeded batch) over the slowest rank's step time."""
    ms = _reduce(ms_step, ws, "max")
    return _reduce(post, ws, "sum") / (ms / 60000.0), ms


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _hmc_workload(rank: int, n_gal: int | None = None, iters=None):
    wl = W.config(3, n_gal=n_gal, seed_offset=rank)
    if iters is not None:                      # reduced run for profiling captures only
        wl.extra["n_warm"], wl.extra["n_samp"] = iters
    return wl


def _config(tables, G, C, n_warm, n_samp, L, sampler, mdf_age, ws):
    """The workload description of the bench line (both arms)."""
    return {"workload": W.CONFIG_NAMES[3], "galaxies": G, "chains_per_gal": C,
            "n_warm": n_warm, "n_samp": n_samp, "L": list(L), "target_accept": TARGET_ACCEPT,
            "ssp_grid": [tables.n_age, tables.n_met, tables.n_lam],
            "bands": tables.n_band, "photometry": "approx", "sampler": sampler,
            "mdf": "age-dependent" if mdf_age else "separable",
            "l2": "flushed (256 MB write) between timed steps; working set > L2",
            "parallelism": f"replicas{ws}"}


def run_ours(args):
    import torch

    import paper_2506_19919_gb300 as pkg
    from paper_2506_19919_gb300 import _lib

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = _hmc_workload(rank, args.gal, (args.warm, args.samp) if args.warm is not None else None)
    if args.mdf_age:
        wl.tables = W.with_mdf_offset(wl.tables, W.mzr_offsets(wl.tables.age_yr, slope=0.25))
    G, C = wl.n_gal, wl.chains
    n_warm, n_samp = wl.extra["n_warm"], wl.extra["n_samp"]
    ctx = pkg.Context(wl.tables, device=local)
    ctx.set_galaxies(wl.z, build_approx=True)
    # data: the model at the seeded truth plus seeded noise
    mtrue = ctx.photometry(torch.as_tensor(wl.theta_true, dtype=torch.float32, device=dev),
                           mode="approx")
    mobs = (mtrue + torch.as_tensor(wl.noise, dtype=torch.float32, device=dev)).contiguous()
    sigma = torch.as_tensor(wl.sigma, dtype=torch.float32, device=dev)
    mask = torch.as_tensor(wl.mask.view(np.int32), device=dev)
    x0 = torch.as_tensor(wl.extra["theta0_unb"], dtype=torch.float32, device=dev)
    NC = G * C
    samples = torch.empty((NC, n_samp, 12), dtype=torch.float32, device=dev)
    stats = {k: torch.empty(NC, dtype=t, device=dev) for k, t in
             (("accept_prob", torch.float32), ("step_size", torch.float32),
              ("divergences", torch.int32), ("grad_evals", torch.int64), ("status", torch.int32))}
    cfg = _lib.sps_hmc_config()
    lib = _lib.load()
    lib.sps_hmc_config_default(__import__("ctypes").byref(cfg))
    cfg.chains_per_gal, cfg.n_warm, cfg.n_samp = C, n_warm, n_samp
    cfg.L_min, cfg.L_max = wl.extra["L_min"], wl.extra["L_max"]
    cfg.seed = 2506199190 + rank
    cfg.target_accept = TARGET_ACCEPT
    cfg.use_graph, cfg.autotune = 1, 1
    cfg.sampler = 1 if args.sampler == "nuts" else 0
    import ctypes as Ct
    st = _lib.sps_hmc_stats(*(Ct.c_void_p(stats[k].data_ptr()) for k in
                              ("accept_prob", "step_size", "divergences", "grad_evals", "status")))
    stream = torch.cuda.current_stream(dev)
    sp = Ct.c_void_p(stream.cuda_stream)
    vp = lambda t: Ct.c_void_p(t.data_ptr())
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        _lib.check(lib.sps_hmc_run(ctx.h, Ct.byref(cfg), vp(x0), vp(mobs), vp(sigma), vp(mask),
                                   vp(samples), Ct.byref(st), sp), "sps_hmc_run")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    _barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))                    # L2 flush between timed steps
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    ms_local = float(np.mean(kern_ms))

    # ESS from the last step's draws (host diagnostics, outside the timed region)
    ess, rhat = pkg.diagnostics(samples, G, C)
    ess_g = ess.min(1)
    post = float(np.minimum(1.0, ess_g / ESS_TARGET).sum())
    value, ms_step = job_value(post, ms_local, ws)
    nev = stats["grad_evals"].cpu().numpy()
    nb = np.array([bin(int(m)).count("1") for m in wl.mask])
    K = wl.tables.n_age * wl.tables.n_met
    flop = float(((4 * nb * K)[:, None] * nev.reshape(G, C)).sum())
    peaks, src = _peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12          # TFLOP/s, FMA pipe
    achieved = flop / (ms_step / 1e3) / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(wl.tables, G, C, n_warm, n_samp, (cfg.L_min, cfg.L_max), args.sampler,
                          args.mdf_age, ws),
        "ess": {"target": ESS_TARGET, "galaxies_at_target": int((ess_g >= ESS_TARGET).sum()),
                "median_ess": float(np.median(ess_g)), "median_rhat_max": float(np.median(rhat.max(1))),
                "frac_rhat_lt_1p2": float((rhat.max(1) < 1.2).mean()),
                "accept_mean": float(stats["accept_prob"].mean()),
                "divergences": int(stats["divergences"].sum())},
        "grad_evals_per_s": _reduce(float(nev.sum()), ws, "sum") / (ms_step / 1e3),
        "roofline": {"kernel": "k_hmc_team", "bound": "alu", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": TRAFFIC["bytes"] if _kernel_sha() == TRAFFIC["sha"] else None,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (derived)",
                     "algorithmic": "4 * n_obs_bands * K FLOP per gradient evaluation"},
        "clocks": clocks,
        "gpu_launches": args.steps * max(1, int(ctx.info().get("hmc_launches", 1))),
        "wall_s": wall,
    }
    if rank == 0 and not args.skip_extra:
        out["loglike_grad"] = _loglike_grad_rates(ctx, dev)
    if rank == 0 and not args.skip_errors:
        out["error"] = _errors(dev)
    if rank == 0 and not args.skip_survey:
        out["survey"] = _survey(dev)
    if rank == 0 and not args.skip_plain:
        out["plain_hmc"] = _plain_hmc(ctx, wl, x0, mobs, post, value, ms_step, args.plain_full)
        out["plain_hmc"]["own_ess_full_runs"] = _own_ess_runs(dev)
    if rank == 0 and not args.skip_nuts:
        out["nuts"] = _nuts(ctx, wl, x0, mobs, value, float(nev.sum()) / (ms_local / 1e3))
    if rank == 0 and not args.skip_exact_hmc:
        out["hmc_exact"] = _hmc_exact(ctx, wl, x0, mobs, ms_step / 1e3)
    if rank == 0 and not args.skip_models:
        out["models"] = _models(wl, dev)
    if not args.skip_e2e:                       # every rank (collective timing)
        out["e2e"] = _e2e(ctx, cfg, lib, wl, mobs, x0, post, ws)
    if rank == 0 and ws == 1 and not args.skip_cpu:
        out["cpu_baseline"] = _cpu_baseline(wl, mobs.cpu().numpy(), post / G, budget_s=args.cpu_budget)
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _plain_hmc(ctx, wl, x0, mobs, post, value, ms_step, full):
    """The lock-step forward-mode baseline (sps_hmc_run_forward_mode) on the
    same workload and sampler.  By default a bounded run (its cost per
    iteration is fixed: L_max rounds of every chain) is timed and scaled to the
    full iteration count; the two paths run the same sampler on the same Philox
    streams, so posteriors/min is compared at the fused run's ESS.  With full,
    the whole run is timed and its own ESS reported as well."""
    import torch

    import paper_2506_19919_gb300 as pkg
    G, C = wl.n_gal, wl.chains
    n_it = wl.extra["n_warm"] + wl.extra["n_samp"]
    kw = dict(chains_per_gal=C, L_min=wl.extra["L_min"], L_max=wl.extra["L_max"],
              seed=2506199190, path="plain", target_accept=TARGET_ACCEPT)
    res = {"path": "sps_hmc_run_forward_mode: chains in lock step, L_max rounds per iteration, "
                   "unfused forward-mode gradient of every chain every round"}
    if full:
        nw, ns = wl.extra["n_warm"], wl.extra["n_samp"]
    else:
        nw, ns = 12, 12
    ctx.hmc_run(x0, mobs, wl.sigma, wl.mask, n_warm=2, n_samp=2, samples=False, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    o = ctx.hmc_run(x0, mobs, wl.sigma, wl.mask, n_warm=nw, n_samp=ns, samples=full, **kw)
    e1.record()
    torch.cuda.synchronize()
    s_run = e0.elapsed_time(e1) / 1e3
    s_step = s_run * n_it / (nw + ns)
    nev = float(o["grad_evals"].sum())
    res.update({"iterations_timed": nw + ns, "s_timed": s_run, "s_per_step": s_step,
                "grad_evals_per_s": nev / s_run,
                "posteriors_per_min_at_equal_ess": post / (s_step / 60.0),
                "fused_vs_plain_posteriors_per_min": value / (post / (s_step / 60.0)),
                "fused_vs_plain_step_time": s_step / (ms_step / 1e3)})
    if full:
        ess, rhat = pkg.diagnostics(o["samples"], G, C)
        ess_g = ess.min(1)
        own = float(np.minimum(1.0, ess_g / ESS_TARGET).sum())
        res.update({"own_median_ess": float(np.median(ess_g)),
                    "own_posteriors_per_min": own / (s_run / 60.0),
                    "own_frac_rhat_lt_1p2": float((rhat.max(1) < 1.2).mean())})
    return res


def _own_ess_runs(dev, n_gal=512):
    """Both samplers run in full (500 + 500 iterations) on 512 galaxies of
    the bench recipe, 4 chains each, each scored by the ESS of its own draws:
    the fused-vs-baseline comparison measured end to end, without scaling
    iterations or borrowing the other run's ESS."""
    import torch

    import paper_2506_19919_gb300 as pkg
    wl = _hmc_workload(0, n_gal)
    G, C = wl.n_gal, wl.chains
    ctx = pkg.Context(wl.tables, device=dev.index)
    ctx.set_galaxies(wl.z, build_approx=True)
    mt = ctx.photometry(torch.as_tensor(wl.theta_true, dtype=torch.float32, device=dev), mode="approx")
    mobs = (mt + torch.as_tensor(wl.noise, dtype=torch.float32, device=dev)).contiguous()
    x0 = torch.as_tensor(wl.extra["theta0_unb"], dtype=torch.float32, device=dev)
    kw = dict(chains_per_gal=C, L_min=wl.extra["L_min"], L_max=wl.extra["L_max"], seed=2506199190,
              target_accept=TARGET_ACCEPT)
    n_warm, n_samp = wl.extra["n_warm"], wl.extra["n_samp"]
    out = {"galaxies": G, "chains_per_gal": C, "n_warm": n_warm, "n_samp": n_samp}
    for path in ("fused", "plain"):
        ctx.hmc_run(x0, mobs, wl.sigma, wl.mask, n_warm=2, n_samp=2, samples=False, path=path, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        o = ctx.hmc_run(x0, mobs, wl.sigma, wl.mask, n_warm=n_warm, n_samp=n_samp, path=path, **kw)
        e1.record()
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1e3
        ess, rhat = pkg.diagnostics(o["samples"], G, C)
        ess_g = ess.min(1)
        post = float(np.minimum(1.0, ess_g / ESS_TARGET).sum())
        out[path] = {"s": s, "median_ess": float(np.median(ess_g)), "posteriors_per_min": post / (s / 60.0),
                     "frac_rhat_lt_1p2": float((rhat.max(1) < 1.2).mean())}
    out["fused_vs_plain_posteriors_per_min"] = (out["fused"]["posteriors_per_min"] /
                                                max(out["plain"]["posteriors_per_min"], 1e-30))
    ctx.close()
    return out


def _hmc_exact(ctx, wl, x0, mobs, hmc_s_per_step):
    """HMC on the exact photometry (BF16 contraction on the tensor cores) on
    the bench galaxies and start points: every round evaluates every chain's
    gradient through the exact path and takes one trajectory-asynchronous
    leapfrog step.  A bounded run (10 + 10 iterations) is timed and scaled to
    the workload's 500 + 500 by its cost per round; the paper's comparison is
    the exact-photometry run against the approximate one."""
    import torch
    G, C = wl.n_gal, wl.chains
    nw = ns = 10
    kw = dict(chains_per_gal=C, L_min=wl.extra["L_min"], L_max=wl.extra["L_max"], seed=2506199190,
              mode="exact", prec="bf16", samples=False, target_accept=TARGET_ACCEPT)
    ctx.hmc_run(x0, mobs, wl.sigma, wl.mask, n_warm=1, n_samp=0, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    o = ctx.hmc_run(x0, mobs, wl.sigma, wl.mask, n_warm=nw, n_samp=ns, **kw)
    e1.record()
    torch.cuda.synchronize()
    s_run = e0.elapsed_time(e1) / 1e3
    nev = float(o["grad_evals"].sum())
    n_it = wl.extra["n_warm"] + wl.extra["n_samp"]
    s_full = s_run * n_it / (nw + ns)
    return {"path": "sps_hmc_run mode EXACT, BF16 tcgen05 contraction, one gradient per chain per round",
            "iterations_timed": nw + ns, "s_timed": s_run, "grad_evals_per_s": nev / s_run,
            "projected_s_for_500_plus_500": s_full,
            "exact_vs_approx_step_time": s_full / hmc_s_per_step,
            "accept_mean": float(o["accept_prob"].mean()), "divergences": int(o["divergences"].sum())}


def _nuts(ctx, wl, x0, mobs, hmc_value, hmc_evals_per_s):
    """NUTS (multinomial, generalised U-turn, depth limit 10, identity metric)
    in the same persistent kernel on the same galaxies and start points, run
    for 100 warm-up + 100 sampling iterations (a full 500 + 500 run takes
    about 100 s), and scored by the same metric with its own ESS."""
    import torch

    import paper_2506_19919_gb300 as pkg
    G, C = wl.n_gal, wl.chains
    nw = ns = 100
    kw = dict(chains_per_gal=C, seed=2506199190, sampler="nuts", max_depth=10)
    ctx.hmc_run(x0, mobs, wl.sigma, wl.mask, n_warm=2, n_samp=2, samples=False, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    o = ctx.hmc_run(x0, mobs, wl.sigma, wl.mask, n_warm=nw, n_samp=ns, **kw)
    e1.record()
    torch.cuda.synchronize()
    s_run = e0.elapsed_time(e1) / 1e3
    ess, rhat = pkg.diagnostics(o["samples"], G, C)
    ess_g = ess.min(1)
    post = float(np.minimum(1.0, ess_g / ESS_TARGET).sum())
    nev = o["grad_evals"].cpu().numpy().astype(np.float64)
    eps = float(nev.sum()) / s_run
    return {"sampler": "NUTS, multinomial, generalised U-turn, max depth 10, identity metric",
            "n_warm": nw, "n_samp": ns, "s": s_run, "posteriors_per_min": post / (s_run / 60.0),
            "vs_hmc_posteriors_per_min": post / (s_run / 60.0) / hmc_value,
            "median_ess": float(np.median(ess_g)), "frac_rhat_lt_1p2": float((rhat.max(1) < 1.2).mean()),
            "leaves_per_iteration": float((nev - 1.0).mean() / (nw + ns)),
            "grad_evals_per_s": eps, "vs_hmc_grad_evals_per_s": eps / hmc_evals_per_s,
            "accept_mean": float(o["accept_prob"].mean()), "divergences": int(o["divergences"].sum())}


def _models(wl, dev):
    """Cost of the model extensions against the base model on the same
    workloads: HMC (100 + 100 iterations on the bench galaxies and start
    points) with the skew-normal prior, and with an age-dependent MDF mean
    (general W; the row-evaluation variant of the kernel); log L + gradient on
    100,000 pairs (the loglike workload) with the age-dependent MDF and with a
    tabulated filter set (synthetic measured-style curves, one sample per 10 A)
    in place of the Gaussian bands."""
    import torch

    import paper_2506_19919_gb300 as pkg
    from paper_2506_19919_gb300 import priors as P

    def hmc_time(tables, **ctx_kw):
        ctx = pkg.Context(tables, device=dev.index, **ctx_kw)
        ctx.set_galaxies(wl.z, build_approx=True)
        mt = ctx.photometry(torch.as_tensor(wl.theta_true, dtype=torch.float32, device=dev), mode="approx")
        mo = (mt + torch.as_tensor(wl.noise, dtype=torch.float32, device=dev)).contiguous()
        x0 = torch.as_tensor(wl.extra["theta0_unb"], dtype=torch.float32, device=dev)
        kw = dict(chains_per_gal=wl.chains, seed=2506199190, L_min=wl.extra["L_min"], L_max=wl.extra["L_max"],
                  samples=False, target_accept=TARGET_ACCEPT)
        ctx.hmc_run(x0, mo, wl.sigma, wl.mask, n_warm=2, n_samp=2, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        o = ctx.hmc_run(x0, mo, wl.sigma, wl.mask, n_warm=100, n_samp=100, **kw)
        e1.record()
        torch.cuda.synchronize()
        s_run = e0.elapsed_time(e1) / 1e3
        nev = float(o["grad_evals"].sum())
        ctx.close()
        return {"s": s_run, "grad_evals_per_s": nev / s_run}

    def ll_times(tables):
        w2 = W.config(2)
        ctx = pkg.Context(tables, device=dev.index)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_galaxies(w2.z, build_approx=True)
        torch.cuda.synchronize()
        res = {"set_galaxies_s": time.perf_counter() - t0}
        th = torch.as_tensor(w2.theta, dtype=torch.float32, device=dev)
        mobs = ctx.photometry(torch.as_tensor(w2.theta_true, dtype=torch.float32, device=dev),
                              mode="approx") + torch.as_tensor(w2.noise, dtype=torch.float32, device=dev)
        sg = torch.as_tensor(w2.sigma, dtype=torch.float32, device=dev)
        mk = torch.as_tensor(w2.mask.view(np.int32), device=dev)
        for mode, prec, reps in (("approx", "fp32", 10), ("exact", "bf16", 3)):
            ctx.loglike_grad(th, mobs, sg, mk, mode=mode, prec=prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                ctx.loglike_grad(th, mobs, sg, mk, mode=mode, prec=prec)
            e1.record()
            torch.cuda.synchronize()
            res[f"{mode}_{prec}_ms"] = e0.elapsed_time(e1) / reps
        ctx.close()
        return res

    base2 = W.config(2).tables
    off = W.mzr_offsets(wl.tables.age_yr, slope=0.25)
    tab = W.tabulated_bands(np.random.default_rng(7), [360, 482, 604, 726, 848, 970, 1092])
    res = {"workloads": "HMC: the bench galaxies, 100 + 100 iterations; log L + gradient: "
                        + W.CONFIG_NAMES[2],
           "hmc_base": hmc_time(wl.tables),
           "hmc_skew_prior": hmc_time(wl.tables, skew=P.skew_normal_prior(wl.theta_true, W.PRIOR_LO, W.PRIOR_HI)),
           "hmc_age_dependent_mdf": hmc_time(W.with_mdf_offset(wl.tables, off)),
           "loglike_base": ll_times(base2),
           "loglike_age_dependent_mdf": ll_times(W.with_mdf_offset(base2, W.mzr_offsets(base2.age_yr, 0.25))),
           "loglike_tabulated_bands": ll_times(W.with_bands(base2, *tab))}
    return res


def _e2e(ctx, cfg, lib, wl, mobs_dev, x0_dev, post, ws):
    """Same metric through the C ABI with pinned host buffers: the call stages
    the inputs to the device and copies the draws back inside the timed region."""
    import ctypes as Ct

    from paper_2506_19919_gb300 import _lib
    import torch
    G, C = wl.n_gal, wl.chains
    NC = G * C
    keep = []                                     # the pinned tensors behind the arrays

    def pinned(shape, dtype, src=None):
        t = torch.empty(shape, dtype=dtype, pin_memory=True)
        keep.append(t)
        a = t.numpy()
        if src is not None:
            a[...] = src
        return a

    x0 = pinned(tuple(x0_dev.shape), torch.float32, x0_dev.cpu().numpy())
    mobs = pinned(tuple(mobs_dev.shape), torch.float32, mobs_dev.cpu().numpy())
    sigma = pinned(wl.sigma.shape, torch.float32, wl.sigma)
    mask = pinned(wl.mask.shape, torch.int32, wl.mask.view(np.int32)).view(np.uint32)
    samples = pinned((NC, cfg.n_samp, 12), torch.float32)
    acc = pinned((NC,), torch.float32)
    st = _lib.sps_hmc_stats(acc.ctypes.data, None, None, None, None)
    vp = lambda a: Ct.c_void_p(a.ctypes.data)
    times = []
    for _ in range(2):
        _barrier(ws)
        t0 = time.perf_counter()
        _lib.check(lib.sps_hmc_run(ctx.h, Ct.byref(cfg), vp(x0), vp(mobs), vp(sigma), vp(mask),
                                   vp(samples), Ct.byref(st), None), "sps_hmc_run (host)")
        times.append(_reduce(time.perf_counter() - t0, ws, "max"))
    t = min(times)
    h2d = x0.nbytes + mobs.nbytes + sigma.nbytes + mask.nbytes + 4 * G
    d2h = samples.nbytes + acc.nbytes
    return {"value": _reduce(post, ws, "sum") / (t / 60.0), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "s_per_step": t}


def _errors(dev):
    """Error of every path and precision against the FP64 oracle on sampled
    rows of the workloads: magnitudes (|dm| in mag), log L (relative) and the
    13-column gradient (12 parameters and z; per row the max-component error
    over the largest component), max and median over the rows.  The oracle's
    values were stored by tests/golden/make_bench_reference.py; the GPU side
    runs the library's public calls on the same rows (no oracle is run here)."""
    import torch

    import paper_2506_19919_gb300 as pkg
    with open(os.path.join(ROOT, "tests", "golden", "bench_error_reference.json")) as f:
        ref = json.load(f)
    tables = {W.CONFIG_NAMES[2]: W.config(2, n_gal=1).tables, W.CONFIG_NAMES[3]: W.config(3, n_gal=1).tables}
    stat = lambda v: {"max": float(np.max(v)), "median": float(np.median(v))}
    out = {"reference": "FP64 oracle on the sampled rows (tests/golden/bench_error_reference.json)",
           "gradient_measure": "per row max_k |g_k - g_ref,k| / max_k |g_ref,k| over 12 parameters and z"}
    for name, r in ref.items():
        z = np.asarray(r["z"])
        th = np.asarray(r["theta"], np.float32)
        mobs = np.asarray(r["mag_obs"], np.float32)
        sg = np.asarray(r["sigma"], np.float32)
        mk = np.asarray(r["mask"], np.int64).astype(np.uint32)
        ctx = pkg.Context(tables[name], device=dev.index)
        ctx.set_galaxies(z, build_approx=True)
        res = {"rows": len(z)}
        modes = [("approx", "fp32")] + ([("exact", "fp32"), ("exact", "bf16"), ("exact", "tf32x3")]
                                        if "mag_exact" in r else [])
        for mode, prec in modes:
            m = ctx.photometry(th, mode=mode, prec=prec).cpu().numpy().astype(np.float64)
            dm = np.abs(m - np.asarray(r[f"mag_{mode}"]))
            ll, g = ctx.loglike_grad_z(th, mobs, sg, mk, mode=mode, prec=prec)
            gref = np.asarray(r[f"grad_{mode}"])
            gg = g.cpu().numpy().astype(np.float64)
            grel = np.abs(gg - gref).max(1) / np.abs(gref).max(1)
            lref = np.asarray(r[f"loglike_{mode}"])
            lrel = np.abs(ll.cpu().numpy().astype(np.float64) - lref) / np.abs(lref)
            res[f"{mode}_{prec}"] = {"mag_abs": stat(dm), "loglike_rel": stat(lrel), "gradient_rel": stat(grel)}
            if mode == "approx":       # the 12-column team evaluation the samplers use
                _, g12 = ctx.loglike_grad(th, mobs, sg, mk, mode="approx")
                g12 = g12.cpu().numpy().astype(np.float64)
                res["approx_fp32_team12"] = {"gradient_rel": stat(
                    np.abs(g12 - gref[:, :12]).max(1) / np.abs(gref[:, :12]).max(1))}
        ctx.close()
        out[name] = res
    torch.cuda.synchronize()
    return out


def _loglike_grad_rates(ctx_hmc, dev):
    """loglike + gradient evaluations per second on 100,000 pairs."""
    import torch

    import paper_2506_19919_gb300 as pkg
    wl = W.config(2)
    ctx = pkg.Context(wl.tables, device=dev.index)
    ctx.set_galaxies(wl.z, build_approx=True)
    th = torch.as_tensor(wl.theta, dtype=torch.float32, device=dev)
    mobs = ctx.photometry(torch.as_tensor(wl.theta_true, dtype=torch.float32, device=dev),
                          mode="approx") + torch.as_tensor(wl.noise, dtype=torch.float32, device=dev)
    # inputs resident on the device (uploaded once, outside the timed calls)
    sg = torch.as_tensor(wl.sigma, dtype=torch.float32, device=dev)
    mk = torch.as_tensor(wl.mask.view(np.int32), device=dev)
    res = {"pairs": wl.n_gal, "workload": W.CONFIG_NAMES[2], "inputs": "device-resident"}

    def timed(call, reps):
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            call()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # tensor-core throughput of the exact path: 2 K Lambda FLOP per row and
    # contraction (the unpadded grid), one contraction for photometry and two
    # (forward and adjoint) for log L + gradient; BF16 against the measured
    # BF16 peak, 3xTF32 (three TF32 products per FLOP) against that peak times
    # the nominal TF32 / BF16 ratio 1.1 / 2.25
    peaks, src = _peaks()
    flop_row = 2.0 * wl.tables.n_age * wl.tables.n_met * wl.tables.n_lam

    def tensor(ms, n_gemm, prec):
        if prec not in ("bf16", "tf32x3"):
            return {}
        tf = n_gemm * flop_row * wl.n_gal / (ms / 1e3) / 1e12
        peak = peaks["bf16_tflops"] * (1.0 if prec == "bf16" else 1.1 / 2.25)
        return {"tensor_tflops": tf, "tensor_frac": tf * (3.0 if prec == "tf32x3" else 1.0) / peak,
                "tensor_peak_tflops": peak, "peak_source": src}

    for mode, prec, reps in (("approx", "fp32", 10), ("plain", "fp32", 3), ("exact", "fp32", 2),
                             ("exact", "bf16", 3), ("exact", "tf32x3", 3)):
        def call():
            if mode == "plain":
                ctx.loglike_grad_forward_mode(th, mobs, sg, mk)
            else:
                ctx.loglike_grad(th, mobs, sg, mk, mode=mode, prec=prec)
        ms = timed(call, reps)
        res[f"{mode}_{prec}"] = {"evals_per_s": wl.n_gal / (ms / 1e3), "ms": ms, **tensor(ms, 2, prec)}
    res["fused_adjoint_vs_plain_forward_mode"] = (res["approx_fp32"]["evals_per_s"]
                                                  / res["plain_fp32"]["evals_per_s"])
    # production photometry (magnitudes only) on the same 100,000 galaxies
    phot = {"galaxies": wl.n_gal}
    for mode, prec, reps in (("approx", "fp32", 10), ("exact", "fp32", 2), ("exact", "bf16", 5),
                             ("exact", "tf32x3", 3)):
        ms = timed(lambda: ctx.photometry(th, mode=mode, prec=prec), reps)
        phot[f"{mode}_{prec}"] = {"galaxies_per_s": wl.n_gal / (ms / 1e3), "ms": ms, **tensor(ms, 1, prec)}
    res["photometry"] = phot
    ctx.close()
    return res


def _cpu_baseline(wl, mobs, post_frac, budget_s=20.0):
    """The FP64 oracle's HMC, as it stands, on a bounded sample of the same
    workload (2 galaxies x 4 chains, a few iterations), extrapolated to the
    full 1,000-iteration run per galaxy; the ESS fraction per galaxy is taken
    from the GPU run of the same sampler."""
    import torch

    from oracle import hmc as OH
    n = 2
    tgt = OH.ApproxTarget(wl.tables, wl.z[:n], mobs[:n], wl.sigma[:n], wl.mask[:n],
                          W.PRIOR_LO, W.PRIOR_HI)
    x0 = wl.extra["theta0_unb"][: n * wl.chains]
    it_total = wl.extra["n_warm"] + wl.extra["n_samp"]
    t0 = time.perf_counter()
    c0 = time.process_time()
    iters = 0
    while True:
        OH.run_hmc(tgt, x0, np.repeat(np.arange(n), wl.chains), seed=1, n_warm=1, n_samp=0,
                   L_min=wl.extra["L_min"], L_max=wl.extra["L_max"], target_accept=TARGET_ACCEPT)
        iters += 1
        if time.perf_counter() - t0 > budget_s or iters >= 50:
            break
    wall = time.perf_counter() - t0
    cores_used = (time.process_time() - c0) / wall   # CPU seconds per wall second of the sample
    dt = wall / iters                                 # s per iteration for n galaxies
    s_per_gal = dt * it_total / n
    value = post_frac * 60.0 / s_per_gal
    return {"value": value, "unit": UNIT, "cores": torch.get_num_threads(),
            "cpu_busy": round(cores_used, 2), "nproc": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} galaxies x {wl.chains} chains x {iters} iterations of the FP64 "
                      f"oracle HMC ({dt:.2f} s/iteration), extrapolated to {it_total} iterations "
                      f"per galaxy; " + ("ESS fraction taken as 1, an upper bound for the oracle"
                                         if post_frac == 1.0 else
                                         f"ESS fraction per galaxy {post_frac:.3g} from the GPU run")}


def run_loglike_only(args):
    """loglike + gradient throughput on the 100,000-pair workload only (or a
    smaller galaxy count for profiling captures)."""
    import torch

    import paper_2506_19919_gb300 as pkg
    wl = W.config(2, n_gal=args.gal)
    dev = torch.device("cuda", 0)
    ctx = pkg.Context(wl.tables, device=0)
    ctx.set_galaxies(wl.z, build_approx=True)
    th = torch.as_tensor(wl.theta, dtype=torch.float32, device=dev)
    mobs = ctx.photometry(torch.as_tensor(wl.theta_true, dtype=torch.float32, device=dev),
                          mode="approx") + torch.as_tensor(wl.noise, dtype=torch.float32, device=dev)
    out = {"pairs": wl.n_gal}
    for spec in args.loglike_only.split(","):
        mode, prec = spec.split("_")
        def call():
            if mode == "plain":
                ctx.loglike_grad_forward_mode(th, mobs, wl.sigma, wl.mask)
            else:
                ctx.loglike_grad(th, mobs, wl.sigma, wl.mask, mode=mode, prec=prec)
        for _ in range(args.warmup):
            call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            call()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[spec] = {"ms": ms, "evals_per_s": wl.n_gal / (ms / 1e3)}
    print(json.dumps(out))


def run_survey(args):
    import torch
    print(json.dumps(_survey(torch.device("cuda", 0))))


def _survey(dev):
    """Throughput on the large bursty survey batch (1,000,000 galaxies x 2
    chains, 20 bands, 6-20 observed, burst on, 300 + 300 iterations): table
    build, log L + gradient on all 2,000,000 (galaxy, chain) pairs (FP32
    approximate and BF16 exact), and the HMC kernel on all chains for a few
    iterations, projected to the full run by its cost per iteration."""
    import torch

    import paper_2506_19919_gb300 as pkg
    wl = W.config(4)
    G, C = wl.n_gal, wl.chains
    ctx = pkg.Context(wl.tables, device=dev.index)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.set_galaxies(wl.z, build_approx=True)
    torch.cuda.synchronize()
    t_tables = time.perf_counter() - t0
    th = torch.as_tensor(np.repeat(wl.theta_true, C, axis=0), dtype=torch.float32, device=dev)
    gi = torch.as_tensor(np.repeat(np.arange(G, dtype=np.int32), C), device=dev)
    mobs = torch.as_tensor((np.full((G, 20), 23.0) + wl.noise).astype(np.float32), device=dev)
    sigma = torch.as_tensor(wl.sigma, device=dev)
    mask = torch.as_tensor(wl.mask.view(np.int32), device=dev)
    out = {"workload": W.CONFIG_NAMES[4], "galaxies": G, "chains_per_gal": C, "bands": 20,
           "table_build_s": t_tables}

    def rate(fn, n, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        return {"ms": ms, "evals_per_s": n / (ms / 1e3)}
    out["loglike_grad_approx_fp32"] = rate(
        lambda: ctx.loglike_grad(th, mobs, sigma, mask, gal_idx=gi, mode="approx"), G * C, 3)
    out["loglike_grad_exact_bf16"] = rate(
        lambda: ctx.loglike_grad(th[::C].contiguous(), mobs, sigma, mask, mode="exact", prec="bf16"), G, 2)
    x0 = torch.as_tensor(wl.extra["theta0_unb"], dtype=torch.float32, device=dev)
    n_it = wl.extra["n_warm"] + wl.extra["n_samp"]
    kw = dict(chains_per_gal=C, L_min=wl.extra["L_min"], L_max=wl.extra["L_max"], samples=False)
    ctx.hmc_run(x0, mobs, sigma, mask, n_warm=2, n_samp=0, **kw)
    torch.cuda.synchronize()
    runs = {}
    for it in (4, 12):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        o = ctx.hmc_run(x0, mobs, sigma, mask, n_warm=it, n_samp=0, **kw)
        e1.record()
        torch.cuda.synchronize()
        runs[it] = (e0.elapsed_time(e1) / 1e3, float(o["grad_evals"].sum()))
    per_it = (runs[12][0] - runs[4][0]) / 8.0
    out["hmc"] = {"iterations_timed": [4, 12], "s": [runs[4][0], runs[12][0]],
                  "s_per_iteration": per_it, "grad_evals_per_s": (runs[12][1] - runs[4][1]) / (runs[12][0] - runs[4][0]),
                  "projected_s_for_300_plus_300": runs[4][0] + per_it * (n_it - 4),
                  "note": "warm-up iterations from prior draws; cost per iteration from the 12-4 difference"}
    # exact-photometry HMC (BF16): the cost of one round (a gradient of all
    # 2,000,000 chains and a leapfrog step) from runs of 1 and 3 rounds
    # (L = 1 and 3 in one iteration), projected with the mean L of the workload
    kx = dict(chains_per_gal=C, samples=False, mode="exact", prec="bf16", n_warm=1, n_samp=0)
    tr = {}
    for L in (1, 3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.hmc_run(x0, mobs, sigma, mask, L_min=L, L_max=L, **kx)
        e1.record()
        torch.cuda.synchronize()
        tr[L] = e0.elapsed_time(e1) / 1e3
    per_round = (tr[3] - tr[1]) / 2.0
    mean_L = 0.5 * (wl.extra["L_min"] + wl.extra["L_max"])
    out["hmc_exact_bf16"] = {"s_per_round": per_round, "grad_evals_per_s": G * C / per_round,
                             "projected_s_for_300_plus_300": per_round * mean_L * n_it,
                             "note": "rounds of 1 and 3 leapfrog steps timed; projected with the mean trajectory length"}
    ctx.close()
    return out


def run_reference(args):
    """The FP64 oracle timed on the host cores (rank 0 only)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    wl = _hmc_workload(0, n_gal=2)
    full = _hmc_workload(0)                  # the workload the sample stands for (its description only)
    from oracle import sps as O
    mobs = O.photometry(torch.as_tensor(wl.theta_true, dtype=torch.float64), wl.z, wl.tables,
                        "approx").numpy() + wl.noise
    steps = []
    for _ in range(args.warmup + args.steps):
        cb = _cpu_baseline(wl, mobs, 1.0, budget_s=max(2.0, 60.0 / (args.warmup + args.steps)))
        steps.append(cb)
    vals = [s["value"] for s in steps[args.warmup:]]
    v = float(np.mean(vals))
    cb = dict(steps[-1])
    cb["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(full.tables, full.n_gal, full.chains, full.extra["n_warm"], full.extra["n_samp"],
                             (full.extra["L_min"], full.extra["L_max"]), "hmc", False, ws),
           "note": "ESS fraction assumed 1 per galaxy (upper bound for the oracle)",
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def _parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-extra", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-nuts", action="store_true")
    ap.add_argument("--skip-models", action="store_true")
    ap.add_argument("--skip-errors", action="store_true")
    ap.add_argument("--skip-survey", action="store_true")
    ap.add_argument("--skip-exact-hmc", action="store_true")
    ap.add_argument("--plain-full", action="store_true",
                    help="run the whole lock-step baseline HMC (minutes) and report its own ESS")
    # profiling captures only (not bench values): smaller galaxy count / iterations
    ap.add_argument("--gal", type=int, default=None)
    ap.add_argument("--warm", type=int, default=None)
    ap.add_argument("--samp", type=int, default=None)
    ap.add_argument("--sampler", default="hmc", choices=["hmc", "nuts"],
                    help="sampler of the timed step (profiling captures; the bench line is HMC)")
    ap.add_argument("--mdf-age", action="store_true",
                    help="age-dependent MDF (row-evaluation kernel variant; profiling captures)")
    ap.add_argument("--survey", action="store_true",
                    help="throughput on the 1,000,000-galaxy survey batch (not the bench line)")
    ap.add_argument("--loglike-only", default=None,
                    help="comma list of mode_prec (e.g. exact_bf16,approx_fp32)")
    return ap


def _launch_ranks(args):
    """--gpus N outside a launcher: start N ranks of this script on this node
    with torch.distributed.run (one process per GPU, rendezvous on 127.0.0.1),
    as the launcher would, and return its exit status."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__),
           *sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    args = _parser().parse_args()
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus < 1:
        sys.exit("--gpus must be >= 1")
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        sys.exit(_launch_ranks(args))
    if "WORLD_SIZE" in os.environ and ws != args.gpus:
        sys.exit(f"--gpus {args.gpus} does not match the launcher's WORLD_SIZE {ws}")
    if args.warmup < 3:
        args.warmup = 3
    if args.warm is not None and args.samp is None:
        args.samp = args.warm
    if args.impl == "reference":
        run_reference(args)
    elif args.loglike_only:
        run_loglike_only(args)
    elif args.survey:
        run_survey(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
