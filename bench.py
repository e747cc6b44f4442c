"""Benchmark: assimilation cycles of the SCH particle filter on one GB300.

One step = one assimilation cycle over the whole ensemble: draw the window
noise, propagate every particle through the window (fused likelihood), then
adaptive tempering, systematic resampling and PCN jittering until the
temperature reaches one.  Default workload, the large run: n = 4096 cells,
K = 32 SALT modes (amplitude 0.05/j), N = 8192 particles, 10 steps per window,
128 observations (sigma 0.02), ESS threshold N/2, 10 jitter steps per stage,
rho = 0.9999, FP32 fields with FP64 weights (`--workload cfg2_f32`: n = 1024,
K = 8, N = 1024, M = 64, sigma = 0.05).  Synthetic twin experiment: the truth
starts from u0 = 0.2 sech(x-27) + 0.5 sech(x-13) and is propagated by the same
kernels.

Metric: particle-timesteps/s, counting every forward model step the cycle
executes (the first window plus every PCN re-run).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "cfg5_f32"
WORKLOADS = ["cfg5_f32", "cfg2_f32", "cfg2m_f32"]
METRIC = "particle-timesteps/s"
E2E_CYCLES, E2E_RUNS = 100, 3   # the end-to-end measurement: runs of cycles through the public API
# Algorithmic flops per node of the implicit-midpoint step, counted on the plain
# algorithm (each +, -, *, / is one flop).  Per Picard iteration:
#  linearly implicit (LI): dv 3, left operator 7, right-hand side 8, cyclic
#    variable tridiagonal solve 14 (Thomas 8 + Sherman-Morrison 6), Helmholtz 10
#    (mass product 4 + factored cyclic solve 6), convergence 2 -> 44;
#  explicit advection (EA): dv 3, mbar 2, advection 6, right-hand side 1,
#    factored cyclic solve of M + mu dt/2 K 6, Helmholtz 10, convergence 2 -> 30.
# Per step: noise synthesis 2K, and for EA the right operator (M - mu dt/2 K) m0 5.
FLOPS_PER_NODE_ITER = {"li": 44, "ea": 30}
FLOPS_PER_NODE_STEP_EXTRA = {"li": 0, "ea": 5}
# a warm-started step (the warp-group jitter with its workspace) first forms u = H^-1 M m of its
# guess: the mass right-hand side (3 flops a node) and the Helmholtz solve (9)
FLOPS_PER_NODE_WARM_START = 12


# Matern noise synthesis per node and step (Eq. noise_solve2, k solves): staging 3
# (dW + lambda dt, scale), load 1, per solve of the factored constant cyclic matrix
# 6, per later load the mass product 4 -> 4 + 6k + 4(k - 1).
def matern_flops_per_node(k):
    return 4 + 6 * k + 4 * (k - 1)


def step_flops(n, K, solver, iters, steps, noise_per_node=None):
    """Algorithmic flops of `steps` particle-steps that took `iters` Picard iterations in total.
    The noise costs 2K per node and step for the mode expansion, else noise_per_node."""
    noise = 2 * K if noise_per_node is None else noise_per_node
    return n * (FLOPS_PER_NODE_ITER[solver] * iters + (noise + FLOPS_PER_NODE_STEP_EXTRA[solver]) * steps)


# DRAM traffic of the dominant kernel (dram__bytes_read.sum + dram__bytes_write.sum
# per launch) from one ncu capture of the bench workload, keyed by the sha1 of the
# kernel's sources: a capture describes only the sources it was taken on, so the
# bench reports null once they change, until the kernel is captured again.
JITTER_SOURCES = ["paper_2402_06927_gb300/csrc/sch_warp.cuh", "paper_2402_06927_gb300/csrc/sch_kernels.cuh",
                  "paper_2402_06927_gb300/csrc/sch_internal.h", "paper_2402_06927_gb300/csrc/sch_device.cuh",
                  "paper_2402_06927_gb300/csrc/sch_window_warp.cu"]
# the large run's kernel (warp-group layout) also depends on these
GROUP_SOURCES = ["paper_2402_06927_gb300/csrc/sch_group.cuh", "paper_2402_06927_gb300/csrc/sch_window_group.cu"]
JITTER_TRAFFIC_BYTES = {"cfg2_f32": {
    # wjitter_kernel<8,2>, profiles/wjitter_kernel_cfg2_n1024_N1024.md: 4.611328 MB read, 0 written
    "569ce94c7b5361360ae675fc15d9adc45ab3190e": 4611328,
    # the same kernel after the Matern noise, MALA and Exp 1 additions to the shared headers:
    # 4.622592 MB read, 0 written
    "ecefad989d372e75eda023fb3639b7cbe1c64e76": 4622592,
    # with the FP32 Picard stop on the contraction estimate: 4.612352 MB read, 0 written
    "22baeb3a1bb63575765e2dcac5f140564fee8914": 4612352,
    # after the FP32 Box-Muller on the FP32 pipes and the Matern warp-layout split of wstep:
    # 4.611840 MB read, 0 written
    "fffa6c0bddf68b535b57adff1b518f66dc04a74e": 4611840,
    # with the Matern adjoint and nudging declarations in sch_internal.h: 4.611840 MB read, 0 written
    "a333a572af81817824d9debd3df0fe94d9cf5baa": 4611840,
    # wjitter_kernel<8,2,1,2>, specialised to a diagonal Picard and a PCR Helmholtz reduced
    # solve: 4.609792 MB read, 0 written
    "9a63bdc05dd81bd373a067cd982f7c3df6d28ae3": 4609792,
    # with the mode noise synthesised about each lane's centre: 4.606208 MB read, 0 written
    "89f00e16f90e5da10455045dc964eaeb5a808c25": 4606208,
    # the same kernel code with the warm-start pointer in the jitter arguments: 4.606976 MB read
    "a427e129ded961349af95ad6c01aef863a98e170": 4606976,
    # the same kernel code with the noise sums split into the table and finishing steps (the
    # warp-group kernels' polynomial form beside them): 4.607488 MB read, 0 written
    "c896a3cbb09194ec47c129fb655b2a831423f7b2": 4607488,
    # the same sources with one comment corrected (no code change): the capture above
    "0128ccf827d69e0960f91b1175216b6f6335b443": 4607488,
}, "cfg5_f32": {
    # gjitter_kernel<8,2,4,1>, profiles/gjitter_kernel_cfg5_n4096_N8192.md: 148.514304 MB read,
    # 226.438400 MB written
    "6fce80f5f13a05b4970ec3ed280a4c0d9d5f84c0": 374952704,
    # with the mode noise about each lane's centre and the cross-warp boundary sums spread over
    # the lanes: 146.914304 MB read, 224.452352 MB written
    "ca8b3fbf873a39287412fb86b247418fef952395": 371366656,
    # the same kernel code with the n = 1024 two-warp instantiation in the shared sources:
    # 146.407424 MB read, 223.907072 MB written
    "6d734c792c38fc1efbfce31cd3ea97b59f2aea75": 370314496,
    # proposals warm-started from the previous proposal's m (the guess cache written back to DRAM,
    # its reads mostly from L2): 3.053932032 GB read, 12.257600512 GB written
    "f8446f016778ac151f65880205d47b94f8188858": 15311532544,
    # with the guess read before the step's first barrier: 2.879922944 GB read, 12.160525824 GB written
    "8a9b29a4326730ba1429bc98e5937ed108b1c148": 15040448768,
    # with the lane-centred noise summed through host-fitted polynomials of the node offsets:
    # 2.718679552 GB read, 12.011711744 GB written
    "ec426efb5be03e8d31ac2ad15955f84c151614a3": 14730391296,
    # the same, with the coefficients in the warp-group arguments: 2.737210880 GB read,
    # 12.007459072 GB written
    "2232e9971dc678b5866299aa75c91b0b7672ad08": 14744669952,
    # the same sources with one comment corrected (no code change): the capture above
    "e4040ce2ae15928553e68f8ca69e7f19b0e8e742": 14744669952,
}}


def jitter_traffic(workload):
    """DRAM bytes per launch of the dominant kernel on `workload`, or None when the kernel's
    sources have changed since the capture (or the workload was never captured)."""
    import hashlib
    h = hashlib.sha1()
    try:
        for f in JITTER_SOURCES + (GROUP_SOURCES if workload == "cfg5_f32" else []):
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(hashlib.sha1(fh.read()).digest())
    except OSError:
        return None
    return JITTER_TRAFFIC_BYTES.get(workload, {}).get(h.hexdigest())


# The oracle solves every step by linearly implicit Picard iteration to 1e-13 (FP64); the GPU
# path solves the FP32 workloads by explicit-advection Picard to 1e-6.  The CPU baseline is
# therefore not like for like; its sample says so.
ORACLE_SOLVER_NOTE = ("; the oracle solves each step by linearly implicit Picard iteration to 1e-13 in FP64, "
                      "the GPU FP32 path by explicit-advection Picard to 1e-6")


def jitter_kernel_name(g, cfg, solver, warm=False):
    """The dominant (PCN jitter) kernel instantiation the filter launches."""
    matern = cfg.noise == "matern"
    if g.layout == "warp":
        return ("wmatern_jitter_kernel<8,2,DIAG,PCR,PCR> (one warp per particle, EA)" if matern
                else "wjitter_kernel<8,2,DIAG,PCR> (one warp per particle, EA)")
    if g.layout in ("group", "group16"):
        return (f"gjitter_kernel<{g.group_cs},2,{g.group_warps}> ({g.group_warps} warps per particle, EA"
                + (", proposals warm-started from the previous one)" if warm else ")"))
    return (f"matern_jitter_kernel<float,8,128,{solver.upper()}>" if matern
            else f"jitter_kernel<float,8,{cfg.n // 8},{solver.upper()}> (one CTA per particle)")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def sm_count() -> int:
    """Streaming multiprocessors of device 0 (queried; 152 on a GB300 when no device is visible)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(0).multi_processor_count)
    except Exception:
        pass
    return 152


def fp32_peak_tflops():
    """FP32 FMA pipe: SMs x 128 lanes x 2 flops x max SM clock."""
    mhz = _peaks().get("sm_max_mhz", 2070.0)
    return sm_count() * 128 * 2 * mhz * 1e6 / 1e12


def fp64_peak_tflops():
    """FP64 pipe: SMs x 2 DFMA lanes x 2 flops x max SM clock."""
    mhz = _peaks().get("sm_max_mhz", 2070.0)
    return sm_count() * 2 * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.proc = None
        self.path = None
        self.index = index

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    """(rank, world size) from the launcher's environment; with more than one rank, the
    process group for the timing's barrier and reductions (NCCL where CUDA is, else gloo)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, ws


def _all_reduce(v: float, ws: int, op: str) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def reduce_max(v: float, ws: int) -> float:
    return _all_reduce(v, ws, "max")


def reduce_sum(v: float, ws: int) -> float:
    return _all_reduce(v, ws, "sum")


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------- #
# CPU baseline: the FP64 oracle, as it stands, on a bounded sample
# ---------------------------------------------------------------------- #
def oracle_sample(cfg, budget_s: float = 12.0, min_particles: int = 1, first: int = 0, count: int = 64):
    """The oracle's window propagation (FP64, one thread) of particles first .. first+count-1
    of a seeded sample, for about budget_s seconds.  Returns (steps/s, description, seconds, steps)."""
    import numpy as np
    from oracle.model import Model
    from workloads import random_increments, random_state
    om = Model.from_config(cfg)
    u0 = random_state(cfg, first + count, 123)
    dW = random_increments(cfg, first + count, 124)
    t0 = time.perf_counter()
    done = 0
    while done < count and (done < min_particles or time.perf_counter() - t0 < budget_s):
        m0 = om.m_from_u(u0[first + done])
        om.window(m0, dW[first + done])
        done += 1
    el = time.perf_counter() - t0
    return done * cfg.Ns / el, (f"oracle window propagation (FP64, one thread) of {done} particles x {cfg.Ns} "
                                f"steps of the n={cfg.n} workload"), el, done * cfg.Ns


def _oracle_worker(job):
    name, budget_s, first, count = job
    from workloads import get_config
    _, _, el, steps = oracle_sample(get_config(name), budget_s=budget_s, min_particles=1, first=first, count=count)
    return steps, el


def oracle_parallel(name, budget_s: float = 10.0, per_core: int = 512):
    """The oracle on every host core: particles split across processes (started with spawn),
    as the paper splits its ensemble across ranks.  Returns (steps/s, cores, description)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    # one thread per process: the processes are the parallelism
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    jobs = [(name, budget_s, c * per_core, per_core) for c in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    steps = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    from workloads import get_config
    return steps / wall, cores, (f"oracle window propagation (FP64) on {cores} processes, particles split across "
                                 f"them, {steps} particle-steps of the n={get_config(name).n} workload in "
                                 f"{wall:.1f} s")


def workload_config(cfg, ws):
    """The keys of the bench line's `config` that name the workload (both arms)."""
    matern = cfg.noise == "matern"
    return {"workload": (f"{cfg.name}: SCH twin experiment n={cfg.n} "
                         + (f"Matern noise (kappa={cfg.kappa} eta={cfg.eta} k={cfg.matern_k}, "
                            f"{cfg.n} Brownian motions per step) " if matern else f"K={cfg.K} ")
                         + f"N={cfg.N} Ns={cfg.Ns} M={cfg.M} sigma={cfg.sigma} N*=N/2 "
                           f"jitter={cfg.n_jitter} rho={cfg.rho} "
                           f"({'FP32' if cfg.dtype == 'f32' else 'FP64'} fields, FP64 weights)"),
            "n": cfg.n, "N": cfg.N, "Ns": cfg.Ns, "K": cfg.K, "Q": cfg.Q, "M": cfg.M,
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}


def run_reference(args):
    """--impl reference: the oracle on the host cores, per step a bounded sample."""
    from workloads import get_config
    rank, ws = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    cfg = get_config(args.workload)
    for _ in range(args.warmup):
        oracle_sample(cfg, budget_s=0.0, min_particles=1)
    rates = []
    t_all = 0.0
    sample = ""
    cores = 1
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r, cores, sample = oracle_parallel(args.workload, budget_s=6.0)
        rates.append(r)
        t_all += time.perf_counter() - t0
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_all / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(cfg, ws),
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------- #
# GPU arm
# ---------------------------------------------------------------------- #
def run_ours(args):
    import torch
    from workloads import get_config, u0_profile
    from paper_2402_06927_gb300 import _lib
    from paper_2402_06927_gb300.api import SchModel
    from paper_2402_06927_gb300.filter import EnsembleFilter, KernelTimer

    rank, ws = dist_setup()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    cfg = get_config(args.workload)
    g = SchModel.from_config(cfg, layout=args.layout)
    N = cfg.N
    seed = 1000 + rank          # independent replicas on each rank
    total_cycles = args.warmup + args.steps
    dt = g.dtype
    # twin experiment: truth trajectory and observations, resident in HBM before timing
    u_truth = torch.as_tensor(u0_profile(cfg), dtype=dt, device="cuda")
    m_truth = g.m_from_u(u_truth[None].contiguous())
    ys, truths = [], []
    for c in range(total_cycles + 1):
        dWt = g.draw_increments(1, cfg.Ns, seed, _lib.TAG_TRUTH, c)
        out = g.ensemble_step(m_truth, dWt)
        m_truth = out["m"]
        truths.append(out["u"][0].clone())
        ys.append(g.synth_obs(out["u"][0].contiguous(), seed, c))
    f = EnsembleFilter(g, N, cfg.Ns, cfg.ess_min, cfg.rho, cfg.n_jitter, seed, eager_stages=args.eager_stages,
                       warm_jitter=not args.cold_jitter)
    m0, _ = g.prior_sample(N, u_truth, seed, cfg.prior_scale)
    f.set_state(m0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    diag_ws = torch.empty(cfg.n, dtype=torch.float64, device="cuda")
    diag_out = torch.empty(8, dtype=torch.float64, device="cuda")

    for c in range(args.warmup):
        f.cycle(ys[c], c)
        f.advance()
    torch.cuda.synchronize()
    m_warm = f.m_start.clone()   # the end-to-end runs restart from here, on the timed cycles
    barrier(ws)
    torch.cuda.synchronize()

    timer = KernelTimer()
    step_ms, fwd, launches, stages = [], 0, 0, []
    # clocks sampled from the first timed cycle to the end of the e2e runs
    clk = ClockSampler(local)
    clk.__enter__()
    for k in range(args.steps):
        c = args.warmup + k
        flush.fill_(float(k))                     # evict the ensemble from L2 (untimed)
        e0 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st = f.cycle(ys[c], c, timer=timer)
        f.advance()
        # device time of the cycle: from before its first launch to after its last one
        # (the filter records end_event after the cycle's last launch, before it waits)
        f.end_event.synchronize()
        step_ms.append(e0.elapsed_time(f.end_event))
        fwd += st.forward_steps
        launches += st.launches
        stages.append(len(st.stages))
    torch.cuda.synchronize()
    barrier(ws)
    dev_s = sum(step_ms) / 1000.0
    dev_s_max = reduce_max(dev_s, ws)
    fwd_all = reduce_sum(float(fwd), ws)
    value = fwd_all / dev_s_max

    # roofline of the dominant kernel (the fused PCN jitter kernel)
    jit_ms = timer.elapsed_ms()
    it_sum = sum(int(t.sum().item()) for t in timer.iters)
    n_launch = len(jit_ms)
    solver = "ea" if cfg.dtype == "f32" else "li"
    matern = cfg.noise == "matern"
    flops = step_flops(cfg.n, cfg.K, solver, it_sum, N * cfg.Ns * cfg.n_jitter * n_launch,
                       matern_flops_per_node(cfg.matern_k) if matern else None)
    # warm starts: every proposal after the first of a launch (the bench's windows all finish
    # cleanly) begins its steps with u = H^-1 M m of the guess
    warm_steps = N * cfg.Ns * (cfg.n_jitter - 1) * n_launch if f.warm_jitter else 0
    flops += cfg.n * FLOPS_PER_NODE_WARM_START * warm_steps
    # the guess cache a launch writes and reads back (m of every step, proposals 0 .. n-2 and 1 .. n-1)
    cache_bytes = 2 * N * cfg.Ns * (cfg.n_jitter - 1) * cfg.n * 4 if f.warm_jitter else 0
    jit_s = sum(jit_ms) / 1000.0
    # bytes a jitter launch must move: read m_start and dW, write dW, nll, logG and the
    # accepted end states (m_end, u_end); lower bound assumes the end states of each
    # particle are written once
    algo_bytes = N * (cfg.n * 4 + 2 * cfg.Ns * cfg.Q * 4 + 2 * 8 + 2 * cfg.n * 4)
    achieved = flops / jit_s / 1e12
    peak = fp32_peak_tflops()
    mean_iters = it_sum / (N * cfg.Ns * cfg.n_jitter * n_launch)

    # diagnostics of the last analysis
    g.diagnostics(f.u_end, truths[args.warmup + args.steps - 1], ws=diag_ws, out=diag_out)
    diag = diag_out[:4].cpu().tolist()

    # end to end through the public API with host buffers: observations H2D,
    # ensemble mean and diagnostics D2H, every step
    y_host = [y.cpu().pin_memory() for y in ys]
    mean_host = torch.empty(cfg.n, dtype=torch.float64).pin_memory()
    dg_host = torch.empty(8, dtype=torch.float64).pin_memory()
    y_dev = [torch.empty_like(ys[0]) for _ in range(2)]
    # E2E_RUNS runs of up to E2E_CYCLES cycles, the same cycles as the timed loop (from the
    # state after the warm-up cycles); the median run is reported (a host stall on a shared
    # machine moves a single short run by tens of percent), with every run's value beside it
    e2e_steps = min(args.steps, E2E_CYCLES if cfg.N * cfg.n <= (1 << 20) else E2E_CYCLES // 3)
    c0 = args.warmup
    e2e_runs = []
    for _ in range(E2E_RUNS):
        f2 = EnsembleFilter(g, N, cfg.Ns, cfg.ess_min, cfg.rho, cfg.n_jitter, seed, eager_stages=args.eager_stages,
                            warm_jitter=not args.cold_jitter)
        f2.set_state(m_warm)
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        fwd2 = 0
        y_dev[0].copy_(y_host[c0], non_blocking=True)
        for k in range(e2e_steps):
            c = c0 + k
            def post(k=k, c=c, f2=f2):
                # enqueued by the cycle before it waits for its stages: diagnostics of the analysis,
                # their copy to the host, and the next step's observations to the device
                g.diagnostics(f2.u_end, truths[c], ws=diag_ws, out=diag_out)
                mean_host.copy_(diag_ws, non_blocking=True)
                dg_host.copy_(diag_out, non_blocking=True)
                if k + 1 < e2e_steps:
                    y_dev[(k + 1) % 2].copy_(y_host[c + 1], non_blocking=True)
            st = f2.cycle(y_dev[k % 2], c, post=post)   # returns once its stages and post's work are done
            f2.advance()
            fwd2 += st.forward_steps
        e2e_s = reduce_max(time.perf_counter() - t0, ws)
        e2e_runs.append(reduce_sum(float(fwd2), ws) / e2e_s)
    e2e_val = statistics.median(e2e_runs)
    clk.__exit__(None, None, None)
    clocks = clk.summary()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        v1, sample1, _, _ = oracle_sample(cfg, budget_s=8.0)
        v, cores, sample = oracle_parallel(args.workload, budget_s=8.0)
        cpu = {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
               "sample": sample + ORACLE_SOLVER_NOTE,
               "single_core": {"value": v1, "sample": sample1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * dev_s_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": cfg.dtype, "data": "synthetic",
            "config": {**workload_config(cfg, ws), "layout": g.layout, "noise_form": g.noise_form,
                       "jitter_picard_start": ("the previous proposal's per-step states" if f.warm_jitter
                                               else "each step's start state"),
                       "l2": "flushed between timed steps (256 MB write)",
                       "cycles_per_s": args.steps * ws / dev_s_max,
                       "mean_tempering_stages": statistics.mean(stages),
                       "mean_picard_iters_per_step": mean_iters, "picard_solver": solver,
                       "analysis_emre_rb_res_rmse": diag},
            "roofline": {"bound": "alu", "kernel": jitter_kernel_name(g, cfg, solver, f.warm_jitter),
                         "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": jitter_traffic(args.workload),
                         "algorithmic_bytes_per_launch": algo_bytes,
                         "warm_start_cache_bytes_per_launch": cache_bytes,
                         "peak_note": f"FP32 FMA pipe {sm_count()} SMs x 128 lanes x 2 x max SM clock"},
            "gpu_launches": launches,
            "e2e": {"value": e2e_val, "unit": METRIC, "runs": e2e_runs, "cycles_per_run": e2e_steps,
                    "h2d_bytes_per_step": cfg.M * 4,
                    "d2h_bytes_per_step": cfg.n * 8 + 64},
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_nudging(args):
    """--nudging: learned vs optimiser nudging (learned-proposal workload cfg4_f32 by default:
    n = 1024, K = 16 modes, 20-step windows, N = 1024, M = 64, sigma = 0.05; or
    --nudging-workload cfg5_f32, the large run: n = 4096, K = 32, Ns = 10, N = 8192, M = 128,
    sigma = 0.02), FP32 fields, the network in BF16 with FP32 accumulation.

    Training pairs: pf_nudge (open loop, L-BFGS to max|grad| <= 1e-6) on `--train-cycles`
    cycles of a twin experiment x min(N, 1024) particles (every N/1024-th); the network is trained with its own GPU
    kernels.  Then `--twins` fresh twin experiments are assimilated `--steps` cycles each with
    learned nudging backed by the optimiser (pf_nudge for any cycle whose forecast ESS under
    the network's drift is below N/4: the product path), the network alone, optimiser
    nudging, the hybrid (the network's drift refined by one L-BFGS iteration) and no nudging
    (tempering + jitter steps each).  Reported per source: cycles/s, analysis RMSE and
    forecast ESS as mean and spread over the twins, fallback cycles, and the paired
    learned/optimiser RMSE ratios."""
    import math
    import torch
    from workloads import get_config, u0_profile
    from paper_2402_06927_gb300.api import ProposalNet, SchModel
    from paper_2402_06927_gb300 import proposal as PR

    torch.cuda.set_device(0)
    cfg = get_config(args.nudging_workload)
    g = SchModel.from_config(cfg)
    u0 = torch.tensor(u0_profile(cfg), dtype=torch.float32, device="cuda")
    # at most 1024 particles nudged per cycle: N = 8192 spreads its pairs over eight times the cycles
    keep = min(cfg.N, 1024)
    U, Y, T, gst = PR.generate_pairs(g, cfg.N, cfg.Ns, args.train_cycles, 7, u0, cfg.ess_min, cfg.rho,
                                     cfg.n_jitter, cfg.prior_scale, max_iter=60, gtol=1e-6, keep=keep)
    net = ProposalNet(cfg.n, cfg.K, cfg.Ns, cfg.M, cfg.sigma, C=64, seed=1, precision="bf16")
    tst = PR.train(net, U, Y, T, epochs=args.epochs, batch=256, lr=1e-3)
    sources = ("learned_fb", "learned", "hybrid", "optimiser", "none")
    runs = {src: [] for src in sources}
    for t in range(args.twins):
        tseed = 99 + 17 * t
        twin = PR.make_twin(g, cfg.Ns, args.steps, tseed, u0)
        for src in sources:
            runs[src].append(PR.run_nudged(g, src, net, cfg.N, cfg.Ns, args.steps, tseed, u0, cfg.ess_min, cfg.rho,
                                           cfg.n_jitter, cfg.prior_scale, twin, max_iter=60, gtol=1e-6, refine=1))

    def stats(vals):
        m = sum(vals) / len(vals)
        sd = math.sqrt(sum((v - m) ** 2 for v in vals) / max(1, len(vals) - 1))
        return {"mean": m, "sd": sd, "values": vals}

    res = {src: {k: stats([r[k] for r in runs[src]])
                 for k in ("cycles_per_s", "rmse", "mean_forecast_ess", "fallback_cycles")} for src in sources}
    ratios = [a["rmse"] / b["rmse"] for a, b in zip(runs["learned_fb"], runs["optimiser"])]
    line = {
        "metric": "assim. cycles/s (learned nudging with optimiser fallback)",
        "value": res["learned_fb"]["cycles_per_s"]["mean"], "unit": "cycles/s",
        "n_gpus": 1, "steps": args.steps, "warmup": 0, "higher_is_better": True, "dtype": "f32 fields, bf16 network",
        "data": "synthetic",
        "config": {"workload": f"{cfg.name}: SCH twin experiment n={cfg.n} K={cfg.K} Ns={cfg.Ns} N={cfg.N} "
                               f"M={cfg.M} sigma={cfg.sigma}, learned vs optimiser nudging + tempering + "
                               f"{cfg.n_jitter} jitter steps, {args.twins} twins x {args.steps} cycles",
                   "train_pairs": int(U.shape[0]), "generation": gst, "training": tst},
        "comparison": res,
        "paired_rmse_ratio_learned_fb_over_optimiser": stats(ratios),
    }
    print(json.dumps(line))
    return 0


# Algorithmic flops per node of the reverse-mode adjoint of one converged step
# (the transpose of the linearised Eq. fde1 solved by a fixed point):
# per adjoint iteration: right-hand side 1, variable cyclic tridiagonal solve 14,
# B^T psi 4, Helmholtz solve 6 and mass product 4 of the correction, its scaling 1,
# convergence 2 -> 32; per step: dv 3, mbar 2, its edge sums 1, the transposed
# rows 4, dJ/dm of the previous state 6, and the projection on the K modes 2K.
ADJ_FLOPS_PER_NODE_ITER = 32
ADJ_FLOPS_PER_NODE_STEP = 16


def _nudging_inputs(g, cfg):
    """Twin inputs of the nudging workload: the truth runs one window from u0, the
    particles start from the prior around u0 with prior noise and a random drift."""
    import torch
    from workloads import u0_profile, random_drift
    N, Ns = cfg.N, cfg.Ns
    u0 = torch.tensor(u0_profile(cfg), dtype=g.dtype, device="cuda")
    mt = g.m_from_u(u0[None].contiguous())
    tr = g.ensemble_step(mt, g.draw_increments(1, Ns, 21, 5, 0), None)
    y = g.synth_obs(tr["u"][0].contiguous(), 22, 1)
    m0, _ = g.prior_sample(N, u0, 23, cfg.prior_scale)
    dW = g.draw_increments(N, Ns, 24, 1, 0)
    lam = torch.tensor(random_drift(cfg, N, 25, steps=Ns, scale=0.2), dtype=g.dtype, device="cuda")
    return m0, dW, lam, y


def _adjoint_flops(n, K, N, Ns, it_fwd, it_adj, matern_k=None, solver="li"):
    """Algorithmic flops of an adjoint window call.  The forward window is credited with
    the Picard solver's count (LI for FP64, EA for FP32).  The noise (and its transpose in
    the reverse sweep) costs 2K per node and step for the mode expansion; with the Matern
    noise the forward noise is matern_flops_per_node(k) and the transposed map the same
    count again (k solves, k - 1 mass products, the B^T stencil)."""
    if matern_k is None:
        return (step_flops(n, K, solver, it_fwd, N * Ns)
                + n * (ADJ_FLOPS_PER_NODE_ITER * it_adj + (ADJ_FLOPS_PER_NODE_STEP + 2 * K) * N * Ns))
    mf = matern_flops_per_node(matern_k)
    return (step_flops(n, K, solver, it_fwd, N * Ns, mf)
            + n * (ADJ_FLOPS_PER_NODE_ITER * it_adj + (ADJ_FLOPS_PER_NODE_STEP + 2 * mf) * N * Ns))


def _nudging_config(args, name):
    """The nudging workload, on FP32 fields (EA Picard, tolerance 1e-6) with --f32."""
    from workloads import get_config
    return get_config(name, dtype="f32", tol=1e-6, max_iter=40) if args.f32 else get_config(name)


def _precision(args):
    """(dtype, solver label, adjoint kernel instantiation, roofline peak, peak note)"""
    if args.f32:
        return ("f32", "EA", "float,8,128,EA", fp32_peak_tflops(),
                f"FP32 FMA pipe {sm_count()} SMs x 128 lanes x 2 x max SM clock")
    return ("f64", "LI", "double,4,256,LI", fp64_peak_tflops(),
            f"FP64 pipe {sm_count()} SMs x 2 DFMA lanes x 2 x max SM clock")


def _ckpt_note(ckpt):
    return "every state kept, nothing recomputed" if ckpt is None else f"checkpoints every {ckpt} steps"


def run_adjoint(args):
    """--adjoint: gradient evaluations on the nudging workload (n = 1024, K = 8,
    20-step windows, N = 256, FP64; every state of the window kept from the forward
    pass, or checkpoints every --ckpt steps).  One evaluation is
    sch_adjoint_window on one particle: the forward window and its reverse-mode
    adjoint, J and dJ/dlambda, dJ/ddW, dJ/dm0.  Inputs resident, L2 flushed
    between timed calls, CUDA events; the oracle's gradient (tangent linear,
    dense Jacobians) is timed on the host beside it."""
    import torch
    from workloads import get_config
    from paper_2402_06927_gb300.api import SchModel
    torch.cuda.set_device(0)
    cfg = _nudging_config(args, "cfg3m_f64" if args.matern else "cfg3_f64")
    dtype, slabel, kinst, peak, pnote = _precision(args)
    g = SchModel.from_config(cfg)
    N, Ns, K, n = cfg.N, cfg.Ns, cfg.K, cfg.n
    m0, dW, lam, y = _nudging_inputs(g, cfg)
    fwd = g.ensemble_step(m0, dW, lam, y)
    ws = None
    for _ in range(max(3, args.warmup)):
        out = g.adjoint_window(m0, dW, lam, y, ckpt=args.ckpt)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    times = []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        out = g.adjoint_window(m0, dW, lam, y, ckpt=args.ckpt)
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.median(times)
    assert int(out["status"].abs().sum().item()) == 0, "adjoint status flags"
    it_fwd = int(fwd["iters"].sum().item())
    it_adj = int(out["iters"].sum().item()) - it_fwd
    achieved = _adjoint_flops(n, K, N, Ns, it_fwd, it_adj, cfg.matern_k if args.matern else None,
                              slabel.lower()) / t / 1e12
    cpu = None
    if not args.no_cpu:
        import numpy as np
        from oracle.model import Model
        from oracle import nudge as ON
        om = Model.from_config(cfg)
        m0h, dWh, lamh, yh = (x.double().cpu().numpy() for x in (m0[:4], dW[:4], lam[:4], y))
        t0 = time.perf_counter()
        done = 0
        while done < 4 and (done < 1 or time.perf_counter() - t0 < 20.0):
            ON.cost_and_gradient(om, m0h[done], dWh[done], lamh[done], yh, cfg.sigma)
            done += 1
        el = time.perf_counter() - t0
        # the Matern gradient has Ns n directions: numpy's BLAS runs its dense solves on every core
        cores = (os.cpu_count() or 1) if args.matern else 1
        cpu = {"value": done / el, "unit": "gradient evaluations/s", "cores": cores, "kind": "oracle",
               "sample": f"oracle J and dJ/dlambda by tangent linearisation (dense Jacobians, FP64"
                         f"{', BLAS threads on every core' if args.matern else ', one thread'}) "
                         f"for {done} particles of the same inputs"}
    line = {
        "metric": "gradient evaluations/s", "value": N / t, "unit": "gradient evaluations/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": 1e3 * t, "higher_is_better": True,
        "dtype": dtype, "data": "synthetic",
        "config": {"workload": "adjoint window: n=1024 " + (f"Matern noise (kappa={cfg.kappa} eta={cfg.eta} "
                                                            f"k={cfg.matern_k}) " if args.matern else "K=8 ")
                               + f"Ns=20 N=256 ({dtype.upper()}, {slabel} Picard, {_ckpt_note(args.ckpt)})",
                   "l2": "flushed between timed calls (256 MB write)",
                   "forward_picard_iters_per_step": it_fwd / (N * Ns), "adjoint_iters_per_step": it_adj / (N * Ns)},
        "roofline": {"bound": "alu",
                     "kernel": f"adjoint_kernel<{kinst}" + (",MATERN>" if args.matern else ">"),
                     "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None,
                     "peak_note": pnote + "; recomputation from checkpoints is not credited"},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    return 0


MALA_THETA, MALA_H, MALA_ITERS = 1.0, 0.5, 10


def run_mala(args):
    """--mala: MALA jitter on the nudging workload (n = 1024, K = 8, 20-step windows,
    N = 256, FP64, the adjoint keeping every state, or checkpoints every --ckpt steps) at theta = 1.  One timed step is one
    SchModel.mala_jitter call of MALA_ITERS moves per particle: the initial gradient,
    then per move pf_mala_propose, the adjoint window at the proposal and
    pf_mala_accept, and the final window.  Inputs resident, L2 flushed before each
    call, CUDA events.  The adjoint kernel dominates; its roofline is reported with
    its share of the call, and the oracle's MALA move is timed on the host."""
    import torch
    from workloads import get_config
    from paper_2402_06927_gb300.api import SchModel
    torch.cuda.set_device(0)
    cfg = _nudging_config(args, "cfg3_f64")
    dtype, slabel, kinst, peak, pnote = _precision(args)
    g = SchModel.from_config(cfg)
    N, Ns, K, n = cfg.N, cfg.Ns, cfg.K, cfg.n
    m0, dW0, lam, y = _nudging_inputs(g, cfg)
    dW = dW0.clone()
    S, theta, h = MALA_ITERS, MALA_THETA, (MALA_H if args.mala_h is None else args.mala_h)

    def call(k):
        return g.mala_jitter(m0, dW, lam, y, theta, h, S, 31, 1000 * k, ckpt=args.ckpt)

    for k in range(max(3, args.warmup)):
        dW.copy_(dW0)
        out = call(k)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    times, acc = [], 0
    for k in range(args.steps):
        dW.copy_(dW0)
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        out = call(100 + k)
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        acc += int(out["accepts"].sum().item())
    t = statistics.median(times)
    assert int(out["status"].abs().sum().item()) == 0, "window status flags"
    # parts: the adjoint window (dominant), proposal and decision kernels, each alone
    ws = torch.empty(int(g.adjoint_workspace_bytes(N, Ns, args.ckpt)), dtype=torch.uint8, device="cuda")
    fwd = g.ensemble_step(m0, dW0, lam, y)
    adj = g.adjoint_window(m0, dW0, lam, y, ckpt=args.ckpt, want_m0=False, ws=ws)
    t_adj = _event_time(lambda: g.adjoint_window(m0, dW0, lam, y, ckpt=args.ckpt, want_m0=False, ws=ws), 5,
                        flush)
    dWp, Jp, gJp = torch.empty_like(dW0), adj["J"].clone(), adj["g_dW"].clone()
    J, gJ, dWc = adj["J"].clone(), adj["g_dW"].clone(), dW0.clone()
    t_prop = _event_time(lambda: g.mala_propose(dWc, lam, gJ, dWp, theta, h, 31, 0), 20, flush)
    t_acc = _event_time(lambda: g.mala_accept(dWc, dWp, lam, J, Jp, gJ, gJp, None, theta, h, 31, 0), 20, flush)
    it_fwd = int(fwd["iters"].sum().item())
    it_adj = int(adj["iters"].sum().item()) - it_fwd
    achieved = _adjoint_flops(n, K, N, Ns, it_fwd, it_adj, solver=slabel.lower()) / t_adj / 1e12
    cpu = None
    if not args.no_cpu:
        from oracle.model import Model
        from oracle import filter as OF
        from workloads import mode_amplitudes
        om = Model(L=cfg.L, n=n, alpha=cfg.alpha, mu=cfg.mu, dt=cfg.dt, amps=mode_amplitudes(cfg))
        m0h, dWh, lamh, yh = (x.double().cpu().numpy() for x in (m0[:1], dW0[:1], lam[:1], y))
        t0 = time.perf_counter()
        OF.mala_jitter(om, m0h, dWh, lamh, yh, cfg.sigma, theta, h, 1, 31, 0)
        el = time.perf_counter() - t0
        cpu = {"value": 1.0 / el, "unit": "MALA moves/s", "cores": 1, "kind": "oracle",
               "sample": "one oracle MALA move of one particle (tangent-linear gradients, FP64, one thread) "
                         "and its final window, same inputs"}
    line = {
        "metric": "MALA moves/s", "value": N * S / t, "unit": "MALA moves/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": 1e3 * t, "higher_is_better": True,
        "dtype": dtype, "data": "synthetic",
        "config": {"workload": f"MALA jitter: n=1024 K=8 Ns=20 N=256 ({dtype.upper()}, {slabel} Picard, "
                               f"{_ckpt_note(args.ckpt)}), "
                               f"{S} moves per call, theta={theta}, h={h}",
                   "l2": "flushed between timed calls (256 MB write)",
                   "acceptance": acc / (N * S * args.steps),
                   "adjoint_ms": 1e3 * t_adj, "propose_us": 1e6 * t_prop, "accept_us": 1e6 * t_acc,
                   "adjoint_share": (S + 1) * t_adj / t},
        "roofline": {"bound": "alu", "kernel": f"adjoint_kernel<{kinst}>", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None,
                     "peak_note": pnote + "; recomputation from checkpoints is not credited"},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    return 0


def run_exp1(args):
    """--exp1: Exp 1 of Sec. 4.1 on the exp1_f64 workload (N = 150, Matern noise with eta = 1,
    k = 3, observations every 5 steps at 64 of 128 nodes).  The truth and the particles start
    from the Exp 1 initial ensemble (Eq. init_solve).  Two filters assimilate the same
    observations: the bootstrap filter (each step one tempering stage with the whole step,
    resampling, no jittering) and the filter with adaptive tempering (ESS >= N/2) and 5 PCN
    jittering steps (delta = 0.15) per stage.  EMRE, RB and RES of the analysis ensemble
    against the truth are taken every step; the line reports them at steps 1, 100, 500 and 1000
    and their means over the last 100 steps."""
    import torch
    from workloads import get_config
    from paper_2402_06927_gb300.api import SchModel
    from paper_2402_06927_gb300 import twin
    torch.cuda.set_device(0)
    cfg = get_config("exp1_f64")
    if args.exp1_sigma is not None:
        cfg = cfg.replace(sigma=args.exp1_sigma)
    g = SchModel.from_config(cfg)
    T = args.da_steps
    out = twin.exp2(g, cfg, T) if args.exp2 else twin.exp1(g, cfg, T)
    res = {}
    for name in ("bootstrap", "tempering_jittering"):
        sr = out[name]["series"]
        hv = out[name]["halves"]
        res[name] = {
            "assimilation_steps_per_s": T / out[name]["seconds"],
            "mean_tempering_stages": statistics.mean(out[name]["stages"]),
            "emre_rb_res_at": {str(k): sr[k - 1].tolist() for k in (1, 100, 500, 1000) if k <= T},
            "emre_rb_res_mean_last_100": sr[max(0, T - 100):].mean(axis=0).tolist(),
            "mean_error_first_second_half_last_100": hv[max(0, T - 100):].mean(axis=0).tolist(),
        }
    line = {"metric": "assimilation steps/s", "value": res["tempering_jittering"]["assimilation_steps_per_s"],
            "unit": "assimilation steps/s", "n_gpus": 1, "steps": T, "warmup": 0, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": ("Exp 2 (only [0, L/2] observed)" if args.exp2 else "Exp 1")
                                   + f": exp1_f64 (N={cfg.N}, n={cfg.n}, Matern eta={cfg.eta} k={cfg.matern_k} "
                                   f"kappa={cfg.kappa}, Ns={cfg.Ns}, M={cfg.M}, sigma={cfg.sigma:.4g}, delta=0.15, "
                                   f"{cfg.n_jitter} jitter steps per stage), {T} assimilation steps",
                       "initial_emre_rb_res": out["initial"].tolist()},
            "filters": res}
    print(json.dumps(line))
    return 0


def _event_time(fn, reps, flush=None):
    """Median device time of fn() over reps calls (CUDA events; L2 flushed before each if given)."""
    import torch
    st = torch.cuda.current_stream()
    ts = []
    for k in range(reps):
        if flush is not None:
            flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return statistics.median(ts)


def _host_time(fn, budget_s=3.0, min_reps=1):
    t0 = time.perf_counter()
    reps = 0
    while reps < min_reps or time.perf_counter() - t0 < budget_s:
        fn()
        reps += 1
    return (time.perf_counter() - t0) / reps


def run_filter_kernels(args):
    """--filter-kernels: the filter steps between the model runs, at the bench ensemble
    size (N = 1024) and the large one (N = 8192, n = 4096): adaptive tempering (a search
    and a whole-step call), systematic resampling, and the row gather that copies the
    resampled particles (HBM-bound, against the measured copy bandwidth).  Device times
    by CUDA events (median, L2 flushed before each call); the oracle's steps timed on one
    host core beside them."""
    import numpy as np
    import torch
    from oracle import filter as OF
    from workloads import random_logweights
    from paper_2402_06927_gb300 import api
    torch.cuda.set_device(0)
    hbm = _peaks().get("hbm_gbs", 6800.0)   # measured copy bandwidth, else the earlier GB300 measurement
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    reps = max(5, args.steps)
    out = []
    for N, n in ((1024, 1024), (8192, 4096)):
        for label, spread in (("search", 40.0), ("whole step", 0.002)):
            phi = random_logweights(N, N + 1, spread)
            nll = torch.tensor(phi, dtype=torch.float64, device="cuda")
            wbar, res = api.pf_temper(nll, None, 0.0, 0.5 * N)
            t = _event_time(lambda: api.pf_temper(nll, None, 0.0, 0.5 * N, wbar, res), reps, flush)
            th = _host_time(lambda: OF.temper(phi, 0.0, 0.5 * N), 2.0)
            out.append({"step": f"temper ({label})", "N": N, "device_us": 1e6 * t, "oracle_us": 1e6 * th,
                        "dtheta": float(res[0].item()), "bound": "FP64 exp and cluster-barrier latency"})
        wb = wbar.double()
        idx = torch.empty(N, dtype=torch.int32, device="cuda")
        t = _event_time(lambda: api.pf_resample(wb, 7, 3, idx=idx), reps, flush)
        wh = wb.cpu().numpy()
        u53 = OF.resample_offset(7, 3)
        th = _host_time(lambda: OF.systematic_resample(wh, u53), 2.0)
        out.append({"step": "systematic resampling (indices)", "N": N, "device_us": 1e6 * t, "oracle_us": 1e6 * th,
                    "bound": "latency (one CTA: integer scan and N searches)"})
        src = torch.randn(N, n, device="cuda")
        dst = torch.empty_like(src)
        t = _event_time(lambda: api.pf_gather_rows(idx, src, dst), reps, flush)
        nbytes = 2 * N * n * 4
        srch = src.cpu().numpy()
        ih = idx.cpu().numpy()
        th = _host_time(lambda: srch[ih], 2.0)
        out.append({"step": "row gather (m rows)", "N": N, "row_bytes": n * 4, "device_us": 1e6 * t,
                    "oracle_us": 1e6 * th, "bound": "hbm", "achieved_gbs": nbytes / t / 1e9, "peak_gbs": hbm,
                    "frac": nbytes / t / 1e9 / hbm})
    print(json.dumps({"filter_kernels": out, "peak_note": "peak_gbs: measured copy bandwidth (MEASURED_PEAKS.json)",
                      "oracle_cores": 1}))
    return 0


def run_proposal(args):
    """--proposal: the learned proposal network at the learned-proposal workload's size
    (n = 1024, K = 16, Ns = 20, M = 64, 64 channels) on a batch of B = 8192 particles
    (--proposal-batch):
    nn_forward, nn_backward (loss and all gradients) and nn_adam_step, with BF16
    operands and FP32 accumulation on the tensor cores (the product path) and with FP32
    operands on the CUDA cores (the check path).  Algorithmic flops are the
    multiply-adds of the convolutions, the Fourier-mode projection and the head (2 per
    multiply-add).  The FP64 oracle network is timed on one host core beside them."""
    import numpy as np
    import torch
    from workloads import get_config
    from oracle import convnet as OC
    from paper_2402_06927_gb300.api import ProposalNet
    torch.cuda.set_device(0)
    cfg = get_config("cfg4_f32")
    n, K, Ns, M, C, B = cfg.n, cfg.K, cfg.Ns, cfg.M, 64, args.proposal_batch
    net = ProposalNet(n, K, Ns, M, cfg.sigma, C=C, seed=1)
    g = torch.Generator(device="cpu").manual_seed(5)
    u = (0.3 * torch.randn(B, n, generator=g)).cuda()
    y = (0.3 * torch.randn(M, generator=g)).cuda()
    tgt = (0.1 * torch.randn(B, Ns, K, generator=g)).cuda()
    P = n // 16
    conv = sum(2 * (n >> (l + 1)) * C * (2 if l == 0 else C) * 5 for l in range(4))
    fwd = B * (conv + 2 * C * P * K + 2 * (C * K) * (K * Ns))
    # backward: dW of every layer, dX of layers 2..4, the mode projection and the head twice
    conv_dx = sum(2 * (n >> (l + 1)) * C * C * 5 for l in range(1, 4))
    bwd = B * (conv + conv_dx + 2 * C * P * K + 2 * 2 * (C * K) * (K * Ns))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    reps = max(5, args.steps)
    res = {}
    for prec in ("bf16", "fp32"):
        net.set_precision(prec)
        for _ in range(3):
            net.forward(u, y)
            net.loss_and_grad(u, y, tgt)
        tf = _event_time(lambda: net.forward(u, y), reps, flush)
        tb = _event_time(lambda: net.loss_and_grad(u, y, tgt), reps, flush)
        _, gr = net.loss_and_grad(u, y, tgt)
        ta = _event_time(lambda: net.adam_step(gr), reps, flush)
        res[prec] = (tf, tb, ta)
    bf_peak = _peaks().get("bf16_tflops", 1922.7)
    f32_peak = fp32_peak_tflops()
    p_np = OC.init_params(C, K, Ns, n, 1)
    x0 = OC.features(u[:4].double().cpu().numpy(), y.double().cpu().numpy(), cfg.sigma)
    tho_f = _host_time(lambda: OC.forward(p_np, x0, K, Ns), 2.0) / 4
    tho_b = _host_time(lambda: OC.loss_and_grad(p_np, x0, tgt[:4].double().cpu().numpy(), K, Ns), 2.0) / 4
    tf, tb, ta = res["bf16"]
    tf32, tb32, ta32 = res["fp32"]
    line = {
        "metric": "network samples/s (forward)", "value": B / tf, "unit": "samples/s", "n_gpus": 1, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": f"learned proposal: n={n} K={K} Ns={Ns} M={M} C={C}, batch {B}",
                   "l2": "flushed before each timed call (256 MB write)"},
        "forward": {"ms": 1e3 * tf, "tflops": fwd / tf / 1e12, "frac": fwd / tf / 1e12 / bf_peak},
        "backward": {"ms": 1e3 * tb, "tflops": bwd / tb / 1e12, "frac": bwd / tb / 1e12 / bf_peak},
        "adam_ms": 1e3 * ta,
        "fp32_check_path": {"forward_ms": 1e3 * tf32, "backward_ms": 1e3 * tb32,
                            "forward_tflops": fwd / tf32 / 1e12, "forward_frac_of_fp32_peak": fwd / tf32 / 1e12 / f32_peak},
        "roofline": {"bound": "tensor", "kernel": "hgemm_kernel (nn_forward, BF16 mma.sync m16n8k16, FP32 accumulation)",
                     "achieved": fwd / tf / 1e12, "peak": bf_peak, "unit": "TFLOP/s", "frac": fwd / tf / 1e12 / bf_peak,
                     "traffic": None, "peak_note": "measured cuBLAS BF16 burst (MEASURED_PEAKS.json bf16_tflops)"},
        "cpu_baseline": {"value": 1.0 / tho_f, "unit": "samples/s", "cores": 1, "kind": "oracle",
                         "sample": "FP64 oracle network forward on 4 samples (one thread); backward "
                                   f"{1.0 / tho_b:.1f} samples/s"},
    }
    print(json.dumps(line))
    return 0


def run_occupancy(args):
    """--occupancy: one jitter launch of the bench workload (10 PCN proposals of a
    10-step window, n = 1024, K = 8, FP32) at N = 1 .. 16 particles per SM (152 .. 2432 on
    a GB300), i.e. 1 .. 16 warps per SM in the warp layout; best of --steps timed launches
    (CUDA events) each."""
    import torch
    from workloads import get_config, u0_profile
    from paper_2402_06927_gb300.api import SchModel
    torch.cuda.set_device(0)
    cfg = get_config("cfg2_f32")
    g = SchModel.from_config(cfg)
    u0 = torch.tensor(u0_profile(cfg), dtype=torch.float32, device="cuda")
    y = g.synth_obs(u0, 1, 1)
    rows = []
    sms = sm_count()
    for per_sm in (1, 2, 4, 6, 8, 12, 16):
        N = per_sm * sms
        m0, _ = g.prior_sample(N, u0, 3, cfg.prior_scale)
        dW = g.draw_increments(N, cfg.Ns, 5, 1, 0)
        st = g.ensemble_step(m0, dW, None, y)
        nll, logG = st["nll"].clone(), st["logG"].clone()
        ms = []
        for rep in range(max(2, args.steps) + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, it, _ = g.jitter(m0, dW, None, y, nll, logG, st["m"], st["u"], 0.5, cfg.rho, 10, 9, rep * 10,
                                want_iters=True)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        rows.append({"N": N, "warps_per_sm": N / sms, "ms_per_launch": min(ms[1:]),
                     "picard_iters_per_step": it.float().mean().item() / (10 * cfg.Ns)})
    print(json.dumps({"occupancy_sweep": rows, "kernel": f"wjitter ({g.layout} layout)"}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cold-jitter", action="store_true",
                    help="start every PCN proposal's Picard iterations from the steps' start states "
                         "(no warm start from the previous proposal in the warp-group layout)")
    ap.add_argument("--eager-stages", type=int, default=2,
                    help="tempering stages enqueued at once as device-gated stages (0: stage by stage)")
    ap.add_argument("--nudging", action="store_true",
                    help="learned vs optimiser nudging comparison instead of the default workload")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the reverse-mode adjoint (gradient evaluations) on the nudging workload")
    ap.add_argument("--workload", default=WORKLOAD, choices=WORKLOADS,
                    help="filter workload of the main run: cfg5_f32 (the large run, the headline), "
                         "cfg2_f32 (ensemble scale) or cfg2m_f32 (cfg2 with the paper's Matern noise)")
    ap.add_argument("--mala-h", type=float, default=None, help="MALA step size h (--mala)")
    ap.add_argument("--layout", default="auto", choices=["auto", "warp", "group", "group16", "cta"],
                    help="kernel layout of the filter's propagation (FP32 EA: one warp per particle, several "
                         "warps per particle with 32 or 16 nodes a lane, or one CTA per particle)")
    ap.add_argument("--matern", action="store_true", help="--adjoint on the Matern noise (cfg3m_f64)")
    ap.add_argument("--f32", action="store_true",
                    help="--adjoint, --mala: the nudging workload on FP32 fields (EA Picard)")
    ap.add_argument("--ckpt", type=int, default=None,
                    help="--adjoint, --mala: checkpoint interval of the adjoint (default: keep every state)")
    ap.add_argument("--exp1", action="store_true",
                    help="Exp 1: bootstrap vs tempering + jittering filters over --da-steps assimilation steps")
    ap.add_argument("--da-steps", type=int, default=1000)
    ap.add_argument("--exp2", action="store_true", help="Exp 2: --exp1 with only [0, L/2] observed")
    ap.add_argument("--exp1-sigma", type=float, default=None,
                    help="observation error standard deviation of --exp1 (default 0.05)")
    ap.add_argument("--mala", action="store_true",
                    help="time the MALA jitter (moves/s) on the nudging workload")
    ap.add_argument("--filter-kernels", action="store_true",
                    help="time tempering, resampling and the row gather against their bounds")
    ap.add_argument("--proposal", action="store_true",
                    help="time the learned proposal network (forward, backward, Adam)")
    ap.add_argument("--occupancy", action="store_true",
                    help="jitter launch time at 1 .. 16 warps per SM (occupancy sweep)")
    ap.add_argument("--proposal-batch", type=int, default=8192, help="--proposal: samples per call")
    ap.add_argument("--train-cycles", type=int, default=200)
    ap.add_argument("--twins", type=int, default=5, help="--nudging: independent twin experiments")
    ap.add_argument("--nudging-workload", default="cfg4_f32", choices=["cfg4_f32", "cfg5_f32"],
                    help="--nudging: the learned-proposal workload or the large run")
    ap.add_argument("--epochs", type=int, default=10)
    args = ap.parse_args()
    if args.nudging:
        if args.steps == 100:
            args.steps = 20
        return run_nudging(args)
    if args.filter_kernels:
        if args.steps == 100:
            args.steps = 20
        return run_filter_kernels(args)
    if args.proposal:
        if args.steps == 100:
            args.steps = 20
        return run_proposal(args)
    if args.occupancy:
        if args.steps == 100:
            args.steps = 4
        return run_occupancy(args)
    if args.adjoint:
        if args.steps == 100:
            args.steps = 10
        return run_adjoint(args)
    if args.exp1 or args.exp2:
        return run_exp1(args)
    if args.mala:
        if args.steps == 100:
            args.steps = 5
        return run_mala(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
