"""Benchmark: Hermite DOF-updates/s on one B300 (replicas for N > 1).

Workload (the 3-D grid the throughput target is quoted on): periodic [0,1]^3,
m = 3, N = 128 cells per axis (2,097,152 nodes, 64 u + 27 v coefficients per
node), c dt/h = 0.9, u0 = sum of 8 Gaussian pulses (centres U[0,1)^3, widths
U[0.05,0.1], amplitudes N(0,1), numpy PCG64 seed 0), v0 = 0, dissipative
"full" variant, split precision (headline) and FP64.

One benchmark step = one pass of the whole hot path: 8 full time steps
(16 fused half-step launches) followed by one energy reduction (the energy
is a diagnostic taken every 8 steps).  The arithmetic paths run the same
steps from the same state: `value` is the split-precision path on the CUDA
cores (FP32 hi+lo); `split_tc` the same arithmetic with its products on the
tensor cores; `fp64` the FP64 path.  `accuracy` gives each path's relative
L2 error against the exact solution after the workload's 200 full steps
(the "matched L2 error" of the metric).  One DOF-update = one stored scaled
coefficient of one node written by one half-step.  The 3 GB state is far
larger than the 126 MB L2, so no flush is needed between steps.  The line
also carries compact results of the two other workloads (`batch2d`: 512
ragged 2-D problems; `learned2d`: the learned super-stepper at the bars 1e-3
and 1e-2) and the oracle timed on the host cores (`cpu_baseline`).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--workload grid3d|batch2d|learned2d|paper3d] [--no-extra] [--no-accuracy]
       [--no-cpu-baseline] [--ncu-case NAME [--variant V]]
For N > 1 launch with torch.distributed.run; each rank runs an independent
replica (the method needs no data-path collective here), the slowest rank's
time counts and `value` aggregates all ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hermite DOF-updates/s on 1 B300 (FP64 vs split-FP32/BF16) at matched L2 error"
UNIT = "DOF-updates/s"
D, M, N, LAM = 3, 3, 128, 0.9
FULL_STEPS_PER_STEP = 8
NU, NV = (M + 1) ** D, M ** D
NODES = N ** D
DOF_PER_HALF = NODES * (NU + NV)
WORKLOAD = ("3-D periodic [0,1]^3, m=3, N=128^3, c*dt/h=0.9, 8 seeded Gaussian pulses, v0=0, "
            "dissipative full variant")
# algorithmic flops of one node-half-step in the parity-reduced form: one
# operator row (2*nci multiply-adds) per output plus the corner transform
FLOP_PER_NODE = 2 * (NU + NV) * (NU + NV) + (NU + NV) * D * (1 << D)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except OSError:
        return {}


# Algorithmic HBM bytes of one half-step: every node's (Nu + Nv) coefficients
# read once from the source grid and written once to the target grid, 8 bytes
# each in both arithmetics (FP64, or an FP32 hi + lo pair).
ALG_BYTES_PER_LAUNCH = 2 * DOF_PER_HALF * 8
# DRAM read + write bytes per launch from ncu captures of the same kernels at
# 64^3, scaled to 128^3 by the node count
TRAFFIC_PER_LAUNCH = 373.8e6 * 8
SPLIT_TRAFFIC_PER_LAUNCH = 362.3e6 * 8
TC_TRAFFIC_PER_LAUNCH = 350.2e6 * 8
# tensor-core flops of the digit-split engine per node: 8 output classes x 8
# input classes (K = 16 each) x sum over the six data digits i of N = 16 (7 - i)
# operator-digit columns, two flops per multiply-add
TC_FLOP_PER_NODE = 2 * (1 << D) * (1 << D) * 16 * sum(16 * (7 - i) for i in range(6))
# FP32 operations the compensated (hi + lo) arithmetic spends per node: 12 per
# multiply-add of an operator row, 8 per addition of the corner transform
SPLIT_OPS_PER_NODE = (NU + NV) * (NU + NV) * 12 + (NU + NV) * D * (1 << D) * 8


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, ws):
    """The slowest rank's timing (every rank calls this; replicas run the same
    work, so the job's time is the maximum).  NCCL reduces a device tensor,
    gloo a host one."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, ws, ms_max):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return ws * units_per_rank / (ms_max / 1e3)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def initial_state():
    from paper_1802_05246_b300 import inputs as I

    h = 1.0 / N
    cen, wid, amp = I.pulses_3d_config(0)
    u0 = I.gaussian_data(D, M, N, h, I.PERIODIC, 0, cen, wid, amp)
    v0 = np.zeros((NODES, NV))
    return u0, v0


def cpu_baseline_sample(u0, v0, n_targets, seed=1):
    """The oracle, as it stands, on a bounded sample of the workload: one
    half-step for n_targets random dual nodes.  Returns (DOF-updates/s, seconds)."""
    import oracle

    h = 1.0 / N
    P = oracle.Problem(D, M, N, 1.0, h, LAM * h, oracle.DISSIPATIVE, oracle.PERIODIC)
    t = np.random.default_rng(seed).integers(0, NODES, n_targets)
    t0 = time.perf_counter()
    P.half_step_sample(1, u0, v0, t)
    dt = time.perf_counter() - t0
    return n_targets * (NU + NV) / dt, dt


_POOL_STATE = {}


def _pool_sample(job):
    """One worker's share of an all-cores oracle sample (state inherited by fork)."""
    seed, n_targets = job
    return cpu_baseline_sample(_POOL_STATE["u0"], _POOL_STATE["v0"], n_targets, seed)[1]


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


class OraclePool:
    """The oracle on every host core: one forked worker per core, each taking
    its own random target nodes.  Fork before the process makes any CUDA call
    (the workers inherit the initial state without copying it)."""

    def __init__(self, u0, v0):
        import multiprocessing as mp

        _POOL_STATE["u0"], _POOL_STATE["v0"] = u0, v0
        self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("fork").Pool(self.cores)

    def sample(self, per_core, seed):
        """All cores, per_core target nodes each: (DOF-updates/s, wall seconds)."""
        t0 = time.perf_counter()
        self.pool.map(_pool_sample, [(seed + i, per_core) for i in range(self.cores)], chunksize=1)
        wall = time.perf_counter() - t0
        return self.cores * per_core * (NU + NV) / wall, wall

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(u0, v0):
    """The oracle as it stands, on the host: single-threaded (8192 random dual
    nodes of the workload, one half-step each) and on every core (4096 nodes per
    core).  Runs before any CUDA call."""
    v1, s1 = cpu_baseline_sample(u0, v0, 8192, seed=1)
    pool = OraclePool(u0, v0)
    try:
        pool.sample(64, seed=1000)  # start-up
        va, sa = pool.sample(4096, seed=2000)
    finally:
        pool.close()
    return {"value": va, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "single_core_value": v1, "cpu_model": cpu_model(), "nproc": pool.cores,
            "sample": f"one half-step of random dual nodes of the same 128^3 grid: {pool.cores} cores x 4096 nodes "
                      f"({sa:.1f} s wall); single core 8192 nodes ({s1:.1f} s)"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on every host core."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    u0, v0 = initial_state()
    pool = OraclePool(u0, v0)
    per_core = 1024
    try:
        for k in range(args.warmup):
            pool.sample(128, seed=500 * (k + 1))
        times = [pool.sample(per_core, seed=10_000 * (k + 1))[1] for k in range(args.steps)]
    finally:
        pool.close()
    units = pool.cores * per_core * (NU + NV)
    value = units * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "sample": f"per step {pool.cores} cores x {per_core} random dual nodes, one half-step each"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"{pool.cores} x {per_core} random target nodes x {args.steps} steps of one "
                                   f"half-step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure(hb, torch, dev, u0, v0, precision, args, ws, want_clocks, engine=None):
    """Time W warm-up and K benchmark steps of one context; returns a dict
    (engine: the split-precision engine, None for the default)."""
    h = 1.0 / N
    g = hb.Hermite(D, M, N, 1.0, h, LAM * h, hb.DISSIPATIVE, hb.PERIODIC, precision=precision)
    if engine is not None:
        g.set_split_engine(engine)
    stream = torch.cuda.Stream(device=dev)
    g.set_stream(stream)
    du = torch.from_numpy(u0).to(dev)
    dv = torch.from_numpy(v0).to(dev)
    torch.cuda.synchronize()
    g.set_state_device(du, dv)
    del du, dv

    def one_step(events=None):
        for _ in range(2 * FULL_STEPS_PER_STEP):
            g.advance_half(1)
            if events is not None:
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(stream)
                events.append(ev)
        return g.energy()  # synchronises the stream

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    half_events = []
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(dev.index)
    with clk:
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(args.steps):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            evs = [ev0]
            energy = one_step(evs)
            half_events.append(evs)
        stop.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(start.elapsed_time(stop), ws)
    if ws > 1:
        torch.distributed.barrier()
    halfs = [a.elapsed_time(b) for evs in half_events for a, b in zip(evs[:-1], evs[1:])]
    half_ms = sum(halfs) / len(halfs)
    state = g.get_state()
    return {"g": g, "ms": ms, "half_ms": half_ms, "energy": energy, "state": state, "one_step": one_step,
            "clocks": clk.summary() if want_clocks else None}


ACC_STEPS = 200      # full steps of the 3-D pulse workload
ACC_CELLS = 2048     # cells sampled for the L2 errors (the same cells for every arithmetic)


def accuracy(hb, torch, dev, u0, v0, precision, engine=None):
    """Relative L2 error against the exact solution after the workload's 200
    full steps, by Gauss quadrature (2m+2 points per axis, exact for the
    squared interpolant) over ACC_CELLS seeded random cells; the exact
    solution (radial d'Alembert over periodic images) is evaluated on the
    device."""
    from paper_1802_05246_b300 import inputs as I

    h = 1.0 / N
    g = hb.Hermite(D, M, N, 1.0, h, LAM * h, hb.DISSIPATIVE, hb.PERIODIC, precision=precision)
    if engine is not None:
        g.set_split_engine(engine)
    du = torch.from_numpy(u0).to(dev)
    dv = torch.from_numpy(v0).to(dev)
    g.set_state_device(du, dv)
    del du, dv
    g.step(ACC_STEPS)
    T = g.time
    x, w = np.polynomial.legendre.leggauss(2 * M + 2)
    xq, wq = 0.5 * x, 0.5 * w
    cells = np.sort(np.random.default_rng(12345).choice(NODES, ACC_CELLS, replace=False))
    ax = I.axis_coords(N, h, I.PERIODIC, 1)  # cells of the primal level: centred at dual nodes
    ci = np.stack(np.unravel_index(cells, (N,) * D), -1)
    Q = np.stack(np.meshgrid(*([xq * h] * D), indexing="ij"), -1).reshape(-1, D)
    pts = torch.from_numpy(ax[ci][:, None, :] + Q[None, :, :]).to(dev)
    cen, wid, amp = I.pulses_3d_config(0)
    ex = I.pulse_wave_3d(pts, T, cen, wid, amp, xp=torch).contiguous()
    e2, n2 = g.l2_error(0, xq, wq, ex, torch.from_numpy(cells.astype(np.int64)).to(dev))
    g.close()
    return float(np.sqrt(e2 / n2)), T


def run_ours(args):
    ws, rank, local = dist_env()
    u0, v0 = initial_state()
    # the oracle on the host cores, before this process makes any CUDA call
    cpu = cpu_baseline(u0, v0) if (ws == 1 and rank == 0 and not args.no_cpu_baseline) else None

    import torch

    import paper_1802_05246_b300 as hb

    torch.cuda.set_device(local)  # before the process group, so NCCL binds this rank's GPU
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)

    fp64 = measure(hb, torch, dev, u0, v0, hb.FP64, args, ws, False)
    split = measure(hb, torch, dev, u0, v0, hb.SPLIT32, args, ws, True, engine=0)
    fp64["g"].close()
    tcm = measure(hb, torch, dev, u0, v0, hb.SPLIT32, args, ws, False, engine=1)
    tcm["g"].close()
    # same start, same number of steps: difference of the two arithmetic paths
    a = np.concatenate([fp64["state"][0], fp64["state"][1]], 1)
    b = np.concatenate([split["state"][0], split["state"][1]], 1)
    split_vs_fp64 = float(np.linalg.norm(a - b) / np.linalg.norm(a))
    del a, b

    dof_per_step = 2 * FULL_STEPS_PER_STEP * DOF_PER_HALF
    value = job_throughput(dof_per_step * args.steps, ws, split["ms"])
    value64 = job_throughput(dof_per_step * args.steps, ws, fp64["ms"])

    # end to end through the public API with host buffers: H2D of the state,
    # the step, and D2H of the state and the energy
    g = split["g"]
    one_step = split["one_step"]
    hu = torch.from_numpy(u0).pin_memory()
    hv = torch.from_numpy(v0).pin_memory()
    ou = torch.empty_like(hu).pin_memory()
    ov = torch.empty_like(hv).pin_memory()
    g.set_state(hu.numpy(), hv.numpy())
    one_step()
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.set_state(hu.numpy(), hv.numpy())
        one_step()
        g.get_state(ou.numpy(), ov.numpy())
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws)
    e2e_value = job_throughput(dof_per_step, ws, 1e3 * e2e_s)
    state_bytes = NODES * (NU + NV) * 8
    g.close()
    del hu, hv, ou, ov

    # matched L2 error: both arithmetics against the exact solution after the
    # workload's 200 steps (untimed)
    if args.no_accuracy:
        err64 = errsp = errtc = T = None
    else:
        err64, T = accuracy(hb, torch, dev, u0, v0, hb.FP64)
        errsp, _ = accuracy(hb, torch, dev, u0, v0, hb.SPLIT32, engine=0)
        errtc, _ = accuracy(hb, torch, dev, u0, v0, hb.SPLIT32, engine=1)

    # the other two spec workloads, compact (single GPU; untimed for the headline)
    extra = {}
    if ws == 1 and not args.no_extra:
        by = batch_results(3, 2, variants=(hb.DISSIPATIVE,))
        extra["batch2d"] = {
            "workload": "ragged batch of 512 2-D dissipative problems (N in {32,64,128,256}^2, m in 2..6, "
                        "periodic/Dirichlet/Neumann, 1-4 Gaussian pulses, c*dt/h=0.9), autotuned, graph-captured",
            "unit": UNIT, "fp64": by["dissipative_fp64"], "split": by["dissipative_split"]}
        from paper_1802_05246_b300.learned import SuperStepper

        st = SuperStepper.load(LEARNED_WEIGHTS)
        lr = learned_results(st, [1e-3, 1e-2], 3, 1, ((hb.FP64, "fp64"),))
        extra["learned2d"] = {
            "workload": "256 2-D periodic problems, m=3, N=128^2, c*dt/h=0.9, 1-6 Gaussian pulses, K=16 full "
                        "steps per checked network advance, FP64 check and fallback",
            "kappa": st.kappa, "plain_hermite_fp64_ms": lr["hermite_fp64_ms"],
            "network_only_ms": lr["network_only_ms"],
            "true_error_quantiles": {q: float(np.quantile(lr["e_true"], v))
                                     for q, v in (("10%", 0.1), ("50%", 0.5), ("90%", 0.9))},
            "bars": {f"{bar:.0e}": {"accepted": lr[(bar, "accepted_fp64")],
                                    "false_accepts": lr[(bar, "false_accepts_fp64")],
                                    "checked_advance_ms": lr[(bar, "learned_fp64_ms")],
                                    "gain_vs_plain_fp64": lr["hermite_fp64_ms"] / lr[(bar, "learned_fp64_ms")]}
                     for bar in (1e-3, 1e-2)}}

    if rank != 0:
        return 0
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    probe32 = hb.peak_probe(2) / 1e12  # packed FP32 pairs, the split kernel's form
    probe64 = hb.peak_probe(0) / 1e12

    def roofline(kernel, launch_ms, traffic, pipe, probe, impl_ops=None):
        achieved = ALG_BYTES_PER_LAUNCH / (launch_ms / 1e3) / 1e9
        method = NODES * FLOP_PER_NODE / (launch_ms / 1e3) / 1e12
        r = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": hbm, "unit": "GB/s",
             "frac": achieved / hbm if hbm else None, "traffic": traffic,
             "algorithmic_bytes_per_launch": ALG_BYTES_PER_LAUNCH, "launch_ms": launch_ms,
             "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
             "compute": {"pipe": pipe, "method_flop_per_launch": NODES * FLOP_PER_NODE, "method_tflops": method,
                         "probe_peak_tflops": probe, "method_frac_of_probe": method / probe,
                         "peak_source": "probe: hermite_peak_probe, FMA chains on this GPU"}}
        if impl_ops:
            r["compute"]["impl_ops_per_launch"] = impl_ops
            r["compute"]["impl_tops"] = impl_ops / (launch_ms / 1e3) / 1e12
        return r

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": split["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2", "data": "synthetic",
        "config": {"workload": WORKLOAD, "d": D, "m": M, "N": N, "cfl": LAM, "variant": "dissipative",
                   "bc": "periodic", "precision": "split: FP32 hi+lo state and operator, three split products, "
                                                  "compensated sums (HERMITE_SPLIT32, CUDA-core engine)",
                   "step": "8 full time steps (16 half-steps) + 1 energy reduction",
                   "l2": "inputs larger than L2 (3.05 GB read+written per half-step vs 126 MB)",
                   "parallelism": f"replicas x{ws}"},
        "roofline": roofline("half_step_split_kernel<3,12,10>", split["half_ms"], SPLIT_TRAFFIC_PER_LAUNCH,
                             "FP32 (packed pairs)", probe32, NODES * SPLIT_OPS_PER_NODE),
        "accuracy": None if err64 is None else {
            "l2_err_fp64": err64, "l2_err_split": errsp, "ratio_split_over_fp64": errsp / err64,
            "bar": "split <= 1.2 x fp64 where fp64 >= 1e-9", "meets_bar": errsp <= 1.2 * err64,
            "t": T, "full_steps": ACC_STEPS,
            "measure": f"relative L2 of the I_m interpolant vs the exact solution, {ACC_CELLS} sampled "
                       f"cells, {2 * M + 2}^3 Gauss points each"},
        "split_tc": {"value": job_throughput(dof_per_step * args.steps, ws, tcm["ms"]),
                     "ms_per_step": tcm["ms"] / args.steps, "dtype": "f32x2",
                     "engine": "tensor cores (tcgen05): six BF16 data digits x seven operator digits, exact FP32 "
                               "accumulation (hermite_set_split_engine 1)",
                     "l2_err": errtc, "ratio_over_fp64": None if err64 is None else errtc / err64,
                     "roofline": roofline("half_step_tc_kernel<3>", tcm["half_ms"], TC_TRAFFIC_PER_LAUNCH,
                                          "tensor (BF16 digits)",
                                          pk.get("bf16_tflops"), NODES * TC_FLOP_PER_NODE)},
        "fp64": {"value": value64, "ms_per_step": fp64["ms"] / args.steps, "dtype": "f64",
                 "roofline": roofline("half_step_f64_kernel<3,92>", fp64["half_ms"], TRAFFIC_PER_LAUNCH, "FP64",
                                      probe64),
                 "energy_plain_last": float(fp64["energy"][0])},
        "split_vs_fp64_rel_l2": split_vs_fp64,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes + 24},
        # per step: one half-step kernel per half-step, then the energy: one
        # sum-factorised kernel (both forms) and two partial-sum reductions
        "gpu_launches": (2 * FULL_STEPS_PER_STEP + 3) * args.steps,
        "clocks": split["clocks"],
        # the plain energy int v^2 + c^2 |grad u|^2; the invariant (seminorm)
        # energy of smooth fine-grid data is rounding-level and not reported here
        "energy_plain_last": float(split["energy"][0]),
        **extra,
    }
    print(json.dumps(line), flush=True)
    return 0


def batch_problems(seed=0, n=512, lam=0.9):
    """Ragged 2-D workload: N uniform in {32,64,128,256} (square grids), m
    uniform in {2..6}, boundary uniform in {periodic, Dirichlet, Neumann},
    u0 = 1-4 Gaussian pulses (widths U[0.05,0.2], amplitudes N(0,1), centres
    U[0,1)^2), v0 = 0, c dt/h = 0.9; numpy PCG64 with the given seed."""
    from paper_1802_05246_b300 import inputs as I

    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        Np = int(rng.choice([32, 64, 128, 256]))
        m = int(rng.integers(2, 7))
        bc = int(rng.integers(0, 3))
        cen, wid, amp = I.random_pulses(rng, 2, 1, 4, 0.05, 0.2)
        out.append((Np, m, bc, cen, wid, amp))
    return out


def batch_results(steps, warmup, variants=(0, 1)):
    """Ragged batch of 512 2-D problems: throughput of each variant in FP64 and
    split precision at the autotuned item size and blocks per SM."""
    import torch

    import paper_1802_05246_b300 as hb
    from paper_1802_05246_b300 import inputs as I

    specs = batch_problems()
    lam = 0.9
    results = {}
    for variant in variants:
        probs = [(2, m, Np, 1.0, 1.0 / Np, lam / Np, variant, bc) for (Np, m, bc, _, _, _) in specs]
        for prec in (hb.FP64, hb.SPLIT32):
            b = hb.HermiteBatch(probs, precision=prec)
            s = torch.cuda.Stream()
            b.set_stream(s)
            items, blocks, tune_ms = b.autotune()
            for (Np, m, bc, cen, wid, amp), g in zip(specs, b.problems):
                u0 = I.gaussian_data(2, m, Np, 1.0 / Np, bc, 0, cen, wid, amp)
                g.set_state(u0, np.zeros((g.nodes(0), m * m)))
            b.step(warmup)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(s)
            b.step(steps)
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            results[(variant, prec)] = {"value": b.dof_per_step * steps / (ms / 1e3), "ms_per_step": ms / steps,
                                        "autotune": {"item_nodes": items, "blocks_per_sm": blocks, "ms": tune_ms}}
            b.close()
    return {f"{'dissipative' if v == 0 else 'conservative'}_{'fp64' if p == 0 else 'split'}": r
            for (v, p), r in results.items()}


def run_batch(args):
    """Ragged batch of 512 2-D problems, both variants, FP64 and split."""
    import torch

    torch.cuda.set_device(0)
    by = batch_results(args.steps, args.warmup)
    results = {(0, 1): by["dissipative_split"]}
    line = {
        "metric": METRIC, "value": results[(0, 1)]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": results[(0, 1)]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32x2", "data": "synthetic",
        "config": {"workload": "ragged batch of 512 2-D problems (N in {32,64,128,256}^2, m in 2..6, "
                               "periodic/Dirichlet/Neumann, 1-4 Gaussian pulses, c*dt/h=0.9), one persistent "
                               "launch per size group per half-step, graph-captured full steps",
                   "step": "one full time step of all 512 problems"},
        "by_variant_precision": by,
    }
    print(json.dumps(line), flush=True)
    return 0


# The paper's 3-D performance runs (periodic-type data; "time per iteration"
# on one P100, FP64), read here as one full step: (variant, m, points per
# direction, seconds per iteration or None).  Context only, other hardware.
PAPER_3D_RUNS = [
    ("simple", 1, 160, 0.057), ("simple", 2, 120, 0.087), ("simple", 3, 90, 0.10),
    ("full", 1, 160, 0.11), ("full", 2, 120, 0.17), ("full", 3, 90, None),
    ("conservative", 1, 280, 0.035), ("conservative", 2, 190, 0.052), ("conservative", 3, 140, 0.0579),
]


def run_paper3d(args):
    """3-D at scale: the paper's own performance configurations (simple and
    full dissipative, conservative; periodic) and the 128^3 m=3 grid with
    Dirichlet and Neumann boundaries, FP64 and split precision.  One step =
    one full time step (two half-steps) of one problem."""
    import torch

    import paper_1802_05246_b300 as hb

    torch.cuda.set_device(0)
    vid = {"simple": hb.DISSIPATIVE_SIMPLE, "full": hb.DISSIPATIVE, "conservative": hb.CONSERVATIVE}
    cases = [(v, m, n, hb.PERIODIC, p100) for (v, m, n, p100) in PAPER_3D_RUNS]
    cases += [(v, 3, 128, bc, None) for v in ("full", "simple", "conservative")
              for bc in (hb.PERIODIC, hb.DIRICHLET, hb.NEUMANN)]
    out = []
    gen = torch.Generator(device="cuda").manual_seed(0)
    for (vname, m, n, bc, p100) in cases:
        # "points per direction": n nodes per axis on the primal grid
        N = n if bc == hb.PERIODIC else n - 1
        h = 1.0 / N
        for prec, engine in ((hb.FP64, None), (hb.SPLIT32, 0), (hb.SPLIT32, 1)):
            g = hb.Hermite(3, m, N, 1.0, h, 0.9 * h, vid[vname], bc, precision=prec)
            if engine is not None:
                g.set_split_engine(engine)
            n0 = g.nodes(0)
            u = torch.randn((n0, g.Nu), dtype=torch.float64, device="cuda", generator=gen)
            v = torch.randn((n0, g.Nv), dtype=torch.float64, device="cuda", generator=gen) if g.Nv else None
            g.set_state_device(u, v)
            del u, v
            s = torch.cuda.Stream()
            g.set_stream(s)
            g.step(args.warmup)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(s)
            g.step(args.steps)
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            dof = (g.nodes(0) + g.nodes(1)) * (g.Nu + g.Nv)  # DOF-updates of one full step
            out.append({"variant": vname, "m": m, "points": n, "bc": ["periodic", "dirichlet", "neumann"][bc],
                        "precision": "fp64" if engine is None else ("split" if engine == 0 else "split_tc"),
                        "ms_per_full_step": ms,
                        "dof_updates_per_s": dof / (ms / 1e3),
                        "p100_s_per_iteration": p100,
                        "speedup_vs_p100": (p100 * 1e3 / ms) if p100 else None})
            g.close()
            torch.cuda.empty_cache()
    head = next(r for r in out if r["variant"] == "full" and r["m"] == 3 and r["points"] == 128
                and r["bc"] == "dirichlet" and r["precision"] == "split")
    line = {
        "metric": METRIC, "value": head["dof_updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_full_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2", "data": "synthetic (N(0,1) coefficients; timing does not depend on "
                                                      "the values)",
        "config": {"workload": "3-D at scale: the paper's P100 configurations and m=3 128^3 with "
                               "periodic/Dirichlet/Neumann boundaries, c*dt/h=0.9",
                   "step": "one full time step of one problem", "headline": "full dissipative, m=3, 128^3, "
                                                                            "Dirichlet, split"},
        "cases": out,
    }
    print(json.dumps(line), flush=True)
    return 0


LEARNED_WEIGHTS = os.path.join(ROOT, "paper_1802_05246_b300", "weights", "superstepper_k16.npz")


def learned_results(st, bars, steps, warmup, precisions):
    """The learned super-stepper against plain Hermite steps on 256 fresh 2-D
    problems (m = 3, 128^2 periodic, 1-6 Gaussian pulses, widths U[0.05,0.15]):
    one step advances every problem by K = 16 full steps, checked (one true
    full step, residual estimate) and falling back to plain steps above the
    bar.  Returns the timings, acceptance and false accepts per bar and check
    precision, and the true K-step errors (evaluated untimed)."""
    import torch

    import paper_1802_05246_b300 as hb

    B = 256
    trajs = list(range(3_000_000, 3_000_000 + B))
    stream = torch.cuda.current_stream()
    zero_v = np.zeros((st.n, st.Nv))

    def fresh(prec):
        b = hb.HermiteBatch([st.problem] * B, precision=prec)
        b.set_stream(stream)
        for p, t in enumerate(trajs):
            b.problem(p).set_state(st.initial_u(t), zero_v)
        return b

    def timed(fn, before=None):
        for _ in range(warmup):
            if before:
                before()
            fn()
        ms = []
        for _ in range(steps):
            if before:
                before()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    e_true, resid = st.evaluate(trajs)  # untimed: the true K-step error of every prediction
    res = {"work": B * st.K * 2 * st.n * st.C0, "e_true": e_true, "resid": resid}
    for prec, name in precisions:
        b = fresh(prec)
        res[f"hermite_{name}_ms"] = timed(lambda: b.step(st.K))
        b.close()
        b = fresh(prec)
        X = st._alloc_states(B)
        st.gather(b, *X)
        for bar in bars:
            out = {}

            def run():
                out["acc"], out["est"] = st.advance(b, bar=bar)

            res[(bar, f"learned_{name}_ms")] = timed(run, before=lambda: st.scatter(b, *X))
            res[(bar, f"accepted_{name}")] = float(np.mean(out["acc"]))
            res[(bar, f"false_accepts_{name}")] = int(np.sum(out["acc"] & (e_true > bar)))
        A = st._alloc_states(B)
        res["network_only_ms"] = timed(lambda: st.predict(X[0], X[1], A[0], A[1]))
        b.close()
    return res


def run_learned(args):
    """Learned super-stepper against plain Hermite steps on 256 fresh 2-D
    problems (m = 3, 128^2 periodic, 1-6 Gaussian pulses, widths U[0.05,0.15]):
    one benchmark step advances every problem by K = 16 full steps."""
    import torch

    import paper_1802_05246_b300 as hb
    from paper_1802_05246_b300.learned import SuperStepper

    torch.cuda.set_device(0)
    st = SuperStepper.load(args.weights)
    B, bar = 256, args.bar
    stream = torch.cuda.current_stream()
    r = learned_results(st, [bar], args.steps, args.warmup, ((hb.FP64, "fp64"), (hb.SPLIT32, "split")))
    e_true, resid, work = r["e_true"], r["resid"], r["work"]
    res = {k: v for k, v in r.items() if isinstance(k, str)}
    res.update({k[1]: v for k, v in r.items() if isinstance(k, tuple)})

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    # the dominant kernel: the 64 -> 64 forward convolution at the inference batch
    x = torch.zeros((B, 128, 128, 64), dtype=torch.bfloat16, device="cuda")
    y = torch.empty_like(x)
    w = torch.zeros((64, 9, 64), dtype=torch.bfloat16, device="cuda")
    L = hb.lib()
    conv_ms = timed(lambda: L.hnn_conv3x3_fwd(x.data_ptr(), w.data_ptr(), None, None, B, 128, 128, 64, 64, 8, 1,
                                              y.data_ptr(), None, stream.cuda_stream))
    conv_tflops = 2 * B * st.n * 9 * 64 * 64 / (conv_ms / 1e3) / 1e12
    peak = peaks().get("bf16_tflops", 1800.0)
    quant = lambda q: float(np.quantile(e_true, q))
    sweep = {f"{b_:.0e}": {"accepted_by_estimate": float(np.mean(st.kappa * resid <= b_)),
                           "true_error_within": float(np.mean(e_true <= b_))}
             for b_ in (1e-3, 3e-3, 1e-2, 3e-2, 1e-1)}
    line = {
        "metric": "effective Hermite DOF-updates/s of K=16-step advances at rel. L2 <= bar (learned + fallback)",
        "value": work / (res["learned_fp64_ms"] / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["learned_fp64_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (network) / f64 (check, fallback)", "data": "synthetic",
        "config": {"workload": "256 2-D periodic problems, m=3, N=128^2, c*dt/h=0.9, 1-6 Gaussian pulses "
                               "(widths U[0.05,0.15]), K=16 full steps per advance",
                   "bar": bar, "kappa": st.kappa, "weights": os.path.relpath(args.weights, ROOT)},
        "plain_hermite_fp64": {"value": work / (res["hermite_fp64_ms"] / 1e3), "ms_per_step": res["hermite_fp64_ms"]},
        "plain_hermite_split": {"value": work / (res["hermite_split_ms"] / 1e3),
                                "ms_per_step": res["hermite_split_ms"]},
        "learned_split": {"value": work / (res["learned_split_ms"] / 1e3), "ms_per_step": res["learned_split_ms"],
                          "accepted": res["accepted_split"], "false_accepts": res["false_accepts_split"]},
        "accepted": res["accepted_fp64"], "false_accepts": res["false_accepts_fp64"],
        "gain_vs_fp64": res["hermite_fp64_ms"] / res["learned_fp64_ms"],
        "gain_vs_split": res["hermite_split_ms"] / res["learned_split_ms"],
        "network_only_ms": res["network_only_ms"],
        "true_error_quantiles": {"10%": quant(0.1), "50%": quant(0.5), "90%": quant(0.9), "max": quant(1.0)},
        "bar_sweep": sweep,
        "roofline": {"bound": "tensor", "kernel": "conv_fwd_kernel<64,64>", "achieved": conv_tflops, "peak": peak,
                     "unit": "TFLOP/s", "frac": conv_tflops / peak, "traffic": None},
    }
    print(json.dumps(line), flush=True)
    return 0


NCU_CASES = ("half_step_f64", "half_step_split", "half_step_tc", "energy_f64", "energy_split", "batch_f64", "batch_split", "conv")


def run_ncu_case(args):
    """Small, self-contained cases for Nsight Compute captures (not benchmarks;
    no timing is printed):
      half_step_f64 / half_step_split / half_step_tc: 3-D m=3, 64^3 periodic, c dt/h = 0.9,
        random device data (~380 MB moved per half-step, above the L2), three
        half-steps of --variant (0 full dissipative, 1 conservative, 2 simple);
        the split cases on the CUDA-core and the tensor-core engine;
      energy_f64 / energy_split: the same grid, one energy call (both forms);
      batch_f64 / batch_split: the first 128 problems of the seed-0 ragged 2-D
        workload (dissipative), two full steps at the item size and blocks per
        SM the autotuner picks on the full workload (256 nodes; 2 blocks per
        SM for FP64, 8 for split);
      conv: 64 images of 128 x 128 x 64 channels in BF16 (134 MB), dilation 8,
        three forward launches, then three weight-gradient launches."""
    import torch

    import paper_1802_05246_b300 as hb

    torch.cuda.set_device(0)
    case = args.ncu_case
    if case.startswith(("half_step", "energy")):
        n, m = 64, 3
        h = 1.0 / n
        prec = hb.FP64 if case.endswith("f64") else hb.SPLIT32
        variant = args.variant if case.startswith("half_step") else hb.DISSIPATIVE
        g = hb.Hermite(3, m, n, 1.0, h, 0.9 * h, variant, hb.PERIODIC, precision=prec)
        if prec == hb.SPLIT32:
            g.set_split_engine(1 if case == "half_step_tc" else 0)
        u = torch.randn(n ** 3, (m + 1) ** 3, dtype=torch.float64, device="cuda")
        v = torch.randn(n ** 3, m ** 3, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        g.set_state_device(u, v)
        if case.startswith("half_step"):
            g.advance_half(3)
        else:
            g.energy()
        torch.cuda.synchronize()
        g.close()
    elif case.startswith("batch"):
        fp64 = case == "batch_f64"
        probs = [(2, m, Np, 1.0, 1.0 / Np, 0.9 / Np, hb.DISSIPATIVE, bc)
                 for (Np, m, bc, _, _, _) in batch_problems()[:128]]
        b = hb.HermiteBatch(probs, precision=hb.FP64 if fp64 else hb.SPLIT32)
        b.set_stream(torch.cuda.Stream())
        b.config(256, 2 if fp64 else 8)
        b.step(2)
        torch.cuda.synchronize()
        b.close()
    else:
        B, C, dil = 64, 64, 8
        L = hb.lib()
        s = torch.cuda.current_stream().cuda_stream
        x = torch.randn((B, 128, 128, C), device="cuda").to(torch.bfloat16)
        dy = torch.randn((B, 128, 128, C), device="cuda").to(torch.bfloat16)
        w = (torch.randn((C, 9, C), device="cuda") * 0.05).to(torch.bfloat16)
        y = torch.empty_like(x)
        dw = torch.zeros((C, 9, C), device="cuda")
        for _ in range(3):
            if L.hnn_conv3x3_fwd(x.data_ptr(), w.data_ptr(), None, None, B, 128, 128, C, C, dil, 1, y.data_ptr(),
                                 None, s):
                raise RuntimeError("hnn_conv3x3_fwd failed")
        for _ in range(3):
            if L.hnn_conv3x3_wgrad(x.data_ptr(), dy.data_ptr(), B, 128, 128, C, C, dil, dw.data_ptr(), s):
                raise RuntimeError("hnn_conv3x3_wgrad failed")
        torch.cuda.synchronize()
    print("ncu case", case, "ok", flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid3d", choices=["grid3d", "batch2d", "learned2d", "paper3d"])
    ap.add_argument("--weights", default=LEARNED_WEIGHTS, help="learned2d: trained super-stepper")
    ap.add_argument("--bar", type=float, default=1e-3, help="learned2d: accepted rel. L2 error")
    ap.add_argument("--ncu-case", choices=NCU_CASES, default=None,
                    help="run one small case for an Nsight Compute capture instead of a benchmark")
    ap.add_argument("--variant", type=int, default=0, help="--ncu-case half_step_*: method variant")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing on the host cores")
    ap.add_argument("--no-extra", action="store_true", help="skip the compact batch2d / learned2d sub-objects")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the 200-step error measurements against the exact solution (profiling runs)")
    args = ap.parse_args()
    if args.ncu_case:
        return run_ncu_case(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch2d":
        return run_batch(args)
    if args.workload == "learned2d":
        return run_learned(args)
    if args.workload == "paper3d":
        return run_paper3d(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
