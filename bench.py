#!/usr/bin/env python
"""Throughput of the batched many-particle CTQW propagation on GB300.

One bench step is one pass of the hot path over one batch: write the initial
states of all realizations, then propagate them n_steps Taylor steps (order K)
while sampling P(x) (ensemble-averaged), norms and energies every obs_every
steps.  Default workload: bosons_n256_u2 (2 bosons, open chain N=256, U=2,
eps ~ U[-1,1], J = 1 + U[-0.25,0.25], dt = 0.02, K = 16, 2500 steps, 1024
realizations, complex FP32 with compensated update).  Metric: site-updates/s
= N^m * K * steps * realizations / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank drives one GPU and owns its own block of
realizations (weak scaling); the ranks' ensemble means are combined once per
step in FP64.  --impl reference times the FP64 CPU oracle on the host cores
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import ctqw_workloads as cw  # noqa: E402

METRIC = "site-updates/s (dim x K x steps x realizations)"
UNIT = "site-updates/s"
FP32_FMA_LANES_PER_SM = 128      # FP32 FMA lanes per SM
FP64_FMA_PER_SM = 2              # FP64 FMA per SM per cycle
SM_COUNT = 152                   # replaced by the device's count at run time
SM_MAX_MHZ = 2070.0
FMA_PEAKS = {}                   # measured by measure_fma_peaks() (TFLOP/s)


# ---------------------------------------------------------------- oracle (CPU) legs
def _oracle_chunk(args):
    """Propagate one realization of a workload with the oracle (runs in a worker)."""
    name, r, n_steps = args
    import numpy as np  # noqa: F401

    import oracle

    w = cw.get(name)
    N = int(w.sizes()[r])
    ue, uj = cw.uniform_draws(w.seed, [r], [N])
    eps, J = oracle.workload_parameters(w, ue[0], uj[0], N)
    H = oracle.many_particle_hamiltonian(oracle.single_particle_hamiltonian(eps, J, w.periodic), w.m, w.U)
    psi = oracle.initial_state(N, w.m, w.initial_sites(N), w.statistics)
    t0 = time.perf_counter()
    res = oracle.propagate(H, psi, N, w.m, w.dt, n_steps, w.obs_every, "taylor", w.K)
    dt = time.perf_counter() - t0
    return float(N ** w.m) * w.K * n_steps, dt, float(res["norm"][-1])


def oracle_sample(name: str, cores: int, n_steps: int, first: int = 0):
    """Site-updates/s of the oracle over `cores` realizations run in parallel,
    the units, the wall time and the median single-core rate (each worker
    times its own realization on one core)."""
    ctx = mp.get_context("spawn")
    jobs = [(name, first + k, n_steps) for k in range(cores)]
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_chunk, [(name, 0, 1)] * cores)   # import warm-up in every worker
        t0 = time.perf_counter()
        out = pool.map(_oracle_chunk, jobs)
        wall = time.perf_counter() - t0
    units = sum(o[0] for o in out)
    single = statistics.median(o[0] / o[1] for o in out)
    return units / wall, units, wall, single


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.gpu_id], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sms, maxs, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs),
                "reasons": sorted(reasons), "samples": len(sms),
                "power_w_median": statistics.median(power) if power else None}


# ---------------------------------------------------------------- helpers
def measure_fma_peaks(seconds: float = 0.5):
    """FP32 (packed pairs, the stencil kernels' instruction) and FP64 FMA
    peaks of this GPU, measured now by the project's FMA-chain kernel
    (paper_1612_00746_gb300/peaks/fma_peak.cu), in TFLOP/s."""
    import ctypes

    path = os.path.join(ROOT, "paper_1612_00746_gb300", "libfmapeak.so")
    lib = ctypes.CDLL(path)
    lib.fma_peak_measure.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
    out = {}
    for kind, name in ((0, "fp32"), (2, "fp64")):
        v, e = ctypes.c_double(), ctypes.c_double()
        if lib.fma_peak_measure(kind, seconds, ctypes.byref(v), ctypes.byref(e)) == 0:
            out[name] = 2.0 * v.value / 1e12
    return out


def set_sm_count(dev) -> None:
    global SM_COUNT
    import torch

    SM_COUNT = int(torch.cuda.get_device_properties(dev).multi_processor_count)


def alu_peak(fp64: bool = False) -> float:
    """Derived peak: SMs x FMA lanes x 2 flop x maximum SM clock (TFLOP/s)."""
    lanes = FP64_FMA_PER_SM if fp64 else FP32_FMA_LANES_PER_SM
    return SM_COUNT * lanes * 2 * SM_MAX_MHZ * 1e6 / 1e12


def with_measured(entry: dict, key: str) -> dict:
    """Add the measured FMA peak and the fraction of it to a roofline entry."""
    if key in FMA_PEAKS and entry.get("achieved") is not None:
        entry["peak_measured"] = FMA_PEAKS[key]
        entry["frac_of_measured"] = entry["achieved"] / FMA_PEAKS[key]
        entry["peak_measured_basis"] = ("FMA-chain kernel (fma.rn.f32x2)" if key == "fp32"
                                        else "FMA-chain kernel (FP64 fma)") + ", this run"
    return entry


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fused_traffic(workload: str):
    """DRAM bytes per launch of the fused kernel from the committed ncu capture,
    or None when the kernel source changed since the counters were taken."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "taylor_fused_traffic.json")) as f:
            rec = json.load(f)
        src = os.path.join(ROOT, "paper_1612_00746_gb300", "csrc", "k_fused_rows.cu")
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except (OSError, ValueError):
        return None
    ent = rec.get(workload)
    if not ent or ent.get("source_sha256") != digest:
        return None
    return ent.get("dram_bytes_per_launch")


def propagation_path(w, dtype, flags, switching=False):
    """Which kernels ctqw_propagate_taylor runs for this workload (mirrors the library)."""
    from paper_1612_00746_gb300 import ctqw

    shape = (flags >> 8) & 0xF
    if flags & ctqw.FLAG_PLAIN:
        return "plain"
    if switching:
        return "tiled" if dtype == ctqw.C64 and w.m == 2 else "plain"
    if shape == ctqw.SHAPE_WAVEFRONT:
        return "wavefront"
    if shape >= 9:
        return "tiled"
    uniform = w.ragged_sizes is None
    if dtype == ctqw.C64 and w.m == 2 and uniform and w.N in (64, 128, 192, 256):
        return "rows" if shape < 4 else "banded"
    if dtype == ctqw.C64 and w.m == 2 and shape == 0:
        return "tiled"   # the library's default for the other two-particle FP32 handles
    return "plain"


def roofline_of(w, dtype, flags, units, kernel_ms, peaks, traffic, switching=False):
    """Roofline entry of the kernel that dominates the propagate call.

    Fused kernels (every Taylor term on chip) are bound by the FP32 FMA pipe:
    8m+4 algorithmic flops per site-update against the SMs x 128 lanes x 2
    flop x 2070 MHz.  The FP32 per-term kernels stream the state through HBM:
    per site-update ((K-1) 24 + 40)/K bytes (Horner stages and the
    compensated final stage), against the measured copy bandwidth.  The FP64
    per-term kernels move 64 bytes per site-update but are bound by the FP64
    pipe (2 DFMA per SM per cycle).
    """
    from paper_1612_00746_gb300 import ctqw

    path = propagation_path(w, dtype, flags, switching)
    sec = kernel_ms / 1000.0
    if path in ("rows", "banded", "wavefront", "tiled"):
        flops_per_unit = 8 * w.m + 4
        achieved = units * flops_per_unit / sec / 1e12
        peak = alu_peak()
        kernel = {"rows": "taylor_fused_rows_kernel", "banded": "taylor_fused_kernel",
                  "wavefront": "taylor_wavefront_kernel", "tiled": "taylor_tiled_reg_kernel"}[path]
        return with_measured({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                              "frac": achieved / peak, "traffic": traffic if path == "rows" else None,
                              "kernel": kernel, "kernel_ms": kernel_ms, "flops_per_site_update": flops_per_unit,
                              "peak_basis": f"{SM_COUNT} SMs x 128 FP32 FMA lanes x 2 flop x 2070 MHz (derived)",
                              "hbm_gbs_measured": peaks.get("hbm_gbs")}, "fp32")
    if dtype == ctqw.C128:
        # FP64 on GB300 runs 2 DFMA per SM per cycle: the per-term FP64
        # kernels are bound by that pipe, not by HBM (64 B per site-update)
        flops_per_unit = 8 * w.m + 4
        achieved = units * flops_per_unit / sec / 1e12
        peak = alu_peak(fp64=True)
        return with_measured({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                              "frac": achieved / peak, "traffic": None, "kernel": "taylor_term_kernel<double>",
                              "kernel_ms": kernel_ms, "flops_per_site_update": flops_per_unit,
                              "hbm_gbs_achieved": units * 64.0 / sec / 1e9, "bytes_per_site_update": 64.0,
                              "peak_basis": f"{SM_COUNT} SMs x 2 DFMA x 2 flop x 2070 MHz (FP64, derived)",
                              "timing": "the whole propagate call (observables kernels included)"}, "fp64")
    bpu = ((w.K - 1) * 24.0 + 40.0) / w.K
    kernel = "horner_stage_kernel + horner_final_kernel"
    gbs = units * bpu / sec / 1e9
    peak = peaks.get("hbm_gbs")
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak if peak else None, "traffic": None, "kernel": kernel,
            "kernel_ms": kernel_ms, "bytes_per_site_update": bpu,
            "peak_basis": "measured copy bandwidth" if peak else None,
            "timing": "the whole propagate call (observables kernels included)"}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def visible_gpu_id(local_rank: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = cw.get(args.workload)
    cores = host_cores()
    steps_per_sample = args.ref_steps
    for _ in range(args.warmup):
        oracle_sample(w.name, cores, steps_per_sample)
    vals, singles = [], []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        v, units, wall, single = oracle_sample(w.name, cores, steps_per_sample)
        vals.append((units, wall))
        singles.append(single)
    units = sum(u for u, _ in vals)
    wall = sum(t for _, t in vals)
    value = units / wall
    sample = (f"{cores} realizations (one per host core) x {steps_per_sample} of "
              f"{w.n_steps} steps of {w.name} per bench step, K={w.K}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "m": w.m, "N": w.N, "R": w.R,
                                         "K": w.K, "dt": w.dt, "n_steps": w.n_steps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "single_core_value": statistics.median(singles), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t_all,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def ragged_leg(args, dev, stream):
    """The batching workload at full size: 2048 realizations of two walkers on
    open chains of N in {128, 192, ..., 1024} drawn per realization, 1000
    steps, K from the order autotuner over 8..20, observables every 10
    steps, complex FP32 on the library's default path (temporally blocked
    register tiles).  One timed call after a short warm-up call."""
    import numpy as np
    import torch

    from paper_1612_00746_gb300 import ctqw

    w = cw.get("ragged_n128_1024")
    u_eps, u_J, sizes, _ = cw.packed_draws(w)
    h = ctqw.Hamiltonian(w.m, w.statistics, w.periodic, sizes, w.J0, w.U, w.eps_halfwidth,
                         w.J_halfwidth, u_eps, u_J)
    K = ctqw.ctqw_autotune_order(h, ctqw.C64, w.dt, w.n_steps, 8, 20)
    psi = h.new_state(ctqw.C64, dev)
    sites = ctqw.initial_sites(w, h)
    n_obs = h.n_obs(w.n_steps, w.obs_every)
    P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device=dev)
    nr = torch.empty((n_obs, h.R), dtype=torch.float64, device=dev)
    en = torch.empty((n_obs, h.R), dtype=torch.float64, device=dev)
    ws = h.workspace(ctqw.C64, ctqw.TAYLOR, 0, dev)
    ctqw.ctqw_init_state(h, psi, sites, ctqw.C64)
    ctqw.ctqw_propagate_taylor(h, psi, ctqw.C64, w.dt, K, 20, w.obs_every, P, nr, en, 0, ws)
    torch.cuda.synchronize()
    ctqw.ctqw_init_state(h, psi, sites, ctqw.C64)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(visible_gpu_id(0))
    clocks.start()
    e0.record(stream)
    ctqw.ctqw_propagate_taylor(h, psi, ctqw.C64, w.dt, K, w.n_steps, w.obs_every, P, nr, en, 0, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ctqw.ctqw_check_status(h)
    ms = e0.elapsed_time(e1)
    D = float(np.sum(sizes.astype(np.float64) ** w.m))
    units = D * K * w.n_steps
    wk = w.with_(K=K)
    roof = roofline_of(wk, ctqw.C64, 0, units, ms, measured_peaks(), None)
    roof["timing"] = "the whole propagate call (tile launches and the reductions of 101 samples)"
    launches8 = -(-K // 8)
    depth = -(-K // launches8)
    groups_per_launch = 1 if len(h.group_sizes) <= 32 else len(h.group_sizes)   # all groups in one launch
    launches = 1 + w.n_steps * (-(-K // depth)) * groups_per_launch + n_obs + 1
    out = {"workload": w.name, "value": units / (ms / 1000.0), "unit": UNIT, "ms": ms,
           "R": w.R, "sizes": "N in {128, 192, ..., 1024} per realization (15 groups)",
           "K": K, "K_range": [8, 20], "n_steps": w.n_steps, "obs_every": w.obs_every,
           "site_updates": units, "gpu_launches": launches,
           "norm_drift": float((nr - 1.0).abs().max().item()),
           "roofline": roof, "clocks": clk,
           "l2": "inputs larger than L2 (states %.1f GB)" % (D * 8 / 1e9)}
    h.close()
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1612_00746_gb300 import ctqw
    from paper_1612_00746_gb300.ensemble import combine_means, max_over_ranks

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    set_sm_count(dev)
    ctqw.load()

    w = cw.get(args.workload)
    if args.realizations:
        w = w.with_(R=args.realizations)
    if args.n_steps:
        w = w.with_(n_steps=args.n_steps)
    # cpu baseline first (spawned workers, before heavy GPU use), rank 0 at N=1 only
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        v, units, wall, single = oracle_sample(w.name, cores, args.cpu_steps)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "single_core_value": single,
               "sample": f"{cores} realizations (one per host core) x {args.cpu_steps} of "
                         f"{w.n_steps} steps of {w.name}, K={w.K}, FP64 ({wall:.1f} s); "
                         f"single_core_value: median rate of one worker"}

    if not args.no_fma_peaks:
        FMA_PEAKS.update(measure_fma_peaks())

    # realizations of this rank: its own block of the (weakly scaled) ensemble
    realizations = list(range(rank * w.R, (rank + 1) * w.R))
    u_eps, u_J, sizes, _ = cw.packed_draws(w, realizations)
    dtype = w.dtype if not args.dtype else {"c64": ctqw.C64, "c128": ctqw.C128}[args.dtype]
    stream = torch.cuda.current_stream()
    h = ctqw.Hamiltonian(w.m, w.statistics, w.periodic, sizes, w.J0, w.U, w.eps_halfwidth,
                         w.J_halfwidth, u_eps, u_J)
    sites = ctqw.initial_sites(w, h)
    psi = h.new_state(dtype, dev)
    n_obs = h.n_obs(w.n_steps, w.obs_every)
    P = torch.empty((n_obs, h.p_width), dtype=torch.float64, device=dev)
    nr = torch.empty((n_obs, h.R), dtype=torch.float64, device=dev)
    en = torch.empty((n_obs, h.R), dtype=torch.float64, device=dev)
    D = float(np.sum(sizes.astype(np.float64) ** w.m))
    units_per_step = D * w.K * w.n_steps
    path = propagation_path(w, dtype, args.flags, args.switch is not None)
    ws = h.workspace(dtype, ctqw.TAYLOR, args.flags | (ctqw.FLAG_PLAIN if args.switch is not None else 0), dev)
    slots = 0
    if path == "rows" and w.obs_every > 0:
        # the fused path stores the state at sample points into workspace
        # slots: 1 + S states run S + 1 sampling intervals per launch
        state_bytes = int(D) * (8 if dtype == ctqw.C64 else 16)
        slots = max(2, min(n_obs - 1, args.snapshots, int(args.snapshot_gb * 1e9) // state_bytes))
        ws = torch.empty((1 + slots) * state_bytes, dtype=torch.uint8, device=dev)
    counts = torch.tensor(np.repeat(h.group_count, h.group_sizes), dtype=torch.float64, device=dev)
    if path == "wavefront":
        # init_state + one observables kernel per sample + one wavefront launch
        # per segment between samples and size group
        n_seg = -(-w.n_steps // w.obs_every) if w.obs_every else 1
        launches_per_step = 1 + n_obs + n_seg * len(h.group_sizes)
    elif path == "plain":
        # init_state + K stage launches per step + one observables kernel per sample
        launches_per_step = 1 + w.n_steps * w.K + n_obs
    elif path == "tiled":
        # ceil(K / D) launches per step and size group, observables, init
        launches8 = -(-w.K // 8)
        depth = {0: -(-w.K // launches8), 9: 4, 10: 8, 11: 8, 12: 4, 13: 8, 14: 2, 15: 7}[(args.flags >> 8) & 0xF]
        # register tiles run every size group in one launch (the shared-memory shapes one per group)
        shared_mem_shape = ((args.flags >> 8) & 0xF) == 9
        per_launch_groups = len(h.group_sizes) if shared_mem_shape or len(h.group_sizes) > 32 else 1
        launches_per_step = 1 + w.n_steps * (-(-w.K // depth)) * per_launch_groups + n_obs
    else:
        # init_state + one fused launch per S + 1 sampling intervals + one
        # reduction kernel per sample
        per_launch = (slots + 1) * w.obs_every if w.obs_every else w.n_steps
        launches_per_step = 1 + -(-w.n_steps // per_launch) + n_obs
    # the fused path's second stream: register tiles for the last realizations
    # (ceil(K / D) launches a step) and their own reduction per sample
    split = ctqw.ctqw_fused_split(h, w.K, args.flags) if path == "rows" and slots >= 2 else 0
    if split:
        tile_depth = -(-w.K // -(-w.K // 8))   # the stages split evenly over ceil(K / 8) launches
        launches_per_step += w.n_steps * -(-w.K // tile_depth) + n_obs
    if args.switch is not None:
        launches_per_step += 1 + w.n_steps   # parameter restore + one update per step
    launches_per_step += 1   # the norm check of the sampled norms

    prop_events = []
    graph = None
    if args.graph:
        # the propagate call (all its launches) captured once, replayed every step
        ctqw.ctqw_init_state(h, psi, sites, dtype)
        torch.cuda.synchronize()
        gs = torch.cuda.Stream()
        gs.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            ctqw.ctqw_propagate_taylor(h, psi, dtype, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en,
                                       args.flags, ws, stream=gs)
        stream.wait_stream(gs)
        torch.cuda.synchronize()

    def step(record=False):
        ctqw.ctqw_init_state(h, psi, sites, dtype)
        if record:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        if graph is not None:
            graph.replay()
        elif args.switch is not None:
            ctqw.ctqw_propagate_taylor_switching(h, psi, dtype, w.dt, w.K, w.n_steps, w.obs_every, P, nr,
                                                 en, 0x5EED, args.switch, args.flags, ws)
        else:
            ctqw.ctqw_propagate_taylor(h, psi, dtype, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en,
                                       args.flags, ws)
        if record:
            e1.record(stream)
            prop_events.append((e0, e1))
        if world > 1:
            combine_means(P, counts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(visible_gpu_id(local))
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        step(record=True)
    t1.record(stream)
    torch.cuda.synchronize()
    # the fused kernel alone (one launch over all steps and realizations, no
    # sampling, no second stream), for its roofline: the timed calls above
    # interleave it with the reductions and the second stream's tiles
    kernel_alone_ms = None
    one_stream = None
    if path == "rows" and graph is None:
        ctqw.ctqw_init_state(h, psi, sites, dtype)
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        ctqw.ctqw_propagate_taylor(h, psi, dtype, w.dt, w.K, w.n_steps, 0, None, None, None,
                                   args.flags | ctqw.FLAG_ONE_STREAM, ws)
        k1.record(stream)
        torch.cuda.synchronize()
        kernel_alone_ms = k0.elapsed_time(k1)
        if split:
            # the same bench step with every realization on the clusters
            ctqw.ctqw_init_state(h, psi, sites, dtype)
            k0.record(stream)
            ctqw.ctqw_propagate_taylor(h, psi, dtype, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en,
                                       args.flags | ctqw.FLAG_ONE_STREAM, ws)
            k1.record(stream)
            torch.cuda.synchronize()
            one_ms = k0.elapsed_time(k1)
            one_stream = {"value": world * units_per_step / (one_ms / 1000.0), "ms": one_ms,
                          "what": "the same step, every realization on the clusters (CTQW_FLAG_ONE_STREAM)"}
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = t0.elapsed_time(t1) / args.steps
    ms_max = max_over_ranks(ms, dev)
    value = world * units_per_step / (ms_max / 1000.0)
    prop_ms = [a.elapsed_time(b) for a, b in prop_events]
    kernel_ms = statistics.mean(prop_ms)

    # accuracy self-check of this run (rank 0's realizations): norm drift
    norm_drift = float((nr - 1.0).abs().max().item())

    # end to end: host draws -> build (H2D) -> init -> propagate -> D2H results
    pin = lambda a: torch.from_numpy(a).pin_memory()
    ue_p, uj_p = pin(u_eps), pin(u_J)
    h2d = ue_p.numel() * 8 + uj_p.numel() * 8 + sites.size * 4
    d2h = (P.numel() + nr.numel() + en.numel()) * 8
    P_host = torch.empty(P.shape, dtype=P.dtype).pin_memory()
    n_host = torch.empty(nr.shape, dtype=nr.dtype).pin_memory()
    e_host = torch.empty(en.shape, dtype=en.dtype).pin_memory()

    def e2e_step():
        h2 = ctqw.Hamiltonian(w.m, w.statistics, w.periodic, sizes, w.J0, w.U, w.eps_halfwidth,
                              w.J_halfwidth, ue_p.numpy(), uj_p.numpy())
        ctqw.ctqw_init_state(h2, psi, sites, dtype)
        ctqw.ctqw_propagate_taylor(h2, psi, dtype, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en,
                                   args.flags, ws)
        P_host.copy_(P, non_blocking=True)
        n_host.copy_(nr, non_blocking=True)
        e_host.copy_(en, non_blocking=True)
        torch.cuda.synchronize()
        h2.close()

    e2e = None
    if not args.no_e2e:
        e2e_steps = max(1, min(args.steps, 3))
        e2e_step()
        torch.cuda.synchronize()
        te = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        e2e_s = max_over_ranks((time.perf_counter() - te) / e2e_steps, dev)
        e2e = {"value": world * units_per_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # plain per-term FP64 path on a subset (the comparison path of the metric)
    fp64 = None
    plain32 = None
    peaks = measured_peaks()
    if not args.no_fp64_plain and rank == 0:
        sub = list(range(args.fp64_realizations))
        ue_s, uj_s, sz_s, _ = cw.packed_draws(w, sub)
        hs = ctqw.Hamiltonian(w.m, w.statistics, w.periodic, sz_s, w.J0, w.U, w.eps_halfwidth,
                              w.J_halfwidth, ue_s, uj_s)
        psi64 = hs.new_state(ctqw.C128, dev)
        ws64 = hs.workspace(ctqw.C128, ctqw.TAYLOR, ctqw.FLAG_PLAIN, dev)
        steps64 = args.fp64_steps
        nobs64 = hs.n_obs(steps64, w.obs_every)
        P64 = torch.empty((nobs64, hs.p_width), dtype=torch.float64, device=dev)
        sites_s = ctqw.initial_sites(w, hs)
        ctqw.ctqw_init_state(hs, psi64, sites_s, ctqw.C128)
        ctqw.ctqw_propagate_taylor(hs, psi64, ctqw.C128, w.dt, w.K, 2, w.obs_every, None, None,
                                   None, ctqw.FLAG_PLAIN, ws64)
        torch.cuda.synchronize()
        ctqw.ctqw_init_state(hs, psi64, sites_s, ctqw.C128)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ctqw.ctqw_propagate_taylor(hs, psi64, ctqw.C128, w.dt, w.K, steps64, w.obs_every, P64,
                                   None, None, ctqw.FLAG_PLAIN, ws64)
        a1.record(stream)
        torch.cuda.synchronize()
        ms64 = a0.elapsed_time(a1)
        units64 = float(np.sum(sz_s.astype(np.float64) ** w.m)) * w.K * steps64
        # same subset, same steps, fused FP32: agreement of the ensemble mean
        psi32 = hs.new_state(ctqw.C64, dev)
        P32 = torch.empty_like(P64)
        ctqw.ctqw_init_state(hs, psi32, sites_s, ctqw.C64)
        ctqw.ctqw_propagate_taylor(hs, psi32, ctqw.C64, w.dt, w.K, steps64, w.obs_every, P32,
                                   None, None, 0, None)
        torch.cuda.synchronize()
        dP = float((P32 - P64).abs().max().item())
        # the plain per-term path in FP32: HBM-bound.  Its K-1 Horner stages
        # read w and psi and write w (24 bytes per amplitude); the last reads
        # w, psi and the rounding word and writes psi and the rounding word
        # (40 bytes).  On enough realizations that the three states exceed L2.
        sub32 = list(range(min(w.R, args.plain32_realizations)))
        ue3, uj3, sz3, _ = cw.packed_draws(w, sub32)
        h32 = ctqw.Hamiltonian(w.m, w.statistics, w.periodic, sz3, w.J0, w.U, w.eps_halfwidth,
                               w.J_halfwidth, ue3, uj3)
        psi32p = h32.new_state(ctqw.C64, dev)
        ws32 = h32.workspace(ctqw.C64, ctqw.TAYLOR, ctqw.FLAG_PLAIN, dev)
        ctqw.ctqw_init_state(h32, psi32p, ctqw.initial_sites(w, h32), ctqw.C64)
        ctqw.ctqw_propagate_taylor(h32, psi32p, ctqw.C64, w.dt, w.K, 2, 0, None, None, None,
                                   ctqw.FLAG_PLAIN, ws32)
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        ctqw.ctqw_propagate_taylor(h32, psi32p, ctqw.C64, w.dt, w.K, steps64, 0, None, None, None,
                                   ctqw.FLAG_PLAIN, ws32)
        b1.record(stream)
        torch.cuda.synchronize()
        ms32p = b0.elapsed_time(b1)
        units32 = float(np.sum(sz3.astype(np.float64) ** w.m)) * w.K * steps64
        bpu = ((w.K - 1) * 24.0 + 40.0) / w.K
        gbs = units32 * bpu / (ms32p / 1000.0) / 1e9
        plain32 = {"value": units32 / (ms32p / 1000.0), "unit": UNIT, "bound": "hbm",
                   "achieved_gbs": gbs, "peak_gbs": peaks.get("hbm_gbs"),
                   "frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
                   "bytes_per_site_update": bpu,
                   "sample": f"{len(sub32)} realizations x {steps64} steps "
                             f"({3 * float(np.sum(sz3.astype(np.float64) ** w.m)) * 8 / 1e6:.0f} MB of states), "
                             "horner_stage_kernel<2> + horner_final_kernel<2>"}
        h32.close()
        fp64 = {"value": units64 / (ms64 / 1000.0), "unit": UNIT,
                "sample": f"{len(sub)} realizations x {steps64} steps, plain per-term FP64 kernels",
                "fp32_speedup": value / world / (units64 / (ms64 / 1000.0)),
                "max_abs_dP_fp32_vs_fp64": dP}
        hs.close()

    peaks = measured_peaks()
    roofline = roofline_of(w, dtype, args.flags, units_per_step,
                           kernel_alone_ms if kernel_alone_ms is not None else kernel_ms, peaks,
                           fused_traffic(w.name) if not (args.realizations or args.n_steps or args.switch) else None,
                           switching=args.switch is not None)
    if kernel_alone_ms is not None:
        roofline["timing"] = ("one launch of the fused kernel over all steps without sampling "
                              "(CUDA events, after the timed region)")
        roofline["achieved_with_sampling"] = units_per_step * (8 * w.m + 4) / (kernel_ms / 1000.0) / 1e12
        roofline["snapshot_slots"] = slots

    ragged = density = adjoint = None
    full_default = world == 1 and rank == 0 and args.workload == "bosons_n256_u2" \
        and not (args.realizations or args.n_steps or args.switch or args.graph)
    if full_default and not args.no_ragged:
        ragged = ragged_leg(args, dev, stream)
    if full_default and not args.no_extra_legs:
        # the one-body density matrix on the tensor cores (states of this
        # workload after 100 steps) and the adjoint gradient at full size
        import types
        d = rho1_line(types.SimpleNamespace(workload="bosons_n256_u2", realizations=0, n_steps=0,
                                            steps=5, warmup=2))
        density = {k: d[k] for k in ("metric", "value", "unit", "ms_per_step", "roofline", "cuda_cores",
                                     "speedup_over_cuda_cores", "max_abs_diff_tc_vs_cuda_cores_rel")}
        a = adjoint_line(types.SimpleNamespace(workload="adjoint_n512", realizations=0, n_steps=0,
                                               steps=1, warmup=1))
        adjoint = {k: a[k] for k in ("metric", "value", "unit", "ms_per_step", "config", "forward_ms",
                                     "adjoint_over_forward")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "propagate_ms": {"best": min(prop_ms), "median": statistics.median(prop_ms),
                         "mean": kernel_ms, "steps": len(prop_ms)},
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if dtype == ctqw.C64 else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "N": w.N, "R_per_gpu": w.R, "K": w.K,
                   "dt": w.dt, "n_steps": w.n_steps, "obs_every": w.obs_every,
                   "statistics": "bosons" if w.statistics == cw.BOSONS else "distinguishable",
                   "precision": ("complex FP32, compensated state update, FP64 reductions"
                                 if dtype == ctqw.C64 else "complex FP64"),
                   "l2": "inputs larger than L2 (states %.0f MB per GPU)" % (D * (8 if dtype == ctqw.C64 else 16) / 1e6),
                   "parallelism": f"realizations sharded, {world} rank(s)",
                   "launch": "cuda graph replay" if args.graph else "eager",
                   "switching_noise_p": args.switch},
        "gpu_launches": launches_per_step * args.steps,
        "fused_split": ({"clusters_realizations": w.R - split, "tiles_realizations": split,
                         "what": "the last realizations on the register tiles on a second stream, "
                                 "on the SMs no 16-CTA cluster can hold"} if path == "rows" else None),
        "one_stream": one_stream,
        "roofline": roofline,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "fp64_plain": fp64,
        "plain_fp32_hbm": plain32,
        "ragged_batch": ragged,
        "density_tensor_cores": density,
        "adjoint": adjoint,
        "norm_drift": norm_drift,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_adjoint(args):
    """Print the adjoint_line JSON line."""
    print(json.dumps(adjoint_line(args)), flush=True)
    return 0


def adjoint_line(args):
    """Time ctqw_adjoint_grad (loss on Pbar(x, T) and its gradient) on one GPU.

    Reported as forward-equivalent site-updates/s (N^m K steps R of the
    forward map per call), next to the forward pass alone on the same inputs.
    """
    import numpy as np
    import torch

    from paper_1612_00746_gb300 import ctqw

    torch.cuda.set_device(0)
    set_sm_count(0)
    dev = torch.device("cuda", 0)
    ctqw.load()
    w = cw.get(args.workload)
    if args.realizations:
        w = w.with_(R=args.realizations)
    if args.n_steps:
        w = w.with_(n_steps=args.n_steps)
    M = 50
    u_eps, u_J, sizes, _ = cw.packed_draws(w, list(range(w.R)))
    em, jm = np.zeros(w.N), np.full(w.N, w.J0)
    h = ctqw.Hamiltonian(w.m, w.statistics, w.periodic, sizes, w.J0, w.U, w.eps_halfwidth,
                         w.J_halfwidth, u_eps, u_J, eps_mean=em, J_mean=jm)
    psi = h.new_state(ctqw.C64, dev)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), ctqw.C64)
    target = torch.full((h.p_width,), 1.0 / w.N, dtype=torch.float64, device=dev)
    ws = ctqw.adjoint_workspace(h, ctqw.C64, w.K, w.n_steps, M, dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ctqw.ctqw_adjoint_grad(h, psi, ctqw.C64, w.dt, w.K, w.n_steps, M, target, workspace=ws,
                               per_realization=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        loss, _, _, _, gem, gJm = ctqw.ctqw_adjoint_grad(h, psi, ctqw.C64, w.dt, w.K, w.n_steps, M,
                                                         target, workspace=ws, per_realization=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the forward pass alone on the library's default path for this handle
    fws = h.workspace(ctqw.C64, ctqw.TAYLOR, 0, dev)
    scratch = psi.clone()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    ctqw.ctqw_propagate_taylor(h, scratch, ctqw.C64, w.dt, w.K, w.n_steps, 0, None, None, None, 0, fws)
    f1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1)
    units = float(np.sum(sizes.astype(np.float64) ** w.m)) * w.K * w.n_steps
    line = {
        "metric": METRIC + ", forward-equivalent, adjoint gradient", "value": units / (ms / 1000.0),
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "N": w.N, "R": w.R, "K": w.K, "n_steps": w.n_steps,
                   "checkpoint_every": M, "precision": "c64 states, FP64 gradient accumulation"},
        "forward_ms": fwd_ms, "adjoint_over_forward": ms / fwd_ms,
        "loss": float(loss.item()), "grad_abs_max": float(max(gem.abs().max().item(), gJm.abs().max().item())),
    }
    h.close()
    del ws, fws, scratch, psi
    torch.cuda.empty_cache()
    return line


def run_rho1(args):
    """Print the rho1_line JSON line."""
    print(json.dumps(rho1_line(args)), flush=True)
    return 0


def rho1_line(args):
    """Time ctqw_one_body_density (ensemble-averaged one-body density matrix)
    on the workload's states after a short propagation, on the tensor cores
    (c64, the default where supported) and on the CUDA cores.

    Algorithmic flops per call: m N^(m+1) R complex multiply-adds, 8 real
    flops each.  The CUDA-core kernel is measured against the FP32 FMA peak.
    The tensor-core kernel computes the 128 x 128 tiles of the upper
    triangle only (the rest is their conjugate transpose) and forms every
    real product from three TF32 piece products: per size group it runs
    n_up 128^2 K 24 flops on the TF32 tensor pipe (n_up = T (T + 1) / 2
    tiles, T = ceil(N / 128), K = R_g m N^(m-1)), whose peak is the measured
    BF16 GEMM rate times the nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s).
    The call's time (slot clearing, the tensor-core kernel, the FP64 sum of
    the slots) is the denominator, so the kernel's own rate is higher by
    the share the launch list gives it.
    """
    import numpy as np
    import torch

    from paper_1612_00746_gb300 import ctqw

    torch.cuda.set_device(0)
    set_sm_count(0)
    dev = torch.device("cuda", 0)
    ctqw.load()
    w = cw.get(args.workload)
    if args.realizations:
        w = w.with_(R=args.realizations)
    u_eps, u_J, sizes, _ = cw.packed_draws(w, list(range(w.R)))
    h = ctqw.Hamiltonian(w.m, w.statistics, w.periodic, sizes, w.J0, w.U, w.eps_halfwidth,
                         w.J_halfwidth, u_eps, u_J)
    psi = h.new_state(ctqw.C64, dev)
    ctqw.ctqw_init_state(h, psi, ctqw.initial_sites(w, h), ctqw.C64)
    ws = h.workspace(ctqw.C64, ctqw.TAYLOR, 0, dev)
    ctqw.ctqw_propagate_taylor(h, psi, ctqw.C64, w.dt, w.K, 100, 0, None, None, None, 0, ws)
    stream = torch.cuda.current_stream()
    flops = float(np.sum(w.m * sizes.astype(np.float64) ** (w.m + 1))) * 8.0
    tensor_flops = 0.0
    for N_g in np.unique(sizes):
        T = (int(N_g) + 127) // 128
        K_g = float(np.sum(sizes == N_g)) * w.m * float(N_g) ** (w.m - 1)
        tensor_flops += T * (T + 1) / 2 * 128.0 ** 2 * K_g * 24.0
    peaks = measured_peaks()

    def timed(method):
        ctqw.ctqw_set_density_method(h, method)
        for _ in range(args.warmup):
            ctqw.ctqw_one_body_density(h, psi, ctqw.C64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            rho = ctqw.ctqw_one_body_density(h, psi, ctqw.C64)
        e1.record(stream)
        torch.cuda.synchronize()
        ctqw.ctqw_check_status(h)
        return e0.elapsed_time(e1) / args.steps, rho

    ms_tc, rho_tc = timed(0)
    ms_cc, rho_cc = timed(1)
    diff = max(float((a - b).abs().max().item()) for a, b in zip(rho_tc, rho_cc))
    big = max(float(b.abs().max().item()) for b in rho_cc)
    alg_tc = flops / (ms_tc / 1000.0) / 1e12
    alg_cc = flops / (ms_cc / 1000.0) / 1e12
    tf32_peak = peaks["bf16_tflops"] * 1.1 / 2.25 if peaks.get("bf16_tflops") else 1900.0 * 1.1 / 2.25
    tensor = tensor_flops / (ms_tc / 1000.0) / 1e12
    trace = float(sum(torch.diagonal(r).real.sum().item() for r in rho_tc))
    line = {
        "metric": "one-body density matrix of the ensemble, TFLOP/s (algorithmic)", "value": alg_tc,
        "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_tc,
        "higher_is_better": True, "dtype": "f32 (TF32 x3 pieces)", "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "N": w.N, "R": w.R, "states_after_steps": 100},
        "roofline": {"bound": "tensor", "achieved": tensor, "peak": tf32_peak, "unit": "TFLOP/s",
                     "frac": tensor / tf32_peak, "kernel": "rho1_tc_kernel (tcgen05 kind::tf32)",
                     "tensor_flops_per_call": tensor_flops, "timed": "whole call",
                     "peak_basis": ("measured BF16 GEMM burst x 1.1/2.25 (nominal TF32/BF16)"
                                    if peaks.get("bf16_tflops") else "fallback 1.9 PF/s BF16 x 1.1/2.25")},
        "cuda_cores": {"ms": ms_cc, "achieved": alg_cc, "peak": alu_peak(), "frac": alg_cc / alu_peak(),
                       "kernel": "rho1_term_kernel<float>"},
        "speedup_over_cuda_cores": ms_cc / ms_tc,
        "max_abs_diff_tc_vs_cuda_cores_rel": diff / big if big else None,
        "trace_sum_over_groups": trace,
    }
    h.close()
    del psi, ws
    torch.cuda.empty_cache()
    return line


def run_lattice(args):
    """Time ctqw_graph_propagate_taylor on a q-dimensional lattice / graph
    workload (default: two bosons on the 15 x 15 torus, 1000 realizations).

    Per-term kernels stream the states through HBM: per site-update
    ((K-1) 24 + 40) / K bytes in FP32 (Horner stages and the compensated
    final stage), the neighbour reads served from L1/L2.
    """
    import torch

    from paper_1612_00746_gb300 import ctqw

    torch.cuda.set_device(0)
    set_sm_count(0)
    dev = torch.device("cuda", 0)
    ctqw.load()
    w = cw.get_graph(args.lattice)
    if args.realizations:
        w = w.with_(R=args.realizations)
    if args.n_steps:
        w = w.with_(n_steps=args.n_steps)
    if args.dtype:
        w = w.with_(dtype=cw.C64 if args.dtype == "c64" else cw.C128)
    g = ctqw.Graph.from_workload(w)
    if args.chunk:
        ctqw.ctqw_graph_set_chunk(g, args.chunk)
    psi = g.new_state(w.dtype, dev)
    ws = g.workspace(w.dtype, dev)
    n_obs = g.n_obs(w.n_steps, w.obs_every)
    P = torch.empty((n_obs, g.N), dtype=torch.float64, device=dev)
    nr = torch.empty((n_obs, g.R), dtype=torch.float64, device=dev)
    en = torch.empty((n_obs, g.R), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ctqw.ctqw_graph_init_state(g, psi, w.sites, w.dtype)
        ctqw.ctqw_graph_propagate_taylor(g, psi, w.dtype, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en,
                                         workspace=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(visible_gpu_id(0))
    clocks.start()
    total = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        ctqw.ctqw_graph_init_state(g, psi, w.sites, w.dtype)
        torch.cuda.synchronize()
        e0.record(stream)
        ctqw.ctqw_graph_propagate_taylor(g, psi, w.dtype, w.dt, w.K, w.n_steps, w.obs_every, P, nr, en,
                                         workspace=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    clk = clocks.stop()
    ms = total / args.steps
    units = w.site_updates()
    value = units / (ms / 1000.0)
    drift = float((nr[-1] - 1.0).abs().max().item()) if n_obs else None
    peaks = measured_peaks()
    if w.dtype == cw.C64:
        bpu = ((w.K - 1) * 24.0 + 40.0) / w.K
        gbs = units * bpu / (ms / 1000.0) / 1e9
        peak = peaks.get("hbm_gbs")
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                "frac": gbs / peak if peak else None, "traffic": None,
                "kernel": "graph_horner_stage_kernel + graph_horner_final_kernel",
                "kernel_ms": ms, "bytes_per_site_update": bpu,
                "peak_basis": "measured copy bandwidth" if peak else None,
                "timing": "the whole propagate call (observables kernels included)"}
    else:
        flops = 8 * w.m + 4
        ach = units * flops / (ms / 1000.0) / 1e12
        peak = alu_peak(fp64=True)
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": "graph_taylor_term_kernel<double>", "kernel_ms": ms,
                "peak_basis": f"{SM_COUNT} SMs x 2 DFMA x 2 flop x 2070 MHz (FP64, derived)"}
    line = {
        "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "dtype": "c64" if w.dtype == cw.C64 else "c128", "data": "synthetic",
        "config": {"workload": w.name, "shape": list(w.shape), "periodic": w.periodic, "m": w.m,
                   "chunk": args.chunk or "all realizations in one pass",
                   "N": w.n_nodes(), "links": int(len(w.edges()[0])), "R": w.R, "K": w.K,
                   "n_steps": w.n_steps, "obs_every": w.obs_every,
                   "l2": "states larger than L2" if g.total_amplitudes * 8 > 129e6 else "L2-resident"},
        "roofline": roof, "norm_drift": drift, "clocks": clk,
        "gpu_launches": int(args.steps * (w.n_steps * w.K + n_obs + 1)),
    }
    print(json.dumps(line), flush=True)
    g.close()
    return 0


def run_exact(args):
    """Time ctqw_propagate_exact (batched Jacobi diagonalisation, FP64) on many
    small realizations: 2 particles, N = 8 (D = 64), 4096 realizations.

    Algorithmic flops: the Jacobi sweeps, about 9 D^3 each (every pair
    rotation updates two rows and two columns of H and two columns of W,
    6 flops per element), against the FP64 pipe (2 DFMA per SM per cycle).
    """
    import numpy as np
    import torch

    from paper_1612_00746_gb300 import ctqw

    torch.cuda.set_device(0)
    set_sm_count(0)
    dev = torch.device("cuda", 0)
    ctqw.load()
    R = args.realizations or 4096
    w = cw.Workload(name="exact_n8_m2", m=2, statistics=cw.BOSONS, periodic=False, N=8, R=R, J0=1.0,
                    U=2.0, eps_halfwidth=1.0, J_halfwidth=0.25, sites=(3, 4), dt=0.05, K=16,
                    n_steps=100, obs_every=10, dtype=cw.C128, seed=0)
    u_eps, u_J, sizes, _ = cw.packed_draws(w, list(range(w.R)))
    h = ctqw.Hamiltonian(w.m, w.statistics, w.periodic, sizes, w.J0, w.U, w.eps_halfwidth,
                         w.J_halfwidth, u_eps, u_J)
    psi = h.new_state(ctqw.C128, dev)
    sites = ctqw.initial_sites(w, h)
    P = torch.empty((h.n_obs(w.n_steps, w.obs_every), h.p_width), dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        ctqw.ctqw_init_state(h, psi, sites, ctqw.C128)
        sweeps = ctqw.ctqw_propagate_exact(h, psi, w.dt, w.n_steps, w.obs_every, P)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    for _ in range(args.steps):
        ctqw.ctqw_init_state(h, psi, sites, ctqw.C128)
        torch.cuda.synchronize()
        e0.record(stream)
        sweeps = ctqw.ctqw_propagate_exact(h, psi, w.dt, w.n_steps, w.obs_every, P)
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    ms = total / args.steps
    D = w.N ** w.m
    flops = 9.0 * D ** 3 * float(np.sum(sweeps))
    peak = alu_peak(fp64=True)
    achieved = flops / (ms / 1000.0) / 1e12
    line = {
        "metric": "realizations diagonalised and propagated per second", "value": R / (ms / 1000.0),
        "unit": "realizations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "N": w.N, "D": D, "R": R, "samples": h.n_obs(w.n_steps, w.obs_every)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "kernel": "exact_eigen_kernel",
                     "peak_basis": f"{SM_COUNT} SMs x 2 DFMA x 2 flop x 2070 MHz (FP64, derived)"},
        "jacobi_sweeps_mean": float(np.mean(sweeps)), "jacobi_sweeps_max": int(np.max(sweeps)),
    }
    print(json.dumps(line), flush=True)
    h.close()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="bosons_n256_u2")
    ap.add_argument("--cpu-steps", type=int, default=120, help="steps per realization of the CPU baseline")
    ap.add_argument("--ref-steps", type=int, default=60, help="steps per realization per reference step")
    ap.add_argument("--fp64-realizations", type=int, default=16)
    ap.add_argument("--fp64-steps", type=int, default=100)
    ap.add_argument("--plain32-realizations", type=int, default=256,
                    help="realizations of the FP32 per-term HBM leg (states larger than L2)")
    ap.add_argument("--realizations", type=int, default=0, help="override R (small profiling cases)")
    ap.add_argument("--n-steps", type=int, default=0, help="override the workload's steps")
    ap.add_argument("--flags", type=int, default=0, help="ctqw propagation flags (e.g. 4 = wide CTA)")
    ap.add_argument("--dtype", choices=["c64", "c128"], default=None, help="override the workload's type")
    ap.add_argument("--graph", action="store_true", help="replay the propagate call from a CUDA graph")
    ap.add_argument("--switch", type=float, default=None,
                    help="propagate with switching noise: redraw probability per parameter and step")
    ap.add_argument("--lattice", default=None,
                    help="time a q-dimensional lattice / graph workload (e.g. lattice2d_15x15_m2)")
    ap.add_argument("--chunk", type=int, default=0,
                    help="--lattice: realizations per pass (0: all in one pass)")
    ap.add_argument("--exact", action="store_true",
                    help="time ctqw_propagate_exact (batched Jacobi, 4096 x N=8 two-particle states)")
    ap.add_argument("--rho1", action="store_true",
                    help="time ctqw_one_body_density on the workload's states")
    ap.add_argument("--adjoint", action="store_true",
                    help="time ctqw_adjoint_grad on the workload (use --workload adjoint_n512)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-plain", action="store_true")
    ap.add_argument("--no-ragged", action="store_true", help="skip the full-size ragged-batch leg")
    ap.add_argument("--no-fma-peaks", action="store_true", help="skip the FMA-chain peak measurement")
    ap.add_argument("--no-extra-legs", action="store_true",
                    help="skip the one-body density and adjoint legs of the default line")
    ap.add_argument("--snapshots", type=int, default=24,
                    help="fused path: sample snapshots per launch (workspace of 1 + S states)")
    ap.add_argument("--snapshot-gb", type=float, default=16.0, help="cap of the snapshot workspace")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.adjoint:
        return run_adjoint(args)
    if args.rho1:
        return run_rho1(args)
    if args.exact:
        return run_exact(args)
    if args.lattice:
        return run_lattice(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
