#!/usr/bin/env python3
"""Benchmark of the essentially entropic lattice Boltzmann step on GB300.

Workload: D3Q27, 256^3 periodic Taylor-Green vortex (u0 = 0.05, beta = 0.999),
FP32 structure-of-arrays populations in ping-pong buffers; one "step" is one
time step of the whole hot path (the fused pull-stream + collide kernel); the
first step of every 100 also takes the FP64 diagnostics (mass, momentum, H,
alpha statistics, per-node H[f*] - H[f]) in the same pass.  Metric: MLUPS (million lattice-node updates per
second), and the fused kernel's fraction of the measured HBM bandwidth.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Defaults: K = 5000 (the length of the Taylor-Green configuration; the step gets
costlier as the vortex breaks down, so K decides what is measured), W = 20.

N > 1 runs under torch.distributed.run as independent replicas (one full
domain per GPU; the domain is not split across GPUs) and reports the aggregate.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L = 256
BETA = 0.999
U0 = 0.05
LATTICE_Q = 27
DIAG_EVERY = 100
FLOW_STEPS = 5000  # length of the Taylor-Green configuration
E2E_CALLS = 3  # end-to-end calls timed; the median is reported
STORAGE = "f32"
ELEM_BYTES = {"f32": 4, "f32dev": 4, "f16dev": 2, "bf16dev": 2}
WORKLOAD = "D3Q27 256^3 periodic Taylor-Green vortex, u0=0.05, beta=0.999, FP32 SoA ping-pong"
METRIC = "MLUPS (D3Q27 256^3 FP32 entropic LBM step)"
PROFILE = os.path.join(ROOT, "profiles", "k_step_d3q27_f32_tgv256.md")
KERNEL_SOURCES = ["paper_2203_12946_gb300/csrc/elbm_device.cuh",
                  "paper_2203_12946_gb300/csrc/elbm_kernels.cuh"]


def set_side(side: int) -> None:
    """Smaller cubes for profiling captures; the reported workload string follows."""
    global L, WORKLOAD, METRIC
    L = int(side)
    WORKLOAD = WORKLOAD.replace("256^3", f"{L}^3")
    METRIC = METRIC.replace("256^3", f"{L}^3")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profiled_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    if not os.path.exists(PROFILE):
        return None
    txt = open(PROFILE).read()
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    m_bytes = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
    if not (m_hash and m_bytes) or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_bytes.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.uuid:
            cmd.insert(1, f"--id={self.uuid}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Replicas:
    """Independent replicas, one per rank: the only collectives are the barrier around the
    timed region and the max over ranks of its duration (no data-path exchange)."""

    def __init__(self, backend: str, device=None):
        self.world, self.rank, self.local = dist_env()
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            kw = {"device_id": device} if (backend == "nccl" and device is not None) else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if not self.dist:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64,
                         device=self.device if self.device is not None else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.barrier()
            self.dist.destroy_process_group()
            self.dist = None


def xmax_bands(d: dict, N: int) -> dict:
    """Shares of nodes by |x|max of the next collision (the diagnostics' bands)."""
    names = ["cutoff_lt_1e-3", "short_series_lt_5e-3", "long_series_lt_4e-2", "per_population_ge_4e-2"]
    return {k: v / N for k, v in zip(names, d["n_xmax_band"])}


def e2e_itemised(E, sim, rho_h, u_h, rho_d, u_d, rho_out, u_out, barrier, h2d, d2h, reps: int = 3) -> dict:
    """The fixed cost of one end-to-end call, by part (median of a few repetitions): the
    initial state from host arrays and from device arrays, the moments into host and into
    device arrays, and plain copies of the same bytes between pinned host memory and the
    device (the library overlaps its copies with its kernels in node ranges, so the
    host-minus-device differences are the part of the copies left exposed)."""
    import torch

    def timed(fn):
        ts = []
        for _ in range(reps):
            barrier()
            t0 = time.perf_counter()
            fn()
            barrier()
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts))

    rho_dd = torch.empty_like(rho_d)
    u_dd = torch.empty_like(u_d)
    t_init_h = timed(lambda: E.elbm_init_equilibrium(sim.h, rho_h.numpy(), u_h.numpy(), E.ELBM_MEM_HOST))
    t_init_d = timed(lambda: E.elbm_init_equilibrium(sim.h, rho_d, u_d, E.ELBM_MEM_DEVICE))
    t_mom_h = timed(lambda: E.elbm_moments(sim.h, rho_out.numpy(), u_out.numpy(), E.ELBM_MEM_HOST))
    t_mom_d = timed(lambda: E.elbm_moments(sim.h, rho_dd, u_dd, E.ELBM_MEM_DEVICE))

    def h2d_copy():
        rho_dd.copy_(rho_h, non_blocking=True)
        u_dd.copy_(u_h, non_blocking=True)

    def d2h_copy():
        rho_out.copy_(rho_dd, non_blocking=True)
        u_out.copy_(u_dd, non_blocking=True)

    t_h2d, t_d2h = timed(h2d_copy), timed(d2h_copy)
    return {"init_from_host_ms": 1e3 * t_init_h, "init_from_device_ms": 1e3 * t_init_d,
            "moments_to_host_ms": 1e3 * t_mom_h, "moments_to_device_ms": 1e3 * t_mom_d,
            "h2d_copy_ms": 1e3 * t_h2d, "d2h_copy_ms": 1e3 * t_d2h,
            "h2d_gbs": h2d / t_h2d / 1e9, "d2h_gbs": d2h / t_d2h / 1e9,
            "note": "copy rates from plain pinned copies of the same bytes; the library overlaps its "
                    "copies with its kernels; staging allocated before timing"}


def late_flow_leg(E, sim, rho_d, u_d, one_step, barrier, steps: int, stream, N: int) -> dict:
    """K steps of the benchmark flow ending at step FLOW_STEPS, timed like the main region
    (per-launch CUDA events on the library's stream; the first of every DIAG_EVERY steps is
    the fused diagnostics step and is left out of the average)."""
    import torch

    E.elbm_init_equilibrium(sim.h, rho_d, u_d, E.ELBM_MEM_DEVICE)
    start_step = FLOW_STEPS - steps
    sim.step(start_step)
    d = sim.diagnostics()
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(steps):
        one_step(k, evs[k])
    b.record(stream)
    barrier()
    kern = [x.elapsed_time(y) for k, (x, y) in enumerate(evs) if k % DIAG_EVERY != 0]
    return {"steps": [start_step, FLOW_STEPS], "kernel_ms_avg": float(np.mean(kern)),
            "ms_per_step": a.elapsed_time(b) / steps, "mlups": N * steps / (a.elapsed_time(b) / 1e3) / 1e6,
            "xmax_band_frac": xmax_bands(d, N), "n_solved_frac": d["n_solved"] / N,
            "alpha_range": [d["alpha_min"], d["alpha_max"]]}


def aggregate_mlups(nodes_per_rank: int, steps: int, world: int, max_elapsed_s: float) -> float:
    """Whole-job throughput: node updates of all ranks over the slowest rank's time."""
    return world * nodes_per_rank * steps / max_elapsed_s / 1e6


# ----------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------

def oracle_prepare(slab: int):
    """A 256 x 256 x slab periodic slab of the 256^3 Taylor-Green field as oracle populations
    (same per-node work as the full domain)."""
    import oracle as O
    from paper_2203_12946_gb300 import inputs

    dims = (L, L, slab)
    X, Y, Z = inputs.grid(dims)
    rho, u = inputs.taylor_green_3d(X, Y, Z, L, u0=U0)
    return dims, O.init_equilibrium(3, rho, u)


def oracle_time(dims, f, nsteps: int, nthreads: int = 0):
    """Times nsteps oracle steps; returns (MLUPS, threads, seconds, description)."""
    import oracle as O

    t0 = time.perf_counter()
    O.step(3, dims, f, BETA, nsteps=nsteps, nthreads=nthreads)
    dt = time.perf_counter() - t0
    n = f.shape[1] * nsteps
    desc = (f"FP64 C oracle, {nsteps} step(s) of a 256x256x{dims[2]} periodic slab of the 256^3 "
            f"Taylor-Green field ({n} node updates)")
    return n / dt / 1e6, O.max_threads() if nthreads <= 0 else nthreads, dt, desc


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O

    O.build()
    threads = O.max_threads()
    # size the per-step sample so that warm-up + timed steps take about a minute
    probe_rate, _, _, _ = oracle_time(*oracle_prepare(2), 1)
    budget_nodes = probe_rate * 1e6 * 60.0 / max(1, args.steps + args.warmup)
    slab = int(max(1, min(L, budget_nodes // (L * L))))
    dims, f = oracle_prepare(slab)
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        oracle_time(dims, f, 1)
    total = 0.0
    desc = ""
    for _ in range(args.steps):
        _, _, dt, desc = oracle_time(dims, f, 1)
        total += dt
    value = L * L * slab * args.steps / total / 1e6
    wall = time.perf_counter() - t0
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"each step: one step of a 256x256x{slab} slab"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def run_gpu(args):
    import torch

    from paper_2203_12946_gb300 import elbm as E
    from paper_2203_12946_gb300 import inputs

    world, rank, local = dist_env()
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rep = Replicas("nccl", dev)
    E.load()

    dims = (L, L, L)
    N = L ** 3
    X, Y, Z = inputs.grid(dims)
    rho, u = inputs.taylor_green_3d(X, Y, Z, L, u0=U0)
    del X, Y, Z
    # pinned host copies for the end-to-end leg
    rho_h = torch.from_numpy(rho).pin_memory()
    u_h = torch.from_numpy(np.ascontiguousarray(u)).pin_memory()
    rho_d = rho_h.to(dev)
    u_d = u_h.to(dev)

    stream = torch.cuda.current_stream(dev)
    kernel = {"auto": E.ELBM_KERNEL_AUTO, "direct": E.ELBM_KERNEL_DIRECT, "rows": E.ELBM_KERNEL_ROWS}[args.kernel]
    sim = E.Simulation(E.ELBM_D3Q27, dims, BETA, storage=args.storage, device=local, stream=stream,
                       kernel=kernel)
    sim.init_equilibrium(rho_d, u_d)

    def barrier():
        torch.cuda.synchronize(dev)
        rep.barrier()
        torch.cuda.synchronize(dev)

    def one_step(k, ev=None):
        if k % DIAG_EVERY == 0:
            # the first step of every DIAG_EVERY also takes the FP64 diagnostics of the state
            # it advances (row a11), in the same pass over the populations; synchronising
            E.elbm_step_diag(sim.h, 1)
            return
        if ev is not None:
            ev[0].record(stream)
        sim.step(1)
        if ev is not None:
            ev[1].record(stream)

    for k in range(args.warmup):
        one_step(k)
    barrier()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    start.record(stream)
    for k in range(args.steps):
        one_step(k, evs[k])
    stop.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed = start.elapsed_time(stop) / 1e3
    kern = [a.elapsed_time(b) / 1e3 for k, (a, b) in enumerate(evs) if k % DIAG_EVERY != 0]
    kern_avg = float(np.mean(kern))  # the plain step launches (the fused ones carry the diagnostics)
    elapsed = rep.max(elapsed)
    gpu_launches = args.steps  # one step kernel per step; every DIAG_EVERY-th is the fused one
    d = sim.diagnostics(with_hist=True)
    hist = d["alpha_hist"]
    edges = np.linspace(1.9, 2.1, E.ELBM_HIST_BINS + 1)
    nz = np.nonzero(hist[1:-1])[0]
    alpha_hist = {"range": [1.9, 2.1], "bins": E.ELBM_HIST_BINS, "below": int(hist[0]), "above": int(hist[-1]),
                  "nonzero_bins": {"%.5f" % edges[b]: int(hist[1 + b]) for b in nz}}

    # End to end through the C ABI with host buffers: initial rho/u uploaded from pinned
    # host memory, K steps (with the diagnostics cadence), rho/u read back to host.  One
    # untimed round trip first: the library allocates its staging buffer on the first
    # host-memory call, and that allocation is not part of a step.
    rho_out = torch.empty(N, dtype=torch.float64).pin_memory()
    u_out = torch.empty((3, N), dtype=torch.float64).pin_memory()
    E.elbm_init_equilibrium(sim.h, rho_h.numpy(), u_h.numpy(), E.ELBM_MEM_HOST)
    E.elbm_moments(sim.h, rho_out.numpy(), u_out.numpy(), E.ELBM_MEM_HOST)
    # the whole call three times, the median reported (one call on a shared host can
    # stall for tens of milliseconds outside the library)
    runs = []
    for _ in range(E2E_CALLS):
        barrier()
        t0 = time.perf_counter()
        E.elbm_init_equilibrium(sim.h, rho_h.numpy(), u_h.numpy(), E.ELBM_MEM_HOST)
        t1 = time.perf_counter()
        for k in range(args.steps):
            one_step(k)
        t2 = time.perf_counter()
        E.elbm_moments(sim.h, rho_out.numpy(), u_out.numpy(), E.ELBM_MEM_HOST)
        barrier()
        t3 = time.perf_counter()
        runs.append((rep.max(t3 - t0), t0, t1, t2, t3))
    runs.sort()
    e2e_t, t0, t1, t2, t3 = runs[len(runs) // 2]
    e2e_phases = {"init_ms": 1e3 * (t1 - t0), "steps_enqueue_ms": 1e3 * (t2 - t1),
                  "moments_and_drain_ms": 1e3 * (t3 - t2), "calls": E2E_CALLS,
                  "call_ms": [1e3 * r[0] for r in runs]}
    h2d = (rho_h.numel() + u_h.numel()) * 8
    d2h = (rho_out.numel() + u_out.numel()) * 8
    fixed = e2e_itemised(E, sim, rho_h, u_h, rho_d, u_d, rho_out, u_out, barrier, h2d, d2h)

    # The same flow late in the configuration: the vortex breaks down and more nodes need
    # the longer path-length forms, so the step gets costlier.  The state is advanced
    # (untimed) to step FLOW_STEPS - K and K steps are timed as above.
    late = None
    if not args.no_late_flow and args.steps <= FLOW_STEPS // 2:
        late = late_flow_leg(E, sim, rho_d, u_d, one_step, barrier, args.steps, stream, N)

    peak, peak_src = measured_peaks()
    elem = ELEM_BYTES[args.storage]
    bytes_per_node = 2 * LATTICE_Q * elem
    # AUTO launches the DIRECT kernel (elbm.h)
    kname = ("k_step_rows" if args.kernel == "rows" else "k_step") + f"<{args.storage}> (D3Q27)"
    achieved = bytes_per_node * N / kern_avg / 1e9
    traffic = profiled_traffic() if (args.storage == STORAGE and args.kernel != "rows") else None
    value = aggregate_mlups(N, args.steps, world, elapsed)
    if late is not None:
        late["roofline_frac"] = bytes_per_node * N / late["kernel_ms_avg"] * 1e-6 / peak
        late["achieved_gbs"] = bytes_per_node * N / late["kernel_ms_avg"] * 1e-6
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": "D3Q27", "dims": [L, L, L], "beta": BETA,
                   "u0": U0, "storage": args.storage, "diag_every": DIAG_EVERY,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (two %.2f GB population buffers)" % (LATTICE_Q * N * elem / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "kernel": kname,
                     "algorithmic_bytes_per_launch": bytes_per_node * N,
                     "kernel_ms_avg": 1e3 * kern_avg},
        "e2e": {"value": aggregate_mlups(N, args.steps, world, e2e_t), "unit": "MLUPS",
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "what": "elbm_init_equilibrium from pinned host rho,u + K steps + elbm_moments to host "
                        "(median of %d calls)" % E2E_CALLS,
                "phases": e2e_phases, "fixed_cost_per_call": fixed},
        "late_flow": late,
        "gpu_launches": gpu_launches,
        "clocks": clk,
        "physics": {"alpha_min": d["alpha_min"], "alpha_max": d["alpha_max"], "alpha_mean": d["alpha_mean"],
                    "n_solved_frac": d["n_solved"] / N, "n_cutoff_frac": d["n_cutoff"] / N,
                    "n_clamped": d["n_clamped"], "n_nonpositive": d["n_nonpositive"],
                    "dH_max": d["dH_max"], "n_dH_positive": d["n_dH_positive"],
                    "xmax_band_frac": xmax_bands(d, N),
                    "mass": d["mass"], "H": d["H"], "alpha_hist": alpha_hist},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, threads, dt, desc = oracle_time(*oracle_prepare(args.cpu_slab), args.cpu_steps)
        # and on one core: 2 steps of a 256 x 256 x 8 slab (~1M node updates)
        rate1, _, dt1, desc1 = oracle_time(*oracle_prepare(8), 2, nthreads=1)
        line["cpu_baseline"] = {"value": rate, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                                "sample": desc, "seconds": dt,
                                "single_core": {"value": rate1, "sample": desc1, "seconds": dt1}}
    sim.close()
    rep.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_ensemble(args):
    """Batched ensemble: 64 independent periodic D2Q9 domains, sides drawn from
    {64, 96, 128, 192, 256, 384, 512}, beta ~ U[0.9, 0.999], random-phase vortex
    initial velocity (spectrum peaked at k = 4, rms 0.03), FP32.  Both batched forms are
    tuned (work-item widths, then graph against persistent), and K steps are timed in the
    tuned form (ELBM_BATCH_AUTO, the reported value), as one CUDA-graph replay of K
    batched launches, as one persistent cooperative launch (captured in a CUDA graph),
    and as one launch per domain and step.  Each form first runs W and twice K steps
    untimed (so its graphs are captured and instantiated), then restarts from the
    initial state for the timed K steps."""
    import torch

    from paper_2203_12946_gb300 import elbm as E
    from paper_2203_12946_gb300 import inputs

    torch.cuda.set_device(0)
    rng = np.random.default_rng(inputs.DEFAULT_SEED)
    sides = rng.choice([64, 96, 128, 192, 256, 384, 512], size=64)
    betas = rng.uniform(0.9, 0.999, size=64)
    dims = [(int(L_), int(L_), 1) for L_ in sides]
    nodes = int(sum(L_ * L_ for L_ in sides))
    res = {}
    fields = [inputs.random_vortex_2d(d[0], rms=0.03, seed=k) for k, d in enumerate(dims)]
    with E.Ensemble(E.ELBM_D2Q9, dims, list(betas), storage=args.storage) as ens:
        def initial_state():
            for k, (rho, u) in enumerate(fields):
                ens.init_equilibrium(k, rho, u)

        initial_state()
        bx, tune_ms = ens.tune()
        auto_mode, tune_persist_ms = ens.tune_persistent()
        for name, mode in (("auto", E.ELBM_BATCH_AUTO), ("persistent", E.ELBM_BATCH_PERSISTENT),
                           ("graph", E.ELBM_BATCH_GRAPH), ("per_domain", E.ELBM_BATCH_PER_DOMAIN)):
            # every form is timed from the same initial state (the flows decay, and
            # steps near equilibrium are cheaper); the untimed runs capture the graphs
            # of W and K steps for both buffer parities
            ens.step(args.warmup, mode)
            if mode != E.ELBM_BATCH_PER_DOMAIN:
                ens.step(args.steps, mode)
                ens.step(args.steps, mode)
            initial_state()
            ens.synchronize()
            t0 = time.perf_counter()
            ens.step(args.steps, mode)
            ens.synchronize()
            dt = time.perf_counter() - t0
            res[name] = nodes * args.steps / dt / 1e6
        d = ens.diagnostics(0)
    line = {
        "metric": "aggregate MLUPS, 64-domain D2Q9 ensemble (sides 64..512), tuned batched form",
        "value": res["auto"], "unit": "MLUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched ensemble", "domains": 64, "nodes": nodes, "storage": args.storage,
                   "block_width": bx, "tune_ms_per_step": tune_ms,
                   "tuned_form": "persistent" if auto_mode == E.ELBM_BATCH_PERSISTENT else "graph",
                   "tune_persistent_ms_per_step": tune_persist_ms},
        "graph_of_launches_mlups": res["graph"], "persistent_launch_mlups": res["persistent"],
        "per_domain_launches_mlups": res["per_domain"], "speedup_vs_per_domain": res["auto"] / res["per_domain"],
        "domain0_alpha_range": [d["alpha_min"], d["alpha_max"]],
    }
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args):
    """Storage precision study on the doubly periodic shear layer (Sec. IV setup with
    w = delta = 0.05, U0 = 0.04): D2Q9 1024^2, beta = 0.9995, FP64 / FP32 / FP16- and
    BF16-deviation storage on the GPU; velocity and density errors against the FP64 run
    at the checkpoints, MLUPS of each storage, and the FP64 run against the CPU oracle."""
    import torch

    from paper_2203_12946_gb300 import elbm as E
    from paper_2203_12946_gb300 import inputs

    torch.cuda.set_device(0)
    Ls = args.shear_L
    dims = (Ls, Ls, 1)
    beta = 0.9995
    X, Y, _ = inputs.grid(dims)
    rho0, u0 = inputs.shear_layer_2d(X, Y, Ls)
    checkpoints = sorted(int(c) for c in args.checkpoints.split(","))
    fields, rates = {}, {}
    for storage in ("f64", "f32", "f32dev", "f16dev", "bf16dev"):
        with E.Simulation(E.ELBM_D2Q9, dims, beta, storage=storage) as sim:
            sim.init_equilibrium(rho0, u0)
            done = 0
            out = {}
            stream = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t_steps, t_ms = 0, 0.0
            for c in checkpoints:
                e0.record(stream)
                sim.step(c - done)
                e1.record(stream)
                torch.cuda.synchronize()
                t_ms += e0.elapsed_time(e1)
                t_steps += c - done
                done = c
                r, u = sim.moments()
                out[c] = (r.cpu().numpy(), u.cpu().numpy())
                d = sim.diagnostics(allow_nonphysical=True)
                out[c] += (d["n_nonpositive"],)
            fields[storage] = out
            rates[storage] = Ls * Ls * t_steps / (t_ms / 1e3) / 1e6
    table = {}
    for storage in ("f32", "f32dev", "f16dev", "bf16dev"):
        rows = {}
        for c in checkpoints:
            r64, u64, _ = fields["f64"][c]
            r, u, bad = fields[storage][c]
            rows[str(c)] = {
                "u_rel_l2": float(np.linalg.norm(u - u64) / np.linalg.norm(u64)),
                "u_linf_over_U0": float(np.max(np.abs(u - u64)) / 0.04),
                "rho_linf": float(np.max(np.abs(r - r64))),
                "nonpositive_nodes": int(bad),
            }
        table[storage] = rows
    # the FP64 GPU run against the CPU oracle over the first steps
    import oracle as O
    ko = args.oracle_steps
    fo, *_ = O.step(2, dims, O.init_equilibrium(2, rho0, u0), beta, nsteps=ko)
    with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f64") as sim:
        sim.init_equilibrium(rho0, u0)
        sim.step(ko)
        fg = sim.get_populations()
    line = {
        "metric": "velocity error vs FP64 and MLUPS per storage, D2Q9 1024^2 shear layer",
        "config": {"workload": "doubly periodic shear layer", "dims": [Ls, Ls], "beta": beta, "U0": 0.04,
                   "w": 0.05, "delta": 0.05, "checkpoints": checkpoints,
                   "l2": "both buffers fit in L2 at FP32 and below (L2-resident, not HBM-bound)"},
        "errors_vs_fp64": table, "mlups": rates,
        "fp64_vs_oracle": {"steps": ko, "max_rel_f": float(np.max(np.abs(fg - fo) / fo))},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_storage(args):
    """Storage forms from the same initial state in FP64, FP32, FP32, FP16 and BF16
    deviation storage: step time from CUDA events over the run (steps 10..K, K =
    --storage-steps; the moments taken at the checkpoints are outside the events) and the
    velocity error against the FP64 run at each checkpoint (--storage-checkpoints, K by
    default), with the growth exponent of the error between checkpoints (err ~ t^p: p ~ 1/2
    for a random walk of rounding errors, ~1 for a bias) and the step count at which each
    storage's error would cross 1e-3 on that trend.  --storage-lattice d3q27: the benchmark
    flow, D3Q27 L^3 Taylor-Green vortex (u0 = 0.05, beta = 0.999; L = --L, 256 by
    default); d2q9: the doubly periodic shear layer (U0 = 0.04, beta = 0.9995) on a
    --storage-L^2 lattice (4096^2 by default: both FP32 buffers, 1.2 GB each, far above
    L2, so the step is HBM-bound as in the benchmark)."""
    import torch

    from paper_2203_12946_gb300 import elbm as E
    from paper_2203_12946_gb300 import inputs

    torch.cuda.set_device(0)
    K = args.storage_steps
    cps = sorted({int(c) for c in (args.storage_checkpoints or str(K)).split(",")} | {K})
    if cps[0] <= 10:
        raise SystemExit("checkpoints must exceed 10 steps")
    if args.storage_lattice == "d3q27":
        lat, dims, beta, U = E.ELBM_D3Q27, (L, L, L), BETA, U0
        X, Y, Z = inputs.grid(dims)
        rho, u = inputs.taylor_green_3d(X, Y, Z, L, u0=U0)
        del X, Y, Z
        flow = {"flow": "Taylor-Green vortex", "u0": U0}
    else:
        Ls = args.storage_L
        lat, dims, beta, U = E.ELBM_D2Q9, (Ls, Ls, 1), 0.9995, 0.04
        ix, iy = np.meshgrid(np.arange(Ls), np.arange(Ls), indexing="xy")
        rho, u = inputs.shear_layer_2d(ix.ravel(), iy.ravel(), Ls, U0=U)
        flow = {"flow": "doubly periodic shear layer", "U0": U}
    N = int(np.prod(dims))
    u64 = {}
    out = {}
    kinds = [k for k in ("f64", "f32", "f32dev", "f16dev", "bf16dev")
             if not args.storages or k in args.storages.split(",")]
    for st in kinds:
        with E.Simulation(lat, dims, beta, storage=st) as sim:
            sim.init_equilibrium(rho, u)
            sim.step(10)
            stream = torch.cuda.current_stream()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            done, ms_total, errs = 10, 0.0, {}
            for c in cps:
                torch.cuda.synchronize()
                a.record(stream)
                sim.step(c - done)
                b.record(stream)
                torch.cuda.synchronize()
                ms_total += a.elapsed_time(b)
                done = c
                uu = sim.moments()[1].cpu().numpy()
                if st == "f64":
                    u64[c] = uu
                elif c in u64:
                    errs[c] = float(np.linalg.norm(uu - u64[c]) / np.linalg.norm(u64[c]))
            ms = ms_total / (K - 10)
        res = {"ms_per_step": ms, "mlups": N / ms / 1e3}
        if st != "f64" and errs:
            res["u_rel_l2_vs_f64"] = errs[K]
            res["u_rel_l2_at"] = {str(c): e for c, e in errs.items()}
            if len(cps) > 1:
                ts = np.array(cps, dtype=float)
                es = np.array([errs[c] for c in cps])
                slope, icpt = np.polyfit(np.log(ts), np.log(es), 1)
                res["growth_exponent"] = float(slope)
                res["steps_to_1e-3_on_trend"] = float(np.exp((np.log(1e-3) - icpt) / slope)) if slope > 0 else None
        out[st] = res
    line = {"metric": f"step time and velocity error vs FP64 per storage, {args.storage_lattice.upper()} "
                      f"{flow['flow']}",
            "config": {"workload": "storage forms", "dims": list(dims), "beta": beta, **flow, "steps": K,
                       "checkpoints": cps},
            "results": out}
    print(json.dumps(line), flush=True)
    return 0


def run_adjoint(args):
    """Gradient of the final kinetic energy with respect to the initial velocity field and
    to a uniform body force F (evaluated at F = 0): D2Q9 256^2 periodic, beta = 0.9, u0
    from the random-phase vortex generator (rms 0.02), FP32, K steps (default 2000) with
    sqrt(K) checkpointing through the hand-written adjoint.  Reports forward and
    forward+backward throughput, the agreement of <dL/du0, v> with central differences
    (h = 1e-4) of the FP64 forward along seeded directions v, and of dL/dF with central
    differences in each component of F (Richardson-extrapolated from h = 1e-7 and 5e-8)."""
    import torch

    from paper_2203_12946_gb300 import elbm as E
    from paper_2203_12946_gb300 import inputs
    from paper_2203_12946_gb300.adjoint import kinetic_energy_rollout

    torch.cuda.set_device(0)
    Ls, beta, T = args.adjoint_L, 0.9, args.steps
    dims = (Ls, Ls, 1)
    rho0, u0 = inputs.random_vortex_2d(Ls, rms=0.02, seed=inputs.DEFAULT_SEED)
    with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f32", cutoff=False) as sim:
        rt = torch.from_numpy(rho0).cuda()
        # warm-up: one rollout of the same length and the same arguments loads the kernels
        # of both sweeps (the forced reverse step included) and fills the allocator's cache;
        # the first backward of a kind otherwise costs a few hundred milliseconds more
        uw = torch.from_numpy(u0).cuda().requires_grad_(True)
        Fw = torch.zeros(2, dtype=torch.float64, requires_grad=True)
        kinetic_energy_rollout(uw, sim, T, rho0=rt, force=Fw).backward()
        ut = torch.from_numpy(u0).cuda().requires_grad_(True)
        Ft = torch.zeros(2, dtype=torch.float64, requires_grad=True)  # uniform body force, F = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = kinetic_energy_rollout(ut, sim, T, rho0=rt, force=Ft)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        grad = ut.grad.cpu().numpy()
        gradF = Ft.grad.numpy()
    # dL/dF of this zero-mean vortex is close to the time-integrated total momentum, a
    # node sum that cancels far below FP32 resolution: the FP64 reverse sweep is reported too
    with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f64", cutoff=False) as sim:
        u64 = torch.from_numpy(u0).cuda().requires_grad_(True)
        F64 = torch.zeros(2, dtype=torch.float64, requires_grad=True)
        kinetic_energy_rollout(u64, sim, T, rho0=torch.from_numpy(rho0).cuda(), force=F64).backward()
        gradF64 = F64.grad.numpy()
    rng = np.random.default_rng(inputs.DEFAULT_SEED)
    checks = []
    h = 1e-4
    for k in range(args.fd_dirs):
        v = rng.standard_normal(u0.shape) * 0.01
        Lpm = []
        for sgn in (1, -1):
            with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f64", cutoff=False) as sim:
                sim.init_equilibrium(rho0, u0 + sgn * h * v)
                sim.step(T)
                Lpm.append(sim.kinetic_energy())
        fd = (Lpm[0] - Lpm[1]) / (2 * h)
        ad = float(np.sum(grad * v))
        checks.append({"fd": fd, "adjoint": ad, "rel_err": abs(ad - fd) / abs(fd)})
    # dL/dF at F = 0 against central differences of the FP64 forward in each component,
    # Richardson-extrapolated from steps h and h/2 (F acts on every node for K steps, so L
    # is far from linear in F)
    hF = 1e-7
    force_checks = []
    for a in range(2):
        fds = []
        for h in (hF, hF / 2):
            Lpm = []
            for sgn in (1, -1):
                F = np.zeros(2)
                F[a] = sgn * h
                with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f64", cutoff=False) as sim:
                    sim.init_equilibrium(rho0, u0)
                    sim.set_force(F)
                    sim.step(T)
                    Lpm.append(sim.kinetic_energy())
            fds.append((Lpm[0] - Lpm[1]) / (2 * h))
        fd = (4 * fds[1] - fds[0]) / 3
        force_checks.append({"component": a, "fd": fd, "fd_h": fds[0], "fd_h2": fds[1],
                             "adjoint_f32": float(gradF[a]), "rel_err_f32": abs(float(gradF[a]) - fd) / abs(fd),
                             "adjoint_f64": float(gradF64[a]), "rel_err": abs(float(gradF64[a]) - fd) / abs(fd)})
    n = Ls * Ls * T
    line = {
        "metric": "adjoint rollout, D2Q9 256^2, dL/du0 of the final kinetic energy",
        "config": {"workload": "adjoint", "dims": [Ls, Ls], "beta": beta, "steps": T, "storage": "f32",
                   "checkpoint_every": int(np.ceil(np.sqrt(T))), "u0_rms": 0.02},
        "loss": float(loss.detach()), "forward_mlups": n / (t1 - t0) / 1e6,
        "backward_mlups": n / (t2 - t1) / 1e6,
        "fd_checks": checks, "max_rel_err": max(c["rel_err"] for c in checks),
        "force_grad": {"at": [0.0, 0.0], "h": hF, "checks": force_checks,
                       "max_rel_err": max(c["rel_err"] for c in force_checks),
                       "note": "rel_err: FP64 reverse sweep; rel_err_f32: FP32 (near-zero node sum)"},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 5000 for the benchmark workload, the Taylor-Green "
                         "configuration's length; 2000 for the others)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-slab", type=int, default=128,
                    help="z-extent of the 256x256 slab the CPU oracle times (about 10-30 s of work)")
    ap.add_argument("--cpu-steps", type=int, default=24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", choices=["auto", "direct", "rows"], default="auto")
    ap.add_argument("--workload", choices=["tgv3d", "ensemble", "precision", "adjoint", "storage"],
                    default="tgv3d",
                    help="tgv3d: the benchmark (D3Q27 256^3); ensemble: batched D2Q9 domains; "
                         "precision: storage error study on the D2Q9 shear layer; adjoint: gradient "
                         "rollout; storage: storage forms on the D3Q27 flow")
    ap.add_argument("--shear-L", type=int, default=1024)
    ap.add_argument("--checkpoints", default="1000,5000,20000")
    ap.add_argument("--oracle-steps", type=int, default=50)
    ap.add_argument("--adjoint-L", type=int, default=256)
    ap.add_argument("--fd-dirs", type=int, default=4)
    ap.add_argument("--storage-steps", type=int, default=1000)
    ap.add_argument("--storage-checkpoints", default=None,
                    help="comma-separated step counts at which the storage workload compares u with FP64")
    ap.add_argument("--storage-lattice", choices=["d3q27", "d2q9"], default="d3q27")
    ap.add_argument("--storage-L", type=int, default=4096, help="side of the D2Q9 storage workload")
    ap.add_argument("--storage", choices=["f32", "f32dev", "f16dev", "bf16dev"], default=STORAGE)
    ap.add_argument("--storages", default=None,
                    help="comma-separated storage kinds the storage workload runs (default: all; the "
                         "velocity errors need f64 among them)")
    ap.add_argument("--no-late-flow", action="store_true",
                    help="skip the late-flow leg (steps 5000-K .. 5000 of the same flow)")
    ap.add_argument("--L", type=int, default=L, help="domain side (profiling runs only; "
                    "the benchmark workload is 256)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 5000 if args.workload == "tgv3d" else 2000
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.L != L:
        set_side(args.L)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "storage":
        return run_storage(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
