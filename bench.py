#!/usr/bin/env python3
"""Benchmark of the fused nlM lattice-Boltzmann step on GB300.

Workload (default): the single large channel -- 4096 x 4096 nodes, x periodic, bounce-back walls,
FP32 SoA populations stored as deviations from the lattice weights, the 4-component polymer
stress written every step, nlM model theta = 100, gamma_c = 0.1, tau_LB = 0.9, g = 1e-6,
G_inf = 1e-3, start-up from rho = 1 + 1e-6 U(-1,1) (SplitMix64 seed 1).  One benchmark step is
one lattice-Boltzmann time step over all nodes.  The state (1.6 GB) is far larger than L2.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS & % HBM roofline; batched-sweep time-to-steady, plain vs warm-start"
UNIT = "GLUPS"
KERNEL_SOURCES = {
    "k_step_march": ["paper_1310_7450_gb300/csrc/lb_step_march.cuh", "paper_1310_7450_gb300/csrc/lb_device.cuh"],
    "k_step_tile": ["paper_1310_7450_gb300/csrc/lb_step_tile.cuh", "paper_1310_7450_gb300/csrc/lb_device.cuh"],
}


def code_only(text: str) -> str:
    """Source text without comments and blank lines: what the kernel hash covers, so that an edit of
    a comment does not orphan the committed DRAM counters while any change of code does."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(code_only(open(os.path.join(ROOT, f)).read()).encode())
    return h.hexdigest()[:16]


PREC_NAME = {"f32": "FP32", "bf16": "BF16", "f64": "FP64"}


def bytes_per_node(precision: str, store_sigma: bool, stress_mode: int, scheme: str = "paper") -> int:
    """Algorithmic HBM bytes per node and step: 9 population loads + 9 stores in the storage type,
    delta rho read + write, (+ stress write: xx, yy, xy -- the zz plane of the 4-component stress is
    0 in 2-D flow and written once at create), (+ carried stress read + write in stress mode 1).
    Comparison schemes of Sec. II C and the relaxation-time extensions (tile kernel): the
    generalized-Newtonian scheme moves the same bytes; the stress-divergence scheme runs a first
    pass that reads the populations and delta rho and writes Sigma^nN (3 planes), then the step,
    which also reads Sigma^nN; the relaxation model with a fluidity memory reads and writes the
    FP64 fluidity plane."""
    t = {"f64": 8, "f32": 4, "bf16": 2}[precision]
    c = 8 if precision == "f64" else 4
    b = 18 * t + 2 * c
    if store_sigma:
        b += 3 * c
    if stress_mode == 1:
        b += 6 * c
    if scheme == "stress_divergence":
        b += 9 * t + c + 3 * c + 3 * c   # first pass: populations + delta rho in, Sigma^nN out; step: Sigma^nN in
    elif scheme == "relaxation":
        b += 16                          # fluidity plane (FP64) read + write
    return b


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def stored_traffic(kernel: str, precision: str, workload_nodes: int):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, scaled to the
    workload by nodes, or None when missing or taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{precision}_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_hash") != kernel_hash(kernel):
        return None
    return d["dram_bytes_per_launch"] * workload_nodes / d["nodes"]


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if not getattr(self, "out", ""):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(args):
    from paper_1310_7450_gb300 import inputs
    cfg = inputs.single_large_channel(args.nx, args.ny)
    p = dict(cfg["params"], rho_pert_amp=cfg["rho_pert_amp"], seed=cfg["seed"])
    return cfg, p


def cpu_oracle_rate(p, nx, ny, seconds: float, threads: int):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload: a nx x ny crop with
    the same parameters and seeded perturbation; returns (GLUPS, steps, threads)."""
    import oracle
    from paper_1310_7450_gb300 import inputs
    oracle.build()
    st = oracle.init_state(inputs.initial_density(nx, ny, 1.0, p["rho_pert_amp"], p["seed"]))
    t0 = time.perf_counter()
    oracle.run(p, st, 1, nthreads=threads)
    one = max(time.perf_counter() - t0, 1e-4)
    steps = max(2, int(seconds / one))
    t0 = time.perf_counter()
    oracle.run(p, st, steps, nthreads=threads)
    dt = time.perf_counter() - t0
    return nx * ny * steps / dt / 1e9, steps, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cfg, p = workload(args)
    threads = os.cpu_count() or 1
    import oracle
    from paper_1310_7450_gb300 import inputs
    oracle.build()
    cnx, cny = args.ref_crop, args.ref_crop
    st = oracle.init_state(inputs.initial_density(cnx, cny, 1.0, p["rho_pert_amp"], p["seed"]))
    for _ in range(args.warmup):
        oracle.run(p, st, 1, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(p, st, 1, nthreads=threads)
    dt = time.perf_counter() - t0
    val = cnx * cny * args.steps / dt / 1e9
    sample = (f"{cnx}x{cny} crop of the {cfg['nx']}x{cfg['ny']} start-up workload (same parameters and "
              f"seeded perturbation), one oracle step per benchmark step, FP64 C oracle with {threads} OpenMP threads")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"single large channel {cfg['nx']}x{cfg['ny']} start-up (oracle on a crop)",
                       "nx": cnx, "ny": cny},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    from paper_1310_7450_gb300 import build as libbuild
    from paper_1310_7450_gb300 import lbnlm

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    libbuild.build()
    lbnlm.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    cfg, p = workload(args)
    nx, ny = cfg["nx"], cfg["ny"]
    flags = lbnlm.LB_GRID_STORE_SIGMA if args.store_sigma else 0
    if args.tile_only:
        flags |= lbnlm.LB_GRID_TILE_ONLY
    if args.scheme == "relaxation":
        flags |= lbnlm.LB_GRID_RELAXATION_MODEL
    lib_scheme = args.scheme if args.scheme in lbnlm.SCHEME_FLAGS else "paper"
    sim = lbnlm.Channels(nx, ny, p, args.precision, stress_mode=args.stress_mode, flags=flags,
                         stream=stream.cuda_stream, x_mode=args.x_mode, walls=args.walls, scheme=lib_scheme)
    if args.walls == "couette":
        lbnlm.lb_set_wall_velocity(sim.h, -1, args.u_wall)
    if args.scheme == "relaxation":
        # density-dependent Maxwell time and a fluidity memory of tau_M (both extensions at once)
        lbnlm.lb_set_relaxation_model(sim.h, -1, 5.0, 1.0, 2000.0)
    nodes = nx * ny
    kernel = "k_step_march" if lbnlm.lb_uses_row_march(sim.h) else "k_step_tile"
    # pressure-driven ends add one boundary-column kernel before every step (either step kernel);
    # the stress-divergence scheme runs two passes of the tile kernel per step
    launches_per_step = (2 if args.x_mode == "gpbc" else 1) * (2 if args.scheme == "stress_divergence" else 1)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up (includes the CUDA module load and the first residual evaluation)
    sim.step(max(args.warmup, 3))
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(torch.cuda.current_device())
    with sampler:
        time.sleep(0.3)
        barrier()
        ev0.record(stream)
        st = sim.step(args.steps)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    if st != lbnlm.LB_OK:
        print(json.dumps({"error": f"lb_step status {st}: {lbnlm.lb_last_error()}"}), flush=True)
        return 1
    t_max = ms
    if ws > 1:
        tt = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_max = float(tt.item())
    ms_step = t_max / args.steps
    value = ws * nodes / (ms_step * 1e-3) / 1e9
    # K fused steps (+ the GPBC column pass); the tile kernel adds a residual reduction launch (the
    # row-march kernel's last CTA reduces the residual itself)
    launches = launches_per_step * args.steps + (0 if kernel == "k_step_march" else 1)

    # end to end through the C ABI: per step the body force goes host -> device from pinned memory
    # (lb_set_body_force), one step runs, and the step's channel monitor comes back to pinned host
    # memory (lb_monitor_async); the host never waits inside the loop, so step k's diagnostics
    # travel while step k+1 runs.  The headline loop monitors flux and max |u| every step
    # (LB_MONITOR_FLUX_MAX: what the start-up / cessation run reads, its stop being max |u| <
    # 1e-10); e2e_residual: the same loop with the one-step residual every step (velocity saved and
    # re-read every step); e2e_sync: the headline loop with the blocking lb_monitor.
    e2e = None
    if args.e2e_steps > 0:
        g = p["g_x"]
        K = args.e2e_steps
        mon_pinned = torch.zeros((K, 4), dtype=torch.float64, pin_memory=True)

        def timed_loop(mode, blocking):
            lbnlm.lb_set_monitor_mode(sim.h, mode)
            for k in range(3):
                lbnlm.lb_set_body_force(sim.h, -1, g)
                sim.step(1)
                lbnlm.lb_monitor_async(sim.h, mon_pinned[k])
            barrier()
            mon = np.zeros(4)
            t0 = time.perf_counter()
            for k in range(K):
                lbnlm.lb_set_body_force(sim.h, -1, g)
                sim.step(1)
                if blocking:
                    lbnlm.lb_monitor(sim.h, mon)
                else:
                    lbnlm.lb_monitor_async(sim.h, mon_pinned[k])
            stream.synchronize()
            dt = time.perf_counter() - t0
            if not blocking:
                m = mon_pinned.numpy()
                assert np.all(np.isfinite(m)) and float(m[-1, 3]) > 0 and float(m[-1, 2]) > 0
            if ws > 1:
                tt = torch.tensor([dt], device="cuda")
                torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
                dt = float(tt.item())
            return ws * nodes * K / dt / 1e9

        v_flux = timed_loop(lbnlm.LB_MONITOR_FLUX_MAX, False)
        v_resid = timed_loop(lbnlm.LB_MONITOR_RESIDUAL, False)
        v_sync = timed_loop(lbnlm.LB_MONITOR_FLUX_MAX, True)
        e2e = {"value": v_flux, "unit": UNIT, "h2d_bytes_per_step": 8, "d2h_bytes_per_step": 32, "steps": K,
               "call": "lb_set_body_force + lb_step(1) + lb_monitor_async (pinned; flux and max |u| every step, "
                       "LB_MONITOR_FLUX_MAX) per step, one wait at the end",
               "e2e_residual": {"value": v_resid, "unit": UNIT,
                                "call": "the same loop with the one-step residual every step (LB_MONITOR_RESIDUAL)"},
               "e2e_sync": {"value": v_sync, "unit": UNIT,
                            "call": "lb_set_body_force + lb_step(1) + lb_monitor (blocking) per step, LB_MONITOR_FLUX_MAX"}}
    sim.close()

    # the second half of the metric: the warm-started batched sweep against the plain per-channel
    # scheme (compact: a smaller training draw than the full --workload warmstart run)
    sweep = None
    if not args.no_sweep and ws == 1:
        sweep = warm_sweep(stream.cuda_stream, "f32", args.sweep_train, 5, 512, 55, 1e-8, 1000, args.sweep_cap,
                           args.sweep_epochs, 1e-3, plain_sample=args.sweep_plain)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0
    peak, peak_kind = measured_peaks()
    bpn = bytes_per_node(args.precision, args.store_sigma, args.stress_mode, args.scheme)
    achieved = bpn * nodes / (ms_step * 1e-3) / 1e9
    traffic = stored_traffic(kernel, args.precision, nodes)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
            "bytes_per_node": bpn, "kernel": kernel, "duration_ms": ms_step}
    cpu = None
    if not args.no_cpu_baseline and ws >= 1 and rank == 0 and ws == 1:
        threads = os.cpu_count() or 1
        val, steps, dt = cpu_oracle_rate(p, args.cpu_crop, args.cpu_crop, args.cpu_seconds, threads)
        cpu = {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{args.cpu_crop}x{args.cpu_crop} crop of the same workload, {steps} steps in {dt:.1f} s, "
                         f"FP64 C oracle, {threads} OpenMP threads"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"single large channel {nx}x{ny} start-up, nlM theta=100, gamma_c=0.1, "
                                   f"tau_LB=0.9, g=1e-6, G_inf=1e-3; {PREC_NAME[args.precision]} SoA deviations"
                                   + (" + 4-component stress" if args.store_sigma else "")
                                   + ("" if args.x_mode == "periodic" else "; pressure-driven ends (GPBC)")
                                   + ("" if args.walls == "bounce_back" else f"; Couette wall u={args.u_wall:g}"),
                       "x_mode": args.x_mode, "walls": args.walls, "scheme": args.scheme, "kernel": kernel,
                       "nx": nx, "ny": ny, "precision": args.precision, "stress_mode": args.stress_mode,
                       "store_sigma": bool(args.store_sigma),
                       "l2": f"state {bpn * nodes / 2**30:.2f} GiB per step, larger than the 126 MB L2 (no flush)",
                       "parallelism": f"{ws} independent replica(s)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": sampler.summary(),
            "sweep": sweep if sweep is not None else {"skipped": "--no-sweep or more than one GPU"}}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_cessation(args):
    """Start-up then cessation of the single large channel (the throughput workload's parameters):
    `startup` steps with the body force on, the force switched off for every later step
    (lb_set_body_force, stream-ordered), then steps in chunks of `check` with the channel monitor
    (max |u|, flux) between chunks until max |u| < `stop_u` (the stopping time), `max_steps` or
    `seconds` of wall time.  Reports the stopping step if reached, the decay record and GLUPS over
    the whole device-timed run (monitor calls included)."""
    import torch
    from paper_1310_7450_gb300 import build as libbuild
    from paper_1310_7450_gb300 import lbnlm
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    libbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    cfg, p = workload(args)
    nx, ny = cfg["nx"], cfg["ny"]
    flags = lbnlm.LB_GRID_STORE_SIGMA if args.store_sigma else 0
    sim = lbnlm.Channels(nx, ny, p, args.precision, stress_mode=args.stress_mode, flags=flags,
                         stream=stream.cuda_stream)
    mon = np.zeros(4)
    record = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(torch.cuda.current_device())
    t_wall = time.perf_counter()
    with sampler:
        torch.cuda.synchronize()
        ev0.record(stream)
        done = 0
        while done < args.startup:
            n = min(args.check, args.startup - done)
            sim.step(n)
            done += n
            lbnlm.lb_monitor(sim.h, mon)
            record.append((done, float(mon[2]), float(mon[1])))
        u_startup = float(mon[2])
        lbnlm.lb_set_body_force(sim.h, -1, 0.0)
        stop = None
        while done < args.startup + args.max_steps and time.perf_counter() - t_wall < args.seconds:
            st = sim.step(args.check)
            done += args.check
            lbnlm.lb_monitor(sim.h, mon)
            record.append((done, float(mon[2]), float(mon[1])))
            if st != lbnlm.LB_OK:
                print(json.dumps({"error": f"lb_step status {st}: {lbnlm.lb_last_error()}"}), flush=True)
                return 1
            if mon[2] < args.stop_u:
                stop = done - args.startup
                break
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    sim.close()
    keep = sorted(set(np.unique(np.geomspace(1, len(record), 40).astype(int) - 1)))
    line = {"metric": "start-up + cessation: GLUPS and stopping time", "value": nx * ny * done / (ms * 1e-3) / 1e9,
            "unit": UNIT, "higher_is_better": True, "n_gpus": 1, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"single large channel {nx}x{ny}, start-up {args.startup} steps then cessation "
                                   f"until max|u| < {args.stop_u:g}", "check_every": args.check,
                       "store_sigma": bool(args.store_sigma)},
            "steps_total": done, "device_ms": ms, "max_u_after_startup": u_startup,
            "stopping_steps": stop, "stopped": stop is not None,
            "record_step_maxu_flux": [record[i] for i in keep], "clocks": sampler.summary()}
    print(json.dumps(line), flush=True)
    return 0


def plain_per_step(nys, params, args, stream):
    """Seconds per step of the plain per-channel FP32 scheme (one single-channel handle, lb_step in
    chunks of `check` steps with lb_residual between chunks), measured on a stratified sample of
    the channels by width; returns the samples and a linear fit in Ny."""
    import torch
    from paper_1310_7450_gb300 import lbnlm
    order = np.argsort(nys)
    sample = order[np.linspace(0, len(order) - 1, args.baseline_sample).astype(int)]
    per_step = {}
    for c in sample:
        one = lbnlm.Channels(4, nys[c], params[c], args.precision, stream=stream.cuda_stream)
        one.step(args.check)
        torch.cuda.synchronize()
        n_chunks = max(2, args.baseline_steps // args.check)
        t1 = time.perf_counter()
        for _ in range(n_chunks):
            one.step(args.check)
            one.residual()
        per_step[int(c)] = (time.perf_counter() - t1) / (n_chunks * args.check)
        one.close()
    xs = np.array([nys[c] for c in per_step]); ys = np.array([per_step[c] for c in per_step])
    return per_step, np.polyfit(xs, ys, 1)


def run_sweep(args):
    """Batched sweep: the 512-channel draw (Nx = 4, Ny ~ U{32..1024}, g = b (32/Ny)^2 with
    b ~ logU[1e-8, 1e-5], theta = 10^(2 + 10 eps), eps ~ U[-0.1, 0.1], seed 3), FP32, all channels
    from rest to a check-interval residual <= tol (lb_run_until_steady: width classes, persistent
    launches, one graph).  Baseline: the plain per-channel scheme (one single-channel handle per
    channel, lb_step in chunks of `check` steps and lb_residual between chunks); its time per step
    is measured on a stratified sample of channels and multiplied by each channel's own step count
    (converged channels) or the cap (the others) -- the same steps as in the sweep."""
    import torch
    from paper_1310_7450_gb300 import build as libbuild
    from paper_1310_7450_gb300 import inputs, lbnlm, replicas
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        torch.distributed.init_process_group("nccl")
    libbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    params = inputs.sweep_channel_params(args.channels, args.sweep_seed)
    nys = [q.pop("ny") for q in params]
    n_all = len(nys)
    if ws > 1:  # independent channels: each rank runs its share, no collective on the data path
        mine = replicas.partition_channels(nys, ws, rank)
        nys, params = [nys[c] for c in mine], [params[c] for c in mine]
    sim = lbnlm.Channels(4, nys, params, args.precision, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    lbnlm.lb_sweep_tune(sim.h)
    tune_s = time.perf_counter() - t0
    nt, cl, tune_ms = lbnlm.lb_sweep_config(sim.h)
    variant = ("l2", "shared_memory")[lbnlm.lb_sweep_variant(sim.h)]
    classes = [{"kernel": ("l2", "shared_memory")[v], "threads": t, "cluster": c, "channels": k}
               for v, t, c, k in lbnlm.lb_sweep_groups(sim.h)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, res = sim.run_until_steady(args.tol, check_every=args.check, max_steps=args.max_steps)
    wall = time.perf_counter() - t0
    sim.close()
    conv = steps > 0
    per_step, fit = plain_per_step(nys, params, args, stream)
    # the same work as the sweep: converged channels for their steps, the others up to the cap
    cap = int(args.max_steps)
    est = float(sum((steps[c] if steps[c] > 0 else cap) * np.polyval(fit, nys[c]) for c in range(len(nys))))
    job = replicas.reduce_job({"wall": ("max", wall), "est": ("max", est), "converged": ("sum", int(conv.sum()))}, ws)
    if ws > 1:
        torch.distributed.destroy_process_group()
        if rank != 0:
            return 0
        wall, est = job["wall"], job["est"]
        line = {"metric": "batched-sweep time-to-steady (plain per-channel vs one persistent launch)",
                "value": wall, "unit": "s", "higher_is_better": False, "n_gpus": ws, "scaling": "strong",
                "dtype": args.precision, "data": "synthetic",
                "config": {"workload": f"{n_all} channels, Nx=4, Ny~U{{32..1024}}, seed {args.sweep_seed}, "
                                       f"partitioned over {ws} GPUs", "tol": args.tol, "check_every": args.check,
                           "max_steps": args.max_steps},
                "converged": int(job["converged"]), "channels": n_all,
                "baseline_plain_per_channel": {"estimated_s": est}, "speedup_vs_plain": est / wall if wall > 0 else None}
        print(json.dumps(line), flush=True)
        return 0
    line = {"metric": "batched-sweep time-to-steady (plain per-channel vs one persistent launch)",
            "value": wall, "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": args.precision,
            "data": "synthetic", "config": {"workload": f"{len(nys)} channels, Nx=4, Ny~U{{32..1024}}, seed {args.sweep_seed}",
                                            "tol": args.tol, "check_every": args.check, "max_steps": args.max_steps},
            "converged": int(conv.sum()), "channels": len(nys), "max_steps_taken": int(steps.max()),
            "steps_percentiles": [int(v) for v in np.percentile(steps[conv], [0, 50, 90, 100])] if conv.any() else None,
            "node_steps": int(sum(max(steps[c], 0) * 4 * nys[c] for c in range(len(nys)))),
            "autotune": {"kernel": variant, "threads": nt, "cluster": cl, "tune_run_ms": tune_ms, "tune_wall_s": tune_s,
                         "classes": classes},
            "baseline_plain_per_channel": {"estimated_s": est, "sample_channels": len(per_step),
                                           "per_step_us_by_ny": {str(nys[c]): round(1e6 * v, 2) for c, v in per_step.items()}},
            "speedup_vs_plain": est / wall if wall > 0 else None}
    print(json.dumps(line), flush=True)
    return 0


def plain_to_steady(ny, p, precision, sid, tol, check, cap):
    """The plain per-channel FP32 scheme from rest, run for real: one single-channel handle, lb_step in
    chunks of `check` steps, and after each chunk the check-interval residual ||u(t) - u(t-k)|| /
    (k ||u(t)||) of the batched sweep (the same convergence measure) from two velocity fields on the
    device (lb_field_monitor_static).  Returns (steps to converge or -1 at the cap, wall seconds)."""
    import torch
    from paper_1310_7450_gb300 import lbnlm
    sim = lbnlm.Channels(4, ny, p, precision, stream=sid)
    n = 4 * ny
    u_prev = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    u_now = torch.zeros_like(u_prev)
    offs = torch.tensor([0, n], dtype=torch.int64, device="cuda")
    mon = torch.zeros(3, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, done = 0, -1
    lbnlm.lb_get_fields(sim.h, u_prev, None, None, 0, True)
    while steps < cap:
        sim.step(check)
        steps += check
        lbnlm.lb_get_fields(sim.h, u_now, None, None, 0, True)
        lbnlm.lb_field_monitor_static(u_now, u_prev, 0, 1, offs, 4, mon, sid)
        if float(mon[0].item()) / check <= tol:
            done = steps
            break
        u_prev, u_now = u_now, u_prev
    wall = time.perf_counter() - t0
    sim.close()
    return done, wall


def warm_sweep(sid, precision, train_n, train_seed, held_n, held_seed, tol, check, cap, epochs, lr,
               plain_sample=0, judged=False, skip_rest=False):
    """The learned warm start end to end, every profile step on the device: training data = steady
    states of the batched sweep (`train_n` draws like the batched sweep, seed `train_seed`, started
    from the closed form; targets encoded by lb_warmstart_targets); the perceptron trained by the
    library's kernels; `held_n` held-out draws (seed `held_seed`) run to steady from the surrogate's
    start (decoded by lb_warmstart_apply), from the closed form and from rest, all under the step cap
    `cap`; optionally the LB-judged start, and the plain per-channel FP32 scheme from rest run to
    convergence for real on a stratified sample of `plain_sample` held-out channels."""
    import torch
    from paper_1310_7450_gb300 import inputs, lbnlm, warmstart

    def draw(n, seed):
        ps = inputs.sweep_channel_params(n, seed)
        return [q.pop("ny") for q in ps], ps

    def steady(nys, ps, start, keep=False):
        sim = lbnlm.Channels(4, nys, ps, precision, stream=sid)
        if start is not None:
            start(sim)
        lbnlm.lb_sweep_tune(sim.h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps, _ = sim.run_until_steady(tol, check_every=check, max_steps=cap)
        wall = time.perf_counter() - t0
        if keep:
            return steps, wall, sim
        sim.close()
        return steps, wall, None

    t_all = time.perf_counter()
    nys_t, ps_t = draw(train_n, train_seed)
    st_t, wall_t, sim_t = steady(nys_t, ps_t, warmstart.start_closed_form, keep=True)
    ok = st_t > 0
    Y = warmstart.steady_targets(sim_t)[torch.tensor(np.flatnonzero(ok), device="cuda")]
    sim_t.close()
    X = warmstart.features([n for n, o in zip(nys_t, ok) if o], [q for q, o in zip(ps_t, ok) if o])
    # two untimed steps of a throwaway surrogate of the same shape load the training path's kernels
    # (CUDA loads each kernel at its first launch); the timed model is the seeded one below
    warm = warmstart.Surrogate(width=256, max_batch=512, seed=2, stream=sid)
    warm.fit(X[:512], Y[:512], epochs=2, batch=256, lr=lr)
    warm.close()
    torch.cuda.synchronize()
    sur = warmstart.Surrogate(width=256, max_batch=512, seed=1, stream=sid)
    t0 = time.perf_counter()
    losses = sur.fit(X, Y, epochs=epochs, batch=256, lr=lr)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    nys, ps = draw(held_n, held_seed)
    mlp_start = lambda sim: sur.start(sim, nys, ps)

    def start_u(start):  # the velocity field a start writes, before any step
        sim = lbnlm.Channels(4, nys, ps, precision, stream=sid)
        start(sim)
        fl = [f[0][:, 0, 0] for f in sim.fields()]
        sim.close()
        return fl
    arms = [("mlp", mlp_start), ("closed_form", warmstart.start_closed_form)]
    judge_s, pick = None, None
    if judged:
        t0 = time.perf_counter()
        pick = warmstart.judge(4, nys, ps, [mlp_start, warmstart.start_closed_form], precision, sid, check=check)
        torch.cuda.synchronize()
        judge_s = time.perf_counter() - t0
    if not skip_rest:
        arms.append(("rest", None))
    res, conv_u = {}, None
    for name, start in arms:
        st, wall, sim = steady(nys, ps, start, keep=(name == "closed_form"))
        res[name] = {"wall_s": wall, "converged": int((st > 0).sum()), "steps_sum": int(np.where(st > 0, st, cap).sum()),
                     "steps_max": int(st.max()) if (st > 0).all() else cap,
                     "steps_median": float(np.median(np.where(st > 0, st, cap)))}
        if name == "rest":
            st_rest = st
        if sim is not None:
            conv_u = [f[0][:, 0, 0] for f in sim.fields()]
            sim.close()
    errs = {}
    for name, start in (("mlp", mlp_start), ("closed_form", warmstart.start_closed_form)):
        e = [float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) for a, b in zip(start_u(start), conv_u)]
        errs[name] = {"median": float(np.median(e)), "p90": float(np.percentile(e, 90))}
    sur.close()
    plain = None
    if plain_sample > 0:
        order = np.argsort(nys)
        sample = order[np.linspace(0, len(order) - 1, plain_sample).astype(int)]
        runs = []
        for c in sample:
            done, wall = plain_to_steady(nys[c], ps[c], precision, sid, tol, check, cap)
            runs.append({"ny": int(nys[c]), "steps": int(done), "wall_s": wall})
        tot = sum(r["wall_s"] for r in runs)
        plain = {"sample": runs, "sample_wall_s": tot, "sample_converged": int(sum(r["steps"] > 0 for r in runs)),
                 "scaled_to_all_s": tot / len(runs) * len(nys),
                 "how": f"the plain per-channel FP32 scheme from rest, run for real to the same check-interval residual "
                        f"and cap on {len(runs)} held-out channels stratified by width (one handle per channel, lb_step "
                        f"chunks of {check}); scaled_to_all_s = their mean wall time x {len(nys)} channels"}
        if "rest" in res:
            plain["sweep_steps_of_sample_from_rest"] = [int(st_rest[c]) for c in sample]
    train_tflops = sur.flops_per_step(sur.batch_used) * sur.steps_done / train_s / 1e12 if train_s > 0 else None
    return {"train_channels": train_n, "train_converged": int(ok.sum()), "train_data_sweep_s": wall_t, "train_s": train_s,
            "train_tflops": train_tflops, "train_steps": sur.steps_done,
            "epochs": epochs, "final_loss": losses[-1], "held_out": held_n, "held_seed": held_seed, "tol": tol,
            "check_every": check, "cap": cap, "arms": res, "start_error_u_vs_converged": errs,
            "judged": None if pick is None else {"judge_s": judge_s, "picked_mlp": int((pick == 0).sum())},
            "plain_per_channel_from_rest": plain, "total_s": time.perf_counter() - t_all}


def run_warmstart(args):
    """Learned warm start at full size: `train` draws for the training data (seed `train_seed`),
    `channels` held-out draws (seed `sweep_seed`), the LB-judged start, the plain per-channel arm on a
    sample (`baseline_sample` channels)."""
    import torch
    from paper_1310_7450_gb300 import build as libbuild
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    libbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    r = warm_sweep(stream.cuda_stream, args.precision, args.train, args.train_seed, args.channels, args.sweep_seed,
                   args.tol, args.check, args.max_steps, args.epochs, args.lr, plain_sample=args.baseline_sample,
                   judged=True, skip_rest=args.skip_cold)
    line = {"metric": "batched-sweep time-to-steady, plain vs warm-start", "unit": "s", "higher_is_better": False,
            "value": r["arms"]["mlp"]["wall_s"], "n_gpus": 1, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"learned warm start: {args.train} training draws, {args.channels} held out, Nx=4, "
                                   f"Ny~U{{32..1024}}", "tol": args.tol, "check_every": args.check, "cap": args.max_steps},
            "warm_start": r}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--ny", type=int, default=4096)
    ap.add_argument("--precision", default="f32", choices=["f32", "bf16", "f64"])
    ap.add_argument("--stress-mode", type=int, default=0)
    ap.add_argument("--no-store-sigma", dest="store_sigma", action="store_false")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--x-mode", default="periodic", choices=["periodic", "gpbc"])
    ap.add_argument("--walls", default="bounce_back", choices=["bounce_back", "couette"])
    ap.add_argument("--u-wall", type=float, default=0.01)
    ap.add_argument("--tile-only", action="store_true")
    ap.add_argument("--scheme", default="paper",
                    choices=["paper", "generalized_newtonian", "stress_divergence", "relaxation"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep-train", type=int, default=2000)
    ap.add_argument("--sweep-cap", type=int, default=2_000_000)
    ap.add_argument("--sweep-epochs", type=int, default=200)
    ap.add_argument("--sweep-plain", type=int, default=6)
    ap.add_argument("--cpu-crop", type=int, default=512)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-crop", type=int, default=512)
    ap.add_argument("--workload", default="channel", choices=["channel", "sweep", "warmstart", "cessation"])
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--train-seed", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--skip-cold", action="store_true")
    ap.add_argument("--channels", type=int, default=512)
    ap.add_argument("--sweep-seed", type=int, default=3)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--check", type=int, default=1000)
    ap.add_argument("--max-steps", type=int, default=20_000_000)
    ap.add_argument("--baseline-sample", type=int, default=8)
    ap.add_argument("--baseline-steps", type=int, default=2000)
    ap.add_argument("--startup", type=int, default=50000)
    ap.add_argument("--stop-u", type=float, default=1e-10)
    ap.add_argument("--seconds", type=float, default=240.0)
    args = ap.parse_args()
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "cessation":
        return run_cessation(args)
    if args.workload == "warmstart":
        if args.sweep_seed == 3:
            args.sweep_seed = 55
        return run_warmstart(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
