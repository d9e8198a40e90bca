#!/usr/bin/env python
"""Benchmark of the CSPH hot path on GB300.

Workload: the 3D plate impact (50^3 projector at 1 km/s onto a 200x200x25
slab, 1,125,000 particles, cubic lattice 0.1 mm, stiffened gas rho0 = 2700,
c0 = 5.3 km/s, gamma = 2, h = 1.3 spacing), FP32 pair fluxes with FP64
positions, 64 Voronoi work units rebalanced every 10 steps, Verlet lists
with buffer beta = 0.15.  A step is one full CSPH time step (CFL reduction,
kick-drift, list validity check, operand packing, pair evaluation over the
lists, kick), plus the cell mesh, sort and list build whenever the device-side
criterion asks for them (the count is reported in config.list_builds), plus,
every 10th step, balancing + reassignment + renumbering.  --beta 0 gives the
per-step mesh and pair search instead.  Inputs are synthetic
(synth.plate_impact_full) and larger than L2 (the FP64 state is ~190 MB), so
no L2 flush is needed.

Prints one JSON line (rank 0).  At one GPU the line also carries "extras"
(skip with --no-extras): the plain FP64 step against the mixed step on the
same plate; the 256-instance ensemble (one CUDA graph of 100 steps,
autotuned) against 256 sequential single-instance runs; and the forward +
reverse mode of a 203k-particle plate in both precisions.  --impl reference
times the FP64 CPU oracle on the host cores instead, on a bounded sample of
the same workload.
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

METRIC = "CSPH particle-steps/s on 1 GB300 (plate impact, FP32 pair fluxes / FP64 positions)"
UNIT = "particle-steps/s"
WORKLOAD = "plate_impact_1125k"
# named workloads: the plate impact of the benchmark and a smaller one of the
# same shape for profiler captures
WORKLOADS = {
    "plate_impact_1125k": dict(proj=50, target=(200, 200, 25)),
    "plate_impact_387k": dict(proj=30, target=(120, 120, 25)),
}

# Algorithmic FP32 work of the pair loop (counted from the formulas of Sec. 4.1-4.2):
#   per unique candidate pair (interaction test r^2 < (kappa h_ij)^2): 11 flops
#   per interacting half pair (e^R, v^R, acoustic P*, v*, W', three rate terms for both ends): 70 flops
FLOP_TEST = 11.0
FLOP_PAIR = 70.0
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 rate; the FP64 pair kernel is bound by it
BETA = 0.15               # Verlet buffer of the benchmark (best of 0.1 / 0.15 / 0.2 / 0.3 on this workload)


def fp32_peak_tflops() -> float:
    """152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz maximum SM clock."""
    return 152 * 128 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# The oracle baseline runs one process per host core, each on its own copy of
# a 1/14 sample of the workload (same lattice, EOS and impact: a 25^3
# projector on a 50x50x25 slab, 78,125 particles); the job's time is the
# slowest process's.
ORACLE_SAMPLE = dict(proj=25, target=(50, 50, 25))
ORACLE_TIMEOUT_S = 1200


def _oracle_core(steps: int, warmup: int, barrier, results):
    """One host core's share of the oracle baseline (a spawned process): its
    sample, one rate evaluation and `warmup` untimed steps, then `steps` timed
    steps, started together with the other cores."""
    import oracle as O
    import synth
    prob = synth.plate_impact(**ORACLE_SAMPLE)
    p, s = O.from_problem(prob)
    O.eval_rates(p, s)
    if warmup:
        O.step(p, s, warmup, rates_valid=True)
    barrier.wait(ORACLE_TIMEOUT_S)
    t0 = time.perf_counter()
    O.step(p, s, steps, rates_valid=True)
    results.put((prob.n, time.perf_counter() - t0))


def host_cores() -> int:
    """The host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_on_cores(steps: int, warmup: int = 0, cores: int = 0):
    """Time the FP64 CPU oracle, as it stands, on `cores` host cores at once
    (default: all of them): one spawned process per core (spawned, so that no
    CUDA context is forked), each advancing its own ORACLE_SAMPLE plate.
    Returns (particle-steps/s of the whole job, seconds of the slowest
    process, cores, particles per process)."""
    import multiprocessing as mp
    import queue
    import oracle
    oracle.build()                      # compiled once, before the processes load it
    cores = cores or host_cores()
    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(cores), ctx.Queue()
    procs = [ctx.Process(target=_oracle_core, args=(steps, warmup, barrier, results), daemon=True)
             for _ in range(cores)]
    for pr in procs:
        pr.start()
    try:
        out = [results.get(timeout=ORACLE_TIMEOUT_S) for _ in procs]
    except queue.Empty:
        raise RuntimeError("oracle baseline: a host process did not report") from None
    finally:
        for pr in procs:
            pr.join(timeout=10)
            if pr.is_alive():
                pr.terminate()
    n = out[0][0]
    sec = max(t for _, t in out)
    return n * cores * steps / sec, sec, cores, n


def run_reference(args, rank: int):
    """--impl reference: the oracle on the host cores, one bounded sample per
    step and core."""
    if rank != 0:
        return None
    value, sec, cores, n = oracle_on_cores(args.steps, args.warmup)
    sample = (f"oracle (plain FP64 C, single-threaded) in {cores} processes, one per host core, each on its own "
              f"{n:,}-particle sample of the plate impact (25^3 projector, 50x50x25 slab), "
              f"{args.steps} timed steps after {args.warmup} warm-up steps")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_particles": n * cores}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of the ranks' values of x (the slowest rank's time); x
    itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_per_rank: int, world: int, steps: int, ms: float) -> float:
    """Whole-job particle-steps/s of `world` replicas of an n_per_rank-particle
    workload, each advanced `steps` steps, the slowest taking ms."""
    return n_per_rank * world * steps / (ms * 1e-3)


def run_gpu(args, rank: int, world: int, local_rank: int):
    import torch
    import synth
    from paper_1805_05128_gb300 import Simulation, build
    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    prob = synth.plate_impact(units=64, n_steps=500, **WORKLOADS[args.workload])
    gen = synth.problem_generators(prob)
    sim = Simulation(prob, precision=args.precision, generators=gen, n_upd=10, cell_beta=args.beta,
                     list_staging=args.staging, device=dev)
    sim.assign()
    sim.build_cells()
    sim.step(max(args.warmup, 3))
    torch.cuda.synchronize()

    # ---- device-resident timed region
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[0]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local_rank
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    builds0 = sim.list_builds()[0] if args.beta > 0 else 0
    with ClockSampler(gpu_index) as clk:
        sim.profile(True)
        e0.record()
        sim.step(args.steps)            # one sph_step call runs the K steps, as a simulation does
        e1.record()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    pair_ms, pair_launches, launches = sim.profile_read()
    sim.profile(False)
    half_pairs, candidates, fp64_checks = sim.pair_counts()
    builds = (sim.list_builds()[0] - builds0) if args.beta > 0 else args.steps
    status = sim.read_status()
    ms = max_over_ranks(ms, dist, dev)

    # ---- the same K steps captured in one CUDA graph (fewer launch gaps), replayed
    # once untimed and once timed; the state simply advances
    graph_ms, graph_builds = None, 0
    if not args.no_graph:
        from paper_1805_05128_gb300.ensemble import GraphRun
        gr = GraphRun(sim, args.steps)
        gr.replay()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        gb0 = sim.list_builds()[0] if args.beta > 0 else 0
        e0.record()
        gr.replay()
        e1.record()
        torch.cuda.synchronize()
        graph_builds = (sim.list_builds()[0] - gb0) if args.beta > 0 else args.steps
        graph_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        status = status or sim.read_status()
        del gr
    n_total = prob.n * world
    value = job_value(prob.n, world, args.steps, ms)

    # ---- end to end: host state in pinned memory, copied in and out every step
    e2e_value, e2e_steps, h2d, d2h = None, 0, 0, 0
    fields = [k for k in ("x", "y", "z", "vx", "vy", "vz", "rho", "E", "m", "ax", "ay", "az", "drho", "dE")]
    if not args.no_e2e:
        host = {k: torch.empty(prob.n, dtype=torch.float64, pin_memory=True) for k in fields}
        for k in fields:
            host[k].copy_(sim.t[k])
        torch.cuda.synchronize()
        e2e_steps = max(1, min(args.steps, 20))
        h2d = sum(host[k].numel() * 8 for k in fields)
        d2h = h2d
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        main = torch.cuda.current_stream(dev)
        copy = torch.cuda.Stream(dev)
        ready = [torch.cuda.Event() for _ in fields]
        if dist:
            dist.barrier()
        f0.record()
        # every step: the state in from the pinned host arrays, one step, the state
        # out; field k of the next step's input is copied in (on a second stream,
        # the other copy direction) as soon as its read-back has landed
        copy.wait_stream(main)
        with torch.cuda.stream(copy):
            for k in fields:
                sim.t[k].copy_(host[k], non_blocking=True)
        for it in range(e2e_steps):
            main.wait_stream(copy)
            sim.step(1)
            for q, k in enumerate(fields):
                host[k].copy_(sim.t[k], non_blocking=True)
                ready[q].record(main)
            if it + 1 < e2e_steps:
                with torch.cuda.stream(copy):
                    for q, k in enumerate(fields):
                        copy.wait_event(ready[q])
                        sim.t[k].copy_(host[k], non_blocking=True)
        f1.record()
        torch.cuda.synchronize()
        e2e_ms = f0.elapsed_time(f1)
        e2e_ms = max_over_ranks(e2e_ms, dist, dev)
        e2e_value = job_value(prob.n, world, e2e_steps, e2e_ms)

    if rank != 0:
        return None
    # ---- roofline of the dominant kernel (pair loop, FP32 ALU)
    pair_ms_avg = pair_ms / max(pair_launches, 1)
    flops = FLOP_PAIR * half_pairs + FLOP_TEST * candidates / 2.0
    achieved = flops / (pair_ms_avg * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    traffic = pair_traffic_bytes(args) if args.workload == WORKLOAD else None
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "particles": prob.n, "precision": args.precision, "units": 64,
                      "verlet_beta": args.beta, "list_builds": builds, "operand_staging": bool(args.staging),
                      "rebalance_every": 10, "l2": "inputs larger than L2 (no flush)",
                      "parallelism": f"replicas{world}" if world > 1 else "single"},
           "pair_interactions_per_s": half_pairs * world * args.steps / (ms * 1e-3),
           "half_pairs_per_step": half_pairs, "candidates_per_step": candidates,
           "fp64_pair_checks_per_step": fp64_checks,
           "roofline": {"kernel": "k_pair_lists" if args.beta > 0 else "k_pair", "bound": "alu",
                        "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": traffic,
                        "peak_note": "FP32 152 SM x 128 lanes x 2 x 2.07 GHz (derived from unit counts and clock)",
                        "pair_ms_per_launch": pair_ms_avg, "pair_share": pair_ms / ms,
                        "issue_active": None if traffic is None else pair_profile_value(args, "issue_active_frac"),
                        "issue_note": "fraction of the kernel's issue slots used (ncu, the committed summary): "
                                      "the kernel is issue-bound, the FP32 fraction counts algorithmic flops only"},
           "graph": None if graph_ms is None else {
               "ms_per_step": graph_ms / args.steps,
               "value": job_value(prob.n, world, args.steps, graph_ms), "list_builds": graph_builds,
               "form": "the same number of steps captured in one CUDA graph (ensemble.GraphRun) and replayed "
                       "after the timed eager region; no per-kernel events inside the graph"},
           "clocks": clk.summary(), "gpu_launches": launches, "device_status": status,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "form": "14 FP64 state arrays copied in from pinned host memory and out again every step "
                           "(one sph_step call per step); each array's next copy-in on a second stream as soon "
                           "as its copy-out has landed",
                   "steps": e2e_steps}}
    if world == 1 and not args.no_extras:
        sim.close()
        out["extras"] = run_extras(args, dev)
    if world == 1 and not args.no_cpu_baseline:
        cval, csec, cores, cn = oracle_on_cores(args.cpu_steps)
        out["cpu_baseline"] = {"value": cval, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"plain FP64 C oracle (single-threaded) in {cores} processes, one per host "
                                         f"core, each on its own {cn:,}-particle sample of the plate impact, "
                                         f"{args.cpu_steps} steps after one rate evaluation ({csec:.1f} s)"}
    return out


def _fields_rel(a: dict, b: dict, keys) -> dict:
    out = {}
    for k in keys:
        d = np.abs(a[k] - b[k])
        out[k] = {"max_rel": float(d.max() / max(np.abs(b[k]).max(), 1e-300)),
                  "l1_rel": float(d.mean() / max(np.abs(b[k]).mean(), 1e-300))}
    return out


def run_extras(args, dev) -> dict:
    """The other forms on the same GPU: precision (FP64 vs mixed step on the
    benchmark plate, no work units, mesh and search every step), neighbour
    search (per-step mesh and search vs Verlet lists on the benchmark
    configuration), a second 3D workload (the Mie-Grueneisen lead ejecta
    sample), the 10M-particle droplet collision at 1:1000 density (mixed vs
    FP64), batching (256-instance ensemble, 100 steps in one CUDA
    graph, autotuned, vs 256 sequential single-instance runs) and
    differentiation (forward + reverse mode of a 203k-particle plate, 100
    steps, checkpoints every 10); the Voronoi units as the list kernel's work
    partition (global queue, per-unit queues with and without stealing, VD3
    against the static decomposition); and the disk test of Sec. 5."""
    import torch
    import synth
    from paper_1805_05128_gb300 import Simulation
    from paper_1805_05128_gb300 import ensemble as ens
    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)

    # (1) precision: same inputs, same number of steps
    prob = synth.plate_impact(units=0, n_steps=500, **WORKLOADS[args.workload])
    steps, res, states = 20, {}, {}
    for prec in ("fp64", "mixed"):
        sim = Simulation(prob, precision=prec, units=0, device=dev)
        sim.eval_rates()
        sim.step(2)
        torch.cuda.synchronize()
        sim.profile(True)
        e0, e1 = ev(), ev()
        e0.record()
        sim.step(steps)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        pair_ms, pair_launches, _ = sim.profile_read()
        half_pairs, candidates, _ = sim.pair_counts()
        flops = FLOP_PAIR * half_pairs + FLOP_TEST * candidates / 2.0
        peak = fp32_peak_tflops() if prec == "mixed" else FP64_PEAK_TFLOPS
        achieved = flops / (pair_ms / max(pair_launches, 1) * 1e-3) / 1e12
        res[prec] = {"value": prob.n * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                     "pair_ms_per_launch": pair_ms / max(pair_launches, 1),
                     "pair_roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                       "frac": achieved / peak}}
        states[prec] = sim.numpy()
        sim.close()
    res["fp64"]["pair_roofline"]["peak_note"] = "nominal GB300 FP64 (not measured)"
    res["mixed_vs_fp64_after_22_steps"] = _fields_rel(states["mixed"], states["fp64"], ("rho", "vz", "E", "z"))
    res["speedup_mixed_over_fp64"] = res["mixed"]["value"] / res["fp64"]["value"]
    out["precision"] = res

    # (2) neighbour search: the per-step mesh and pair search against Verlet lists (the
    # benchmark's work units and rebalancing, same inputs)
    prob_u = synth.plate_impact(units=64, n_steps=500, **WORKLOADS[args.workload])
    gen = synth.problem_generators(prob_u)
    ns = {}
    for beta in (0.0, args.beta if args.beta > 0 else BETA):
        sim = Simulation(prob_u, precision="mixed", generators=gen, n_upd=10, cell_beta=beta, device=dev)
        sim.assign()
        sim.build_cells()
        sim.step(10)
        b0 = sim.list_builds()[0] if beta > 0 else 0
        torch.cuda.synchronize()
        sim.profile(True)
        e0, e1 = ev(), ev()
        e0.record()
        sim.step(100)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        pair_ms, pair_launches, _ = sim.profile_read()
        ns["per_step_search" if beta == 0 else f"verlet_beta_{beta}"] = {
            "value": prob_u.n * 100 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / 100,
            "pair_kernel_ms": pair_ms / max(pair_launches, 1),
            "mesh_and_search_per_100_steps": 100 if beta == 0 else sim.list_builds()[0] - b0}
        sim.close()
    out["neighbour_search"] = ns

    # (3) a second 3D workload: the grooved lead sample (Mie-Grueneisen) on a rigid wall
    q = synth.ejecta(nx=100, periods=2, lam=40, nz=60, a=1e-7, units=64)
    gen = synth.problem_generators(q)
    sim = Simulation(q, precision="mixed", generators=gen, n_upd=10, cell_beta=BETA, device=dev)
    sim.assign()
    sim.build_cells()
    sim.step(10)
    b0 = sim.list_builds()[0]
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    sim.step(100)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    out["mg_ejecta"] = {"workload": f"grooved lead sample on a rigid wall (mirror copy), Mie-Grueneisen lead, "
                                    f"{q.n} particles, 0.1 um spacing, 64 units, beta {BETA}",
                        "value": q.n * 100 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / 100,
                        "list_builds_per_100_steps": sim.list_builds()[0] - b0, "status": sim.read_status()}
    sim.close()

    # (4) the droplet collision with a 1:1000 density contrast (10.1M particles): the
    # mixed step with lists against the plain FP64 GPU step on the same inputs
    q = synth.droplets()
    gen = synth.problem_generators(q)
    dro = {"workload": f"two Tait droplets (4M particles each, radius 1 mm, 300 m/s) in ideal gas at 1:1000 "
                       f"density, {q.n} particles, 256 units (3D)"}
    for prec, beta, steps in (("mixed", BETA, 20), ("fp64", 0.0, 2)):
        sim = Simulation(q, precision=prec, generators=gen, n_upd=10, cell_beta=beta, device=dev)
        sim.assign()
        sim.build_cells()
        sim.step(2)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        sim.step(steps)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        dro[prec] = {"value": q.n * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
                     "verlet_beta": beta, "status": sim.read_status()}
        sim.close()
    dro["speedup_mixed_over_fp64"] = dro["mixed"]["value"] / dro["fp64"]["value"]
    out["droplets"] = dro
    del q

    # (5) batching
    probs = synth.ensemble()
    n_tot = sum(q.n for q in probs)
    tune = ens.autotune(probs, cell_betas=(0.0, 0.15, 0.3), pair_blocks=(3, 0), n_steps=5, reps=1, device=dev)
    sim, ms_b = ens.run_batched(probs, 100, tuning=tune, device=dev)
    st_b = sim.read_status()
    sim.close()
    sims, ms_s = ens.run_sequential(probs, 100, tuning=tune, device=dev)
    st_s = max(s.read_status() for s in sims)
    for s_ in sims:
        s_.close()
    out["ensemble"] = {
        "workload": "256 plate impacts, N log-uniform 5k-200k (seed 2018), v U[0.5,2] km/s, gamma U[1.5,3]",
        "particles": n_tot, "steps": 100,
        "batched": {"value": n_tot * 100 / (ms_b * 1e-3), "unit": UNIT, "ms": ms_b,
                    "form": "one handle, 256 instances, 100 steps in one CUDA graph replay (about 16 kernel "
                            "launches per step inside the graph, not one persistent kernel)", "status": st_b},
        "sequential": {"value": n_tot * 100 / (ms_s * 1e-3), "unit": UNIT, "ms": ms_s,
                       "form": "256 handles, each stepped 100 times eagerly in turn", "status": st_s},
        "speedup_batched_over_sequential": ms_s / ms_b,
        "tuning": {"cell_beta": tune.cell_beta, "pair_blocks_per_sm": tune.pair_blocks,
                   "ms_per_step": {f"{k[0]}/{k[1]}": v for k, v in tune.timings.items()}}}

    # (6) the Voronoi units as the work partition of the list kernel: the global
    # queue against per-unit queues with stealing and without (each unit owned by
    # the same number of CTAs), each with VD3 balancing (theta 0.25, sigma 0.5)
    # and with the static decomposition (gamma = theta = 0); 500 timed steps each,
    # then the tail ratio max_k / mean_k of the units' completion times in the
    # list kernel, sampled every 10 steps over 100 more steps
    out["unit_partition"] = run_unit_partition(args, dev)

    # (7) the disk test of Sec. 5 on the GPU
    out["disk_balancing"] = run_disk(dev)

    # (8) differentiation
    from paper_1805_05128_gb300.adjoint import RunSpec, csph_run
    q = synth.plate_impact(25, (120, 120, 13), a=1e-4, v=1000.0, units=0)
    A = q.arrays
    pos = torch.tensor(np.stack([A["x"], A["y"], A["z"]], axis=1), dtype=torch.float64, device=dev)
    proj = torch.tensor(A["vz"] < 0.0, device=dev).double()
    rear = torch.tensor(A["z"] < 0.5e-4, device=dev)
    m = torch.tensor(A["m"], dtype=torch.float64, device=dev)
    rho0, c0v, gv = 2700.0, 5300.0, 2.0
    adj = {}

    def grad_run(prec, n_steps, every, reverse="fp64"):
        v = torch.tensor(1000.0, dtype=torch.float64, device=dev, requires_grad=True)
        c0 = torch.tensor(c0v, dtype=torch.float64, device=dev, requires_grad=True)
        g = torch.tensor(gv, dtype=torch.float64, device=dev, requires_grad=True)
        vel = torch.zeros(q.n, 3, dtype=torch.float64, device=dev)
        vel = vel + torch.stack([torch.zeros_like(m), torch.zeros_like(m), -v * proj], dim=1)
        rho = torch.full((q.n,), rho0, dtype=torch.float64, device=dev)
        E = c0 * c0 / (g - 1.0) + 0.5 * vel[:, 2] ** 2
        spec = RunSpec(m=m, n_steps=n_steps, every=every, precision=prec, rho0=rho0, reverse=reverse)
        torch.cuda.synchronize()
        e0, e1, e2 = ev(), ev(), ev()
        e0.record()
        _, v1, _, _ = csph_run(pos, vel, rho, E, c0, g, spec)
        loss = v1[rear, 2].mean()
        e1.record()
        loss.backward()
        e2.record()
        e2.synchronize()
        return e0.elapsed_time(e1), e1.elapsed_time(e2), [v.grad.item(), c0.grad.item(), g.grad.item()]

    # fp64: FP64 forward and reverse; mixed: FP32 forward with FP64 adjoint accumulation (the pair
    # derivatives in FP64); mixed_fp32_reverse: the pair derivatives in FP32 with Kahan sums
    for name, prec, rev in (("fp64", "fp64", "fp64"), ("mixed", "mixed", "fp64"), ("mixed_fp32_reverse", "mixed", "fp32")):
        grad_run(prec, 10, 5, rev)                 # warm-up: first-use costs of the reverse path
        fwd, bwd, grad = grad_run(prec, 100, 10, rev)
        adj[name] = {"forward_ms": fwd, "backward_ms": bwd,
                     "value": q.n * 100 / ((fwd + bwd) * 1e-3), "unit": UNIT + " (forward + reverse)",
                     "grad": grad}
    g64 = np.array(adj["fp64"]["grad"])
    adj["mixed_vs_fp64_grad_max_rel"] = float(np.max(np.abs(np.array(adj["mixed"]["grad"]) - g64) / np.abs(g64)))
    adj["mixed_fp32_reverse_vs_fp64_grad_max_rel"] = float(
        np.max(np.abs(np.array(adj["mixed_fp32_reverse"]["grad"]) - g64) / np.abs(g64)))
    adj["workload"] = f"plate impact {q.n} particles, 100 steps, checkpoints every 10, d(rear-face v_z)/d(v, c0, gamma)"
    out["adjoint"] = adj
    return out


# (name, list-kernel schedule, theta, gamma of eq. (TotalOffset), load measure)
UNIT_FORMS = (("global_queue", "global", 0.25, 1.0, "pairs"), ("units_steal_vd3", "units", 0.25, 1.0, "pairs"),
              ("units_steal_static", "units", 0.0, 0.0, "pairs"),
              ("units_owned_vd3", "units_owned", 0.25, 1.0, "pairs"),
              ("units_owned_vd3_timed_loads", "units_owned", 0.25, 1.0, "time"),
              ("units_owned_static", "units_owned", 0.0, 0.0, "pairs"))


def run_unit_partition(args, dev, steps: int = 500) -> dict:
    """Step time of the benchmark plate for each work partition of the list
    kernel, and the spread of the units' completion times (Sec. 2: the step
    waits for the most loaded unit; balancing evens the loads)."""
    import torch
    import synth
    from paper_1805_05128_gb300 import Simulation
    prob = synth.plate_impact(units=64, n_steps=500, **WORKLOADS[args.workload])
    gen = synth.problem_generators(prob)
    res = {"workload": f"{prob.n} particles, 64 units, beta {BETA}, rebalanced every 10 steps, {steps} steps"}
    for name, sched, theta, gamma_b, load in UNIT_FORMS:
        sim = Simulation(prob, precision="mixed", generators=gen, n_upd=10, cell_beta=BETA, unit_sched=sched,
                         theta=theta, gamma_b=gamma_b, sigma=0.5, load_measure=load, device=dev)
        sim.assign()
        sim.build_cells()
        sim.step(10)
        torch.cuda.synchronize()
        sim.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sim.step(steps)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        pair_ms, pair_launches, _ = sim.profile_read()
        sim.profile(False)
        r = {"ms_per_step": ms / steps, "pair_ms_per_launch": pair_ms / max(pair_launches, 1),
             "value": prob.n * steps / (ms * 1e-3), "unit": UNIT}
        if sched != "global":
            tails = []
            for _ in range(10):
                sim.step(10)
                ends = sim.unit_times()[:, 1]
                tails.append(float(ends.max() / ends.mean()))
            r["tail_ratio_mean"] = float(np.mean(tails))
            r["tail_ratio_max"] = float(np.max(tails))
        r["status"] = sim.read_status()
        res[name] = r
        sim.close()
    return res


def run_disk(dev, iters: int = 45) -> dict:
    """The three-subdomain disk of Sec. 5 (127,230 particles at rest) balanced
    on the GPU through voronoi_assign / the rate evaluation / voronoi_balance;
    iterations until sum_k |g^_k - g_k| < 0.01 (eq. VDConvergence) for the
    paper's four variants.  The paper's initial generators are not given, so
    the counts are reported beside its 21 / 21 / 17 / 11, not compared."""
    import json as _json
    import synth
    from paper_1805_05128_gb300 import Simulation
    gold = _json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))["disk"]
    D = synth.disk(gold["particles"], gold["radius"], gold["height"])
    n, a = len(D["x"]), D["a"]
    prob = synth.Problem("disk", 3, dict(x=D["x"], y=D["y"], z=D["z"], vx=np.zeros(n), vy=np.zeros(n),
                                         vz=np.zeros(n), rho=np.ones(n), E=np.ones(n), m=np.full(n, a ** 3)),
                         [synth.MaterialSpec("ideal", 1.4)], eta=1.3, units=3, unit_dim=2)
    g0 = np.array([[0.0, 0.1], [-0.12, -0.25], [0.12, -0.25]])
    paper = {"two_body": (0.0, 0.0, 21), "three_body": (1.0, 0.0, 21), "both": (0.5, 0.0, 17),
             "both_cumulative": (0.5, 0.25, 11)}
    out = {"workload": f"disk r 0.45, height 0.1, {n} particles, 3 units, initial loads ~0.53/0.24/0.24",
           "criterion": "sum_k |g^_k - g_k| < 0.01"}
    for name, (sigma, theta, ref) in paper.items():
        sim = Simulation(prob, precision="fp64", generators=g0.copy(), n_upd=0, device=dev)
        first, imb = None, None
        for it in range(iters):
            sim.assign()
            sim.eval_rates()
            load, _ = sim.unit_stats()
            imb = float((load.max() - load.min()) / load.mean())
            shift = float(sim.balance(theta=theta, sigma=sigma, gamma_b=1.0, beta_sh=0.45)[0])
            if first is None and shift < 0.01:
                first = it + 1
        out[name] = {"sigma": sigma, "theta": theta, "iterations": first, "paper_iterations": ref,
                     "final_load_imbalance": imb}
        sim.close()
    return out


def pair_profile_value(args, key: str, profiles_dir: str | None = None):
    """A figure of the committed ncu summary of the benchmark's dominant
    kernel (`key: value` line); None unless the summary was taken on the
    current pair-kernel sources (kernel_rev) and the mixed path."""
    import re
    name = "k_pair_lists" if args.beta > 0 else "k_pair"
    path = os.path.join(profiles_dir or os.path.join(ROOT, "profiles"), f"{name}_plate_impact_387k.md")
    if args.precision != "mixed" or not os.path.exists(path):
        return None
    text = open(path).read()
    sha = re.search(r"kernel_sha1:\s*([0-9a-f]+)", text)
    val = re.search(re.escape(key) + r":\s*([0-9.]+)", text)
    if not sha or not val or sha.group(1) != kernel_rev():
        return None
    return float(val.group(1))


def pair_traffic_bytes(args, profiles_dir: str | None = None):
    """DRAM bytes per launch of the dominant kernel at the benchmark size,
    from its committed ncu summary (see pair_profile_value)."""
    v = pair_profile_value(args, "traffic_bytes_per_launch_1125k", profiles_dir)
    return None if v is None else int(v)


def kernel_rev() -> str:
    """Identifier of the pair-kernel sources the stored ncu figures belong to
    (the two pair translation units and the headers they include)."""
    import hashlib
    h = hashlib.sha1()
    for f in ("k_pair.cu", "k_pair_lists.cu", "pair_common.cuh", "step_math.cuh", "csph_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1805_05128_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="csph", choices=["csph", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--beta", type=float, default=BETA,
                    help="Verlet buffer beta (0: mesh and pairs found every step)")
    ap.add_argument("--cpu-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay of the K steps")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64-step, batched-ensemble and adjoint measurements")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--staging", action="store_true",
                    help="stage the list kernel's neighbour operands in shared memory with cp.async")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        out = run_gpu(args, rank, world, local_rank)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
