"""Batched ensembles of independent CSPH instances: a CUDA graph of many
steps over one multi-instance handle, an autotuner for the launch and mesh
knobs, and the sequential single-instance run it is compared against.

The instances are segments of one particle array (one handle, per-instance
mesh, dt and material), so every kernel of a step covers all of them; the
graph holds `n_steps` steps and is replayed with a single host call.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import torch

from .sim import Simulation


@dataclass
class Tuning:
    """Knobs of a handle that change speed but not the method:
    cell_beta   -- beta of eq. (Dcell): cells (1 + beta) times the minimum size;
    pair_blocks -- resident CTAs per SM of the persistent pair kernel
                   (4 warps each, one warp per home cell at a time)."""
    cell_beta: float = 0.0
    pair_blocks: int = 0
    timings: dict = field(default_factory=dict)   # (cell_beta, pair_blocks) -> ms per step


class GraphRun:
    """`n_steps` calls of sph_step captured once into a CUDA graph.

    The handle's rates must be valid before capture (eval_rates or a step),
    so that the captured work is exactly n_steps steps.  Replays advance the
    same state tensors in place."""

    def __init__(self, sim: Simulation, n_steps: int):
        self.sim, self.n_steps = sim, n_steps
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(sim.device)
        side.wait_stream(torch.cuda.current_stream(sim.device))
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                sim.step(n_steps)
        torch.cuda.current_stream(sim.device).wait_stream(side)

    def replay(self):
        self.graph.replay()


def cell_cap(problems) -> int:
    """Mesh capacity for a set of plate-like instances: one cell per particle
    (at least 4096) per instance, several times what their meshes use."""
    return int(sum(max(4096, len(q.arrays["x"])) for q in problems))


def _kw(problems, sim_kw: dict) -> dict:
    kw = dict(sim_kw)
    kw.setdefault("cell_cap", cell_cap(problems))
    return kw


def time_steps(sim: Simulation, n_steps: int, reps: int = 2) -> float:
    """Milliseconds per step of a graph of n_steps steps (best of reps)."""
    sim.eval_rates()
    g = GraphRun(sim, n_steps)
    g.replay()                                   # warm-up replay
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / n_steps)
    return best


def autotune(problems, precision: str = "mixed", cell_betas=(0.0, 0.15, 0.3), pair_blocks=(3, 4, 0),
             n_steps: int = 5, reps: int = 2, **sim_kw) -> Tuning:
    """Time every (cell_beta, pair_blocks) candidate on a scratch copy of the
    problems (a fresh handle each) and return the fastest.  pair_blocks = 0
    means as many CTAs per SM as fit."""
    best, table = None, {}
    for cb, pb in itertools.product(cell_betas, pair_blocks):
        sim = Simulation(problems, precision=precision, units=0, cell_beta=cb, pair_blocks_per_sm=pb,
                         **_kw(problems, sim_kw))
        try:
            ms = time_steps(sim, n_steps, reps)
            status = sim.read_status()
        finally:
            sim.close()
        if status != 0:
            continue                              # e.g. the mesh outgrew its capacity: not a candidate
        table[(cb, pb)] = ms
        if best is None or ms < table[best]:
            best = (cb, pb)
    if best is None:
        raise RuntimeError("no tuning candidate ran cleanly")
    return Tuning(cell_beta=best[0], pair_blocks=best[1], timings=table)


def run_batched(problems, n_steps: int, tuning: Tuning | None = None, precision: str = "mixed",
                **sim_kw) -> tuple[Simulation, float]:
    """All problems as instances of one handle, n_steps captured in one graph
    and replayed once.  Returns the simulation (advanced n_steps) and the
    replay's device time in ms."""
    t = tuning or Tuning()
    sim = Simulation(problems, precision=precision, units=0, cell_beta=t.cell_beta,
                     pair_blocks_per_sm=t.pair_blocks, **_kw(problems, sim_kw))
    sim.eval_rates()
    g = GraphRun(sim, n_steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.replay()
    e1.record()
    e1.synchronize()
    return sim, e0.elapsed_time(e1)


def run_sequential(problems, n_steps: int, tuning: Tuning | None = None, precision: str = "mixed",
                   **sim_kw) -> tuple[list, float]:
    """One handle per problem, created up front; then each instance's n_steps
    are launched eagerly, one instance after the other.  Returns the
    simulations and the device time of all the steps in ms."""
    t = tuning or Tuning()
    sims = [Simulation(q, precision=precision, units=0, cell_beta=t.cell_beta, pair_blocks_per_sm=t.pair_blocks,
                       **_kw([q], sim_kw)) for q in problems]
    for s in sims:
        s.eval_rates()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in sims:
        s.step(n_steps)
    e1.record()
    e1.synchronize()
    return sims, e0.elapsed_time(e1)
