"""The 2D path (dim = 2: the kernels' DIM = 2 instances) against the oracle on
the plate impact in a plane: cell indices and pair sets bit-exact, rates to
1e-10 (FP64) and 1e-4 (mixed), FP64 steps to 1e-10 with the per-step search
and with Verlet lists across rebuilds, mixed steps with lists from the GPU's
own state to 1e-4, conservation, and work units with rebalancing in 2D."""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_05128_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _plate(v=1000.0, seed=7):
    """Jittered 2D plate with a perturbed velocity field (every rate term)."""
    prob = synth.plate_impact_2d(12, (40, 8), a=1e-4, v=v, seed=seed, jitter=0.05)
    A = prob.arrays
    e = A["E"] - 0.5 * (A["vx"] ** 2 + A["vy"] ** 2)
    u = synth.uniform(seed + 100, 2 * prob.n)
    A["vx"] = A["vx"] + 30.0 * (u[0::2] - 0.5)
    A["vy"] = A["vy"] + 30.0 * (u[1::2] - 0.5)
    A["E"] = e + 0.5 * (A["vx"] ** 2 + A["vy"] ** 2)
    return prob


def _sim(prob, precision, **kw):
    from paper_1805_05128_gb300 import Simulation
    return Simulation(prob, precision=precision, units=kw.pop("units", 0), **kw)


KEYS = ("x", "y", "vx", "vy", "rho", "E", "drho", "ax", "ay", "dE")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_2d_pair_set_bitexact(precision):
    prob = _plate()
    sim = _sim(prob, precision)
    gi, gj = sim.pair_list()
    g = sim.numpy()
    p, _ = O.from_problem(prob)
    s = O.State(2, {k: g[k] for k in O.State.FIELDS + O.State.DERIVED if k in g}, prob.mat)
    oi, oj = O.pairs(p, s, "cells")
    assert len(gi) == len(oi) > 0
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
    sim.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_2d_rates_parity(precision, tol):
    prob = _plate()
    sim = _sim(prob, precision)
    sim.eval_rates()
    g = sim.numpy()
    p, s = O.from_problem(prob)
    O.eval_rates(p, s)
    for k in ("drho", "dE", "ax", "ay"):
        assert _rel(g[k], getattr(s, k)) <= tol, (k, _rel(g[k], getattr(s, k)))
    sim.close()


@pytest.mark.parametrize("beta", [0.0, 0.3])
def test_2d_fp64_steps(beta):
    prob = _plate(v=6000.0, seed=3)          # fast: the lists are rebuilt within the run
    sim = _sim(prob, "fp64", cell_beta=beta)
    p, s = O.from_problem(prob)
    t = 0.0
    for step in range(12):
        sim.step(1)
        t, _ = O.step(p, s, 1, rates_valid=step > 0, t=t)
        g = sim.numpy()
        for k in KEYS:
            assert _rel(g[k], getattr(s, k)) <= 1e-10, (step, k, _rel(g[k], getattr(s, k)))
    assert float(sim.time[0]) == pytest.approx(t, rel=1e-13)
    if beta > 0:
        assert 2 <= sim.list_builds()[0] < 12
    assert sim.read_status() == 0
    sim.close()


def test_2d_mixed_lists_one_step_parity():
    prob = _plate(v=6000.0, seed=3)
    sim = _sim(prob, "mixed", cell_beta=0.3)
    sim.step(1)
    for step in range(8):
        g0 = sim.numpy()
        p, _ = O.from_problem(prob)
        s = O.State(2, {k: g0[k] for k in O.State.FIELDS + O.State.DERIVED if k in g0}, prob.mat)
        dt = torch.zeros(1, dtype=torch.float64, device=sim.device)
        sim.step(1)
        sim.last_dt(dt)
        O.step_replay(p, s, [float(dt[0])], rates_valid=True)
        g = sim.numpy()
        for k in ("vx", "vy", "rho", "E", "drho", "ax", "ay", "dE"):
            assert _rel(g[k], getattr(s, k)) <= 1e-4, (step, k, _rel(g[k], getattr(s, k)))
    assert sim.read_status() == 0
    sim.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_2d_conservation_with_units(precision, tol):
    """Work units in the plane (unit_dim 2), rebalanced every 5 steps, with
    lists: mass exact, momentum and energy to the precision's rounding."""
    from paper_1805_05128_gb300 import Simulation
    prob = synth.plate_impact_2d(12, (40, 8), a=1e-4, v=3000.0, units=6, seed=5, jitter=0.05)
    gen = synth.problem_generators(prob)
    sim = Simulation(prob, precision=precision, generators=gen, n_upd=5, cell_beta=0.3)
    sim.assign()
    sim.build_cells()
    c0 = sim.conservation().cpu().numpy()[0]
    sim.step(25)
    c1 = sim.conservation().cpu().numpy()[0]
    g = sim.numpy()
    assert c1[0] == pytest.approx(c0[0], rel=1e-15)
    mom_scale = np.sum(g["m"] * np.sqrt(g["vx"] ** 2 + g["vy"] ** 2))
    for a in (1, 2):
        assert abs(c1[a] - c0[a]) <= tol * mom_scale, (a, abs(c1[a] - c0[a]) / mom_scale)
    assert abs(c1[4] - c0[4]) <= tol * abs(c0[4])
    assert sim.read_status() == 0
    sim.close()
