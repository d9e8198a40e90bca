"""The Wendland C2 kernel (support kappa h, kappa = 1.936) on the GPU against
the oracle: pair sets bit-exact, rates to 1e-10 (FP64) and 1e-4 (mixed),
FP64 steps to 1e-10 with the per-step search and with Verlet lists across
rebuilds, in 1D (Sod) and 3D (jittered plate)."""
import dataclasses

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


def _wendland(prob):
    return dataclasses.replace(prob, kernel="wendland_c2", kappa=1.936)


def _plate(v=1000.0, seed=7):
    prob = synth.plate_impact(6, (16, 16, 5), a=1e-4, v=v, units=0, seed=seed, jitter=0.05)
    A = prob.arrays
    e = A["E"] - 0.5 * (A["vx"] ** 2 + A["vy"] ** 2 + A["vz"] ** 2)
    u = synth.uniform(seed + 50, 3 * prob.n)
    for c, k in enumerate(("vx", "vy", "vz")):
        A[k] = A[k] + 40.0 * (u[c::3] - 0.5)
    A["E"] = e + 0.5 * (A["vx"] ** 2 + A["vy"] ** 2 + A["vz"] ** 2)
    return _wendland(prob)


PROBLEMS = {"sod": lambda: _wendland(synth.sod_1d()), "plate": _plate}


def _sim(prob, precision, **kw):
    from paper_1805_05128_gb300 import Simulation
    return Simulation(prob, precision=precision, units=0, **kw)


def _keys(prob):
    return ["drho", "dE", "ax"] + (["ay", "az"] if prob.dim == 3 else [])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_wendland_pair_set_bitexact(name, precision):
    prob = PROBLEMS[name]()
    sim = _sim(prob, precision)
    gi, gj = sim.pair_list()
    g = sim.numpy()
    p, _ = O.from_problem(prob)
    assert p.kernel == O.KERNEL_WENDLAND_C2
    s = O.State(prob.dim, {k: g[k] for k in O.State.FIELDS + O.State.DERIVED if k in g}, prob.mat)
    oi, oj = O.pairs(p, s, "cells")
    assert len(gi) == len(oi) > 0
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
    sim.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_wendland_rates_parity(name, precision, tol):
    prob = PROBLEMS[name]()
    sim = _sim(prob, precision)
    sim.eval_rates()
    g = sim.numpy()
    p, s = O.from_problem(prob)
    O.eval_rates(p, s)
    for k in _keys(prob):
        assert _rel(g[k], getattr(s, k)) <= tol, (k, _rel(g[k], getattr(s, k)))
    sim.close()


@pytest.mark.parametrize("beta", [0.0, 0.3])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_wendland_fp64_steps(name, beta):
    prob = PROBLEMS[name]() if name == "sod" else _plate(v=6000.0, seed=3)
    sim = _sim(prob, "fp64", cell_beta=beta)
    p, s = O.from_problem(prob)
    t = 0.0
    keys = ["x", "vx", "rho", "E"] + _keys(prob) + (["z", "vz"] if prob.dim == 3 else [])
    for step in range(10):
        sim.step(1)
        t, _ = O.step(p, s, 1, rates_valid=step > 0, t=t)
        g = sim.numpy()
        for k in keys:
            assert _rel(g[k], getattr(s, k)) <= 1e-10, (step, k, _rel(g[k], getattr(s, k)))
    assert float(sim.time[0]) == pytest.approx(t, rel=1e-13)
    assert sim.read_status() == 0
    sim.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_wendland_mixed_list_step(name):
    """Mixed precision over Verlet lists (the list kernel compiled for the
    Wendland kernel): after a few steps with list builds, one step from the
    GPU's own state agrees with the oracle's step from that state to 1e-4."""
    prob = PROBLEMS[name]() if name == "sod" else _plate(v=6000.0, seed=3)
    sim = _sim(prob, "mixed", cell_beta=0.3)
    sim.step(6)
    g0 = sim.numpy()
    p, _ = O.from_problem(prob)
    s = O.State(prob.dim, {k: g0[k] for k in O.State.FIELDS + O.State.DERIVED if k in g0}, prob.mat)
    dt = torch.zeros(1, dtype=torch.float64, device=sim.device)
    sim.step(1)
    sim.last_dt(dt)
    O.step_replay(p, s, [float(dt[0])], rates_valid=True)
    g = sim.numpy()
    for k in ["x", "vx", "rho", "E"] + _keys(prob):
        assert _rel(g[k], getattr(s, k)) <= 1e-4, (k, _rel(g[k], getattr(s, k)))
    assert sim.list_builds()[0] >= 1 and sim.read_status() == 0
    sim.close()
