"""GPU parity for the Tait and Mie-Grueneisen closures (the workloads of the
other tests use ideal and stiffened gases): rates to 1e-10 (FP64) and 1e-4
(mixed) against the oracle, FP64 steps to 1e-10 with the per-step search and
with Verlet lists, on a Tait water block, on the grooved lead ejecta sample
(Mie-Grueneisen lead, symmetric impact at 1 km/s) and on colliding Tait
droplets in an ideal gas at 1:1000 density (two materials in one instance)."""
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


PROBLEMS = {
    "water_tait": lambda: synth.water_block(side=8),
    "lead_ejecta": lambda: synth.ejecta(nx=16, periods=2, lam=8, nz=3, units=0),
    # Tait droplets in ideal gas, 1:1000 density (mass) contrast, two materials in one instance
    "droplets": lambda: synth.droplets(n_sphere=3000, n_gas=1500, units=0),
}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_eos_rates_parity(name, precision, tol):
    from paper_1805_05128_gb300 import Simulation
    prob = PROBLEMS[name]()
    if name == "lead_ejecta":        # compress it first so that P and the MG terms are non-trivial
        p, s = O.from_problem(prob)
        O.step(p, s, 15)
        for k in ("x", "y", "z", "vx", "vy", "vz", "rho", "E"):
            prob.arrays[k] = getattr(s, k).copy()
    sim = Simulation(prob, precision=precision, units=0)
    sim.eval_rates()
    g = sim.numpy()
    p, s = O.from_problem(prob)
    O.eval_rates(p, s)
    for k in ("drho", "dE", "ax", "ay", "az"):
        assert _rel(g[k], getattr(s, k)) <= tol, (k, _rel(g[k], getattr(s, k)))
    for k in ("P", "c"):
        scale = max(np.max(np.abs(getattr(s, k))), 1.0)
        assert np.max(np.abs(g[k] - getattr(s, k))) <= 1e-10 * scale, k
    sim.close()


@pytest.mark.parametrize("beta", [0.0, 0.2])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_eos_steps_fp64(name, beta):
    from paper_1805_05128_gb300 import Simulation
    prob = PROBLEMS[name]()
    sim = Simulation(prob, precision="fp64", units=0, cell_beta=beta)
    p, s = O.from_problem(prob)
    t = 0.0
    for step in range(10):
        sim.step(1)
        t, _ = O.step(p, s, 1, rates_valid=step > 0, t=t)
    g = sim.numpy()
    for k in ("x", "vx", "vz", "rho", "E", "drho", "ax", "az"):
        assert _rel(g[k], getattr(s, k)) <= 1e-10, (k, _rel(g[k], getattr(s, k)))
    assert float(sim.time[0]) == pytest.approx(t, rel=1e-13)
    assert sim.read_status() == 0
    sim.close()
