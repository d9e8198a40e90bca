"""Work-unit loads measured as time (load_measure = SPH_LOAD_TIME: the SM
cycles the pair kernel spends on each unit's particles, the useful time t^u_k
of eq. (load)) instead of pair counts.  The loads are positive for every
occupied unit and grow with the unit's share of the pairs, the balancing runs
on them (the generators move), and the physics is untouched: mass exact and
one step from the GPU's own state within 1e-4 of the oracle, with the
per-step search and with Verlet lists."""
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


@pytest.mark.parametrize("beta", [0.0, 0.3])
def test_timed_loads_drive_the_balance(beta):
    from paper_1805_05128_gb300 import Simulation
    prob = synth.plate_impact(6, (16, 16, 5), a=1e-4, v=3000.0, units=8, seed=7, jitter=0.05)
    gen0 = synth.problem_generators(prob)
    sim = Simulation(prob, precision="mixed", generators=gen0, n_upd=100, cell_beta=beta, load_measure="time")
    sim.assign()
    sim.build_cells()
    sim.step(3)                                   # no rebalance yet: the loads accumulate
    load, _ = sim.unit_stats()
    counts = np.bincount(sim.t["unit"].cpu().numpy(), minlength=8)
    assert np.all(load[counts > 0] > 0), load
    # more particles (so more pairs) take more time: the loads follow the counts
    assert np.corrcoef(load[counts > 0], counts[counts > 0])[0, 1] > 0.5
    sim.close()

    sim = Simulation(prob, precision="mixed", generators=gen0, n_upd=4, cell_beta=beta, load_measure="time")
    sim.assign()
    sim.build_cells()
    m0 = float(sim.conservation().cpu().numpy()[0][0])
    sim.step(9)                                   # two rebalances on timed loads
    assert not np.allclose(sim.gen.cpu().numpy(), gen0)
    assert float(sim.conservation().cpu().numpy()[0][0]) == pytest.approx(m0, rel=1e-15)
    g0 = sim.numpy()
    p, _ = O.from_problem(prob)
    s = O.State(3, {k: g0[k] for k in O.State.FIELDS + O.State.DERIVED if k in g0}, None)
    dt = torch.zeros(1, dtype=torch.float64, device=sim.device)
    sim.step(1)
    sim.last_dt(dt)
    O.step_replay(p, s, [float(dt[0])], rates_valid=True)
    g = sim.numpy()
    for k in ("vz", "rho", "E", "az", "drho"):
        assert _rel(g[k], getattr(s, k)) <= 1e-4, (k, _rel(g[k], getattr(s, k)))
    assert sim.read_status() == 0
    sim.close()


def test_load_measure_validated():
    from paper_1805_05128_gb300 import Simulation
    prob = synth.plate_impact(4, (8, 8, 3), a=1e-4, v=1000.0, units=0)
    with pytest.raises(KeyError):
        Simulation(prob, precision="mixed", load_measure="bytes")
