"""The Voronoi work units as the work partition of the list kernel (the
decomposition of Secs. 3-4 recast on one GPU): slots laid out unit-major,
per-unit queues with stealing (SPH_SCHED_UNITS) or without
(SPH_SCHED_UNITS_OWNED), against the single global queue.

The partition changes only which warp evaluates which slot, not the pair
set nor the order of any sum, so before the first rebalance (same particle
order) the three schedules give the same bits; after rebalances (the units
renumber the state unit-major) they stay within the oracle's tolerances."""
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


def _plate():
    return synth.plate_impact(8, (24, 24, 6), a=1e-4, v=1000.0, units=8, seed=41, jitter=0.05)


def _run(prob, sched, precision, steps, n_upd):
    from paper_1805_05128_gb300 import Simulation
    sim = Simulation(prob, precision=precision, generators=synth.problem_generators(prob), n_upd=n_upd,
                     cell_beta=0.15, unit_sched=sched)
    sim.assign()
    sim.step(steps)
    g = sim.numpy()
    assert sim.read_status() == 0
    return sim, g


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_schedules_agree_bitwise_before_a_rebalance(precision):
    prob = _plate()
    ref = None
    for sched in ("global", "units", "units_owned"):
        sim, g = _run(prob, sched, precision, 4, n_upd=10)
        sim.close()
        if ref is None:
            ref = g
            continue
        for k in ("x", "vx", "vz", "rho", "E", "ax", "az", "drho", "dE"):
            assert np.array_equal(g[k], ref[k]), (sched, k)


@pytest.mark.parametrize("sched", ["units", "units_owned"])
def test_unit_schedules_with_rebalancing_match_oracle(sched):
    prob = _plate()
    sim, g = _run(prob, sched, "fp64", 12, n_upd=4)
    p, s = O.from_problem(prob)
    O.step(p, s, 12)
    order = np.argsort(g["id"])
    for k in ("x", "z", "vx", "vz", "rho", "E"):
        a, b = g[k][order], getattr(s, k)
        assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b)), k
    # renumbered unit-major: each unit's particles are contiguous, in unit order
    u = g["unit"]
    assert np.all(np.diff(u) >= 0)
    # every unit has a start and an end time, ends after starts
    t = sim.unit_times()
    assert t.shape == (8, 2)
    assert np.all(t[:, 1] > t[:, 0]) and np.min(t[:, 0]) == 0.0
    sim.close()


def test_unit_times_need_the_unit_partition():
    from paper_1805_05128_gb300 import abi
    prob = _plate()
    sim, _ = _run(prob, "global", "mixed", 2, n_upd=10)
    with pytest.raises(abi.CsphError) as e:
        sim.unit_times()
    assert e.value.code == abi.SPH_ERR_INVALID


@pytest.mark.parametrize("sched", ["global", "units"])
def test_staged_operands_give_the_same_bits(sched):
    """list_staging = 1 copies each next chunk's neighbour operands into shared
    memory with cp.async; the arithmetic and its order are those of the
    gathers, so the states agree bit for bit, rebalancing included."""
    from paper_1805_05128_gb300 import Simulation
    prob = _plate()
    out = []
    for staging in (False, True):
        sim = Simulation(prob, precision="mixed", generators=synth.problem_generators(prob), n_upd=4,
                         cell_beta=0.15, unit_sched=sched, list_staging=staging)
        sim.assign()
        sim.step(9)
        out.append(sim.numpy())
        assert sim.read_status() == 0
        sim.close()
    for k in ("x", "vx", "vz", "rho", "E", "ax", "drho", "dE"):
        assert np.array_equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_list_evaluation_unit_statistics_match_oracle(precision):
    """The unit statistics of one evaluation over the Verlet lists (the form
    with side outputs: loads as interacting-pair counts, the adjacency
    through each block's shared tile merged into the K x K bits) equal the
    oracle's for the pair set of the evaluated state (Sec. 4.2-4.3)."""
    from paper_1805_05128_gb300 import Simulation
    prob = _plate()
    K = prob.units
    sim = Simulation(prob, precision=precision, generators=synth.problem_generators(prob), n_upd=0,
                     cell_beta=0.15)
    sim.assign()
    sim.eval_rates()
    sim.balance(theta=0.0, sigma=0.0, gamma_b=0.0)     # generators kept; accumulators cleared
    sim.step(1)                                         # one list evaluation with the side outputs
    load_g, adj_g = sim.unit_stats()
    g = sim.numpy()
    assert sim.read_status() == 0
    p, _ = O.from_problem(prob)
    s = O.State(prob.dim, {k: g[k] for k in O.State.FIELDS + O.State.DERIVED if k in g}, None)
    pi, pj = O.pairs(p, s)                              # the evaluated positions and sizes
    st = O.unit_stats(p, s, g["unit"], K, 2, pi, pj, 0.15)
    assert adj_g.sum() > 0 and np.array_equal(adj_g, st["adj"])
    assert np.array_equal(load_g, st["load"])
    sim.close()
