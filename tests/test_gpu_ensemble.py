"""Batched ensembles: independent plate impacts of uneven size, each with its
own impact speed and stiffened-gas gamma, as instances of one handle.

  * per-instance parity with the FP64 oracle run on each problem alone
    (mixed precision: max relative error <= 1e-4 after the steps);
  * a CUDA graph of the steps gives bit-for-bit the eager result;
  * the batched run gives bit-for-bit the sequential single-instance runs
    (same tuning), instance by instance;
  * the autotuner returns a candidate it timed, and the tuned run stays
    within the oracle tolerance.
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("x", "z", "vx", "vz", "rho", "E", "drho", "az", "dE")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_05128_gb300 import build
    build.build()


def _small(n_inst=10, seed=2018):
    return synth.ensemble(n_inst=n_inst, seed=seed, n_min=600, n_max=8000)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _check_oracle(sim, probs, n_steps, tol):
    g = sim.numpy()
    for b, prob in enumerate(probs):
        p, s = O.from_problem(prob)
        O.step(p, s, n_steps)
        lo, hi = sim.inst_offsets[b], sim.inst_offsets[b + 1]
        for k in FIELDS:
            err = _rel(g[k][lo:hi], getattr(s, k))
            assert err <= tol, (b, k, err)


def test_ensemble_instances_have_their_own_materials():
    from paper_1805_05128_gb300 import Simulation
    probs = _small()
    sim = Simulation(probs, precision="mixed", units=0)
    assert len(sim.materials) == len(probs) > 4            # goes through the host material table
    gam = np.array([q.materials[0].gamma for q in probs])
    assert len(np.unique(gam)) == len(probs)
    mat = sim.t["mat"].cpu().numpy()
    for b in range(len(probs)):
        lo, hi = sim.inst_offsets[b], sim.inst_offsets[b + 1]
        assert np.all(mat[lo:hi] == b)
    sim.close()


def test_ensemble_matches_oracle_per_instance():
    from paper_1805_05128_gb300 import Simulation
    probs = _small()
    sim = Simulation(probs, precision="mixed", units=0)
    sim.step(3)
    _check_oracle(sim, probs, 3, 1e-4)
    # per-instance dt: the time of each instance is its own (a mixed step takes
    # the CFL bound in FP32, so it agrees with the FP64 bound to ~1e-7)
    t = sim.time.cpu().numpy()
    for b, prob in enumerate(probs):
        p, s = O.from_problem(prob)
        _, dts = O.step(p, s, 3)
        assert t[b] == pytest.approx(float(np.sum(dts)), rel=1e-6)
    sim.close()


def test_graph_replay_equals_eager():
    from paper_1805_05128_gb300 import Simulation
    from paper_1805_05128_gb300.ensemble import GraphRun
    probs = _small(6, seed=7)
    eager = Simulation(probs, precision="mixed", units=0)
    eager.eval_rates()
    eager.step(8)
    graphed = Simulation(probs, precision="mixed", units=0)
    graphed.eval_rates()
    g = GraphRun(graphed, 4)
    g.replay()
    g.replay()
    a, b = eager.numpy(), graphed.numpy()
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(eager.time.cpu().numpy(), graphed.time.cpu().numpy())
    assert graphed.read_status() == 0
    eager.close()
    graphed.close()


def test_batched_equals_sequential():
    from paper_1805_05128_gb300.ensemble import run_batched, run_sequential
    probs = _small(8, seed=11)
    sim, _ = run_batched(probs, 5)
    sims, _ = run_sequential(probs, 5)
    gb = sim.numpy()
    for b, one in enumerate(sims):
        g1 = one.numpy()
        lo, hi = sim.inst_offsets[b], sim.inst_offsets[b + 1]
        for k in FIELDS:
            assert np.array_equal(gb[k][lo:hi], g1[k]), (b, k)
        assert float(sim.time[b]) == float(one.time[0])
        one.close()
    sim.close()


def test_autotune_picks_a_timed_candidate_and_stays_in_tolerance():
    from paper_1805_05128_gb300.ensemble import autotune, run_batched
    probs = _small(6, seed=3)
    t = autotune(probs, cell_betas=(0.0, 0.3), pair_blocks=(2, 0), n_steps=2, reps=1)
    assert (t.cell_beta, t.pair_blocks) in t.timings
    assert len(t.timings) == 4 and all(v > 0 for v in t.timings.values())
    assert t.timings[(t.cell_beta, t.pair_blocks)] == min(t.timings.values())
    sim, ms = run_batched(probs, 3, tuning=t)
    assert ms > 0 and sim.read_status() == 0
    _check_oracle(sim, probs, 3, 1e-4)
    sim.close()


@pytest.mark.parametrize("cell_beta,blocks", [(0.3, 2), (0.15, 1)])
def test_tuning_knobs_keep_parity(cell_beta, blocks):
    """Larger cells and a thinner persistent grid change the slot order, not
    the pair set: the result stays within the oracle tolerance."""
    from paper_1805_05128_gb300 import Simulation
    probs = _small(4, seed=5)
    sim = Simulation(probs, precision="mixed", units=0, cell_beta=cell_beta, pair_blocks_per_sm=blocks)
    sim.step(2)
    _check_oracle(sim, probs, 2, 1e-4)
    sim.close()


def test_batched_lists_rebuild_per_instance():
    """With Verlet lists each instance of a batched handle rebuilds its mesh,
    slots and lists when its own criterion fails (the others keep theirs), so
    over a run in which the instances rebuild at different steps every
    instance still steps bit for bit as it does alone."""
    from paper_1805_05128_gb300 import Simulation
    probs = _small(6, seed=23)
    batched = Simulation(probs, precision="mixed", units=0, cell_beta=0.15)
    batched.step(30)
    gb = batched.numpy()
    assert batched.read_status() == 0
    alone_builds = []
    for b, q in enumerate(probs):
        one = Simulation(q, precision="mixed", units=0, cell_beta=0.15)
        one.step(30)
        g1 = one.numpy()
        lo, hi = batched.inst_offsets[b], batched.inst_offsets[b + 1]
        for k in FIELDS:
            assert np.array_equal(gb[k][lo:hi], g1[k]), (b, k)
        alone_builds.append(one.list_builds()[0])
        one.close()
    # the instances' schedules differ, and the batched handle served all of them
    assert len(set(alone_builds)) > 1
    assert batched.list_builds()[0] >= max(alone_builds)
    batched.close()
