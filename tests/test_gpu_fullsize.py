"""Parity at the benchmark's full sizes, in the launch configurations that
bench.py times:

  * the 1.125M-particle plate impact (mixed precision, 64 work units
    rebalanced every 10 steps, Verlet lists beta = 0.15), after 20 steps with
    list rebuilds and two rebalances: ownership and the pair set bit-exact
    against the oracle on the GPU's own state, one further step within 1e-4
    of the oracle's step from that state (every particle), conservation;
  * the 10.1M-particle droplet collision (Tait liquid in ideal gas, 1:1000,
    256 units, lists): the rates of 256 sampled particles, each computed by
    the oracle from its own neighbourhood, within 1e-4; conservation;
  * the 256-instance ensemble (13.5M particles, one handle, one CUDA graph,
    the tuning the benchmark's autotuner picks): four sampled instances
    against the oracle run on each alone, within 1e-4.
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BETA = 0.15


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_05128_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _state(g, dim=3):
    return O.State(dim, {k: g[k] for k in O.State.FIELDS + O.State.DERIVED if k in g}, g.get("mat"))


def _conserved(c0, c1, g, tol):
    assert c1[0] == pytest.approx(c0[0], rel=1e-15)                 # mass: exact up to the sum's rounding
    mom = np.sum(g["m"] * np.sqrt(g["vx"] ** 2 + g["vy"] ** 2 + g["vz"] ** 2))
    for a in (1, 2, 3):
        assert abs(c1[a] - c0[a]) <= tol * mom, (a, abs(c1[a] - c0[a]) / mom)


def test_plate_impact_full_size():
    from paper_1805_05128_gb300 import Simulation
    prob = synth.plate_impact(50, (200, 200, 25), units=64, n_steps=500)
    assert prob.n == 1125000
    gen = synth.problem_generators(prob)
    sim = Simulation(prob, precision="mixed", generators=gen, n_upd=10, cell_beta=BETA)
    sim.assign()
    sim.build_cells()
    c0 = sim.conservation().cpu().numpy()[0]
    b0 = sim.list_builds()[0]
    sim.step(20)                                    # two rebalances, several list builds
    assert sim.list_builds()[0] - b0 >= 2
    assert sim.read_status() == 0
    _conserved(c0, sim.conservation().cpu().numpy()[0], sim.numpy(), 1e-6)
    # ownership with the generators the balancing produced, on the current positions
    offs = sim.assign().cpu().numpy()
    g = sim.numpy()
    gen_now = sim.gen.cpu().numpy()
    ref = O.voronoi_assign([g["x"], g["y"]], gen_now)
    assert np.array_equal(g["unit"], ref)
    assert np.array_equal(offs, np.concatenate([[0], np.cumsum(np.bincount(ref, minlength=64))]))
    # the pair set of the current state, given the GPU's sizes d
    gi, gj = sim.pair_list()
    g = sim.numpy()
    p, _ = O.from_problem(prob)
    oi, oj = O.pairs(p, _state(g), "cells")
    assert len(gi) == len(oi) > 35 * prob.n
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
    del gi, gj, oi, oj
    # one more step from the GPU's state, every particle
    sim.step(1)                                     # rates of this state for the next step's first kick
    g0 = sim.numpy()
    s = _state(g0)
    dt = torch.zeros(1, dtype=torch.float64, device=sim.device)
    sim.step(1)
    sim.last_dt(dt)
    O.step_replay(p, s, [float(dt[0])], rates_valid=True)
    g = sim.numpy()
    for k in ("x", "z", "vx", "vz", "rho", "E", "drho", "ax", "az", "dE"):
        assert _rel(g[k], getattr(s, k)) <= 1e-4, (k, _rel(g[k], getattr(s, k)))
    assert sim.read_status() == 0
    sim.close()


def _sampled_rates(prob, g, idx):
    """The oracle's rates of particles idx of state g, each from its own
    neighbourhood: the particles within kappa eta (d_i + d_max) / 2 (a k-d
    tree query), the oracle's sizes, P and c on that sub-state, the pairs
    r < kappa h_ij of i, and the oracle's rate sums over those pairs."""
    from scipy.spatial import cKDTree
    p, _ = O.from_problem(prob)
    pos = np.stack([g["x"], g["y"], g["z"]], axis=1)
    tree = cKDTree(pos)
    d_all = O.State(3, {k: g[k] for k in O.State.FIELDS}, g["mat"])
    O.derive(p, d_all)
    dmax = float(np.max(d_all.d))
    out = {k: np.zeros(len(idx)) for k in ("drho", "ax", "ay", "az", "dE")}
    for q, i in enumerate(idx):
        rad = prob.kappa * prob.eta * 0.5 * (d_all.d[i] + dmax) * (1 + 1e-6)
        nb = np.array(tree.query_ball_point(pos[i], rad), dtype=np.int64)
        nb = np.concatenate([[i], nb[nb != i]])
        sub = O.State(3, {k: g[k][nb] for k in O.State.FIELDS}, g["mat"][nb])
        O.derive(p, sub)
        dx, dy, dz = sub.x[1:] - sub.x[0], sub.y[1:] - sub.y[0], sub.z[1:] - sub.z[0]
        r2 = dx * dx + dy * dy + dz * dz
        R = prob.kappa * (prob.eta * 0.5 * (sub.d[0] + sub.d[1:]))
        j = np.nonzero(r2 < R * R)[0] + 1
        O.rates(p, sub, np.zeros(len(j), dtype=np.int32), j.astype(np.int32))
        for k in out:
            out[k][q] = getattr(sub, k)[0]
    return out


def test_droplets_full_size_sampled():
    from paper_1805_05128_gb300 import Simulation
    prob = synth.droplets()
    gen = synth.problem_generators(prob)
    sim = Simulation(prob, precision="mixed", generators=gen, n_upd=10, cell_beta=BETA)
    sim.assign()
    sim.build_cells()
    c0 = sim.conservation().cpu().numpy()[0]
    sim.step(12)                                    # one rebalance, list builds
    assert sim.read_status() == 0
    g = sim.numpy()
    _conserved(c0, sim.conservation().cpu().numpy()[0], g, 1e-6)
    # rates at the current state: 128 sampled liquid and 128 gas particles
    sim.eval_rates()
    g = sim.numpy()
    rng = np.random.default_rng(5128)
    idx = np.concatenate([rng.choice(np.nonzero(g["mat"] == m)[0], 128, replace=False) for m in (0, 1)])
    ref = _sampled_rates(prob, g, idx)
    for k in ref:
        for m in (0, 1):                            # each material against its own rate scale
            sel = g["mat"][idx] == m
            err = _rel(g[k][idx][sel], ref[k][sel])
            assert err <= 1e-4, (k, m, err)
    assert sim.read_status() == 0
    sim.close()


FIELDS = ("x", "z", "vx", "vz", "rho", "E", "drho", "az", "dE")


def test_ensemble_full_size_sampled():
    from paper_1805_05128_gb300.ensemble import Tuning, run_batched
    probs = synth.ensemble()
    assert len(probs) == 256 and sum(q.n for q in probs) > 13_000_000
    sim, _ = run_batched(probs, 5, tuning=Tuning(cell_beta=BETA, pair_blocks=0))
    assert sim.read_status() == 0
    g = sim.numpy()
    t = sim.time.cpu().numpy()
    sizes = np.array([q.n for q in probs])
    rng = np.random.default_rng(2018)
    picks = [int(np.argmin(sizes)), int(np.argmax(sizes))] + [int(b) for b in rng.choice(256, 2, replace=False)]
    for b in picks:
        p, s = O.from_problem(probs[b])
        _, dts = O.step(p, s, 5)
        lo, hi = sim.inst_offsets[b], sim.inst_offsets[b + 1]
        for k in FIELDS:
            err = _rel(g[k][lo:hi], getattr(s, k))
            assert err <= 1e-4, (b, k, err)
        assert t[b] == pytest.approx(float(np.sum(dts)), rel=1e-6)
    sim.close()
