"""Verlet lists (cell_beta = beta > 0): sph_step keeps the pair lists over
(1 + beta) kappa h_ij, the mesh and the slot order between builds, and
rebuilds them on the device when the displacement/size criterion fails.

The oracle finds the exact pair set afresh every step, so parity with it
after steps that reuse the lists shows that no interacting pair was missing
from them: FP64 steps agree to 1e-10 per field; a mixed step from the GPU's
own previous state agrees to 1e-4.  Rebuild counts, graph capture and the
work-unit path are checked as well.
"""
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
    "sod": lambda: synth.sod_1d(),
    "plate": lambda: synth.plate_impact(6, (16, 16, 5), a=1e-4, v=1000.0, units=0, seed=7, jitter=0.05),
    # fast enough that the lists are rebuilt several times within the run
    "fast_plate": lambda: synth.plate_impact(5, (14, 14, 4), a=1e-4, v=6000.0, units=0, seed=3, jitter=0.05),
}


def _sim(prob, precision, beta=0.3, **kw):
    from paper_1805_05128_gb300 import Simulation
    return Simulation(prob, precision=precision, units=kw.pop("units", 0), cell_beta=beta, **kw)


@pytest.mark.parametrize("name,steps", [("sod", 30), ("plate", 12), ("fast_plate", 16)])
def test_fp64_lists_match_oracle_every_step(name, steps):
    prob = PROBLEMS[name]()
    sim = _sim(prob, "fp64")
    p, s = O.from_problem(prob)
    t = 0.0
    for step in range(steps):
        sim.step(1)
        t, _ = O.step(p, s, 1, rates_valid=step > 0, t=t)
        g = sim.numpy()
        for k in ("x", "vx", "rho", "E", "drho", "ax", "dE") + (("z", "vz", "az") if prob.dim == 3 else ()):
            assert _rel(g[k], getattr(s, k)) <= 1e-10, (step, k, _rel(g[k], getattr(s, k)))
    assert float(sim.time[0]) == pytest.approx(t, rel=1e-13)
    builds, cap = sim.list_builds()
    assert 1 <= builds <= steps and cap > 0
    if name == "fast_plate":
        assert 2 <= builds < steps, builds     # rebuilt, and reused in between
    assert sim.read_status() == 0
    sim.close()


@pytest.mark.parametrize("name", ["sod", "plate", "fast_plate"])
def test_mixed_lists_one_step_parity_along_the_run(name):
    """Each mixed step, taken from the GPU's own state (lists reused or
    rebuilt), against one oracle step from that same state."""
    prob = PROBLEMS[name]()
    sim = _sim(prob, "mixed")
    sim.step(1)
    keys = ("vx", "rho", "E", "drho", "ax", "dE") + (("vz", "az") if prob.dim == 3 else ())
    for step in range(10):
        g0 = sim.numpy()
        p, _ = O.from_problem(prob)
        s = O.State(prob.dim, {k: g0[k] for k in O.State.FIELDS + O.State.DERIVED if k in g0}, prob.mat)
        dt = torch.zeros(1, dtype=torch.float64, device=sim.device)
        sim.step(1)
        sim.last_dt(dt)
        O.step_replay(p, s, [float(dt[0])], rates_valid=True)
        g = sim.numpy()
        for k in keys:
            assert _rel(g[k], getattr(s, k)) <= 1e-4, (step, k, _rel(g[k], getattr(s, k)))
    assert sim.read_status() == 0
    sim.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_lists_conserve(precision, tol):
    prob = PROBLEMS["fast_plate"]()
    sim = _sim(prob, precision)
    c0 = sim.conservation().cpu().numpy()[0]
    sim.step(40)
    c1 = sim.conservation().cpu().numpy()[0]
    g = sim.numpy()
    assert c1[0] == pytest.approx(c0[0], rel=1e-15)
    mom_scale = np.sum(g["m"] * np.sqrt(g["vx"] ** 2 + g["vy"] ** 2 + g["vz"] ** 2))
    for a in (1, 2, 3):
        assert abs(c1[a] - c0[a]) <= tol * mom_scale, (a, abs(c1[a] - c0[a]) / mom_scale)
    assert abs(c1[4] - c0[4]) <= tol * abs(c0[4])
    assert sim.list_builds()[0] >= 2
    sim.close()


def test_slow_flow_reuses_one_build():
    prob = synth.plate_impact(5, (14, 14, 4), a=1e-4, v=20.0, units=0, seed=3, jitter=0.05)
    sim = _sim(prob, "mixed", beta=0.4)
    sim.step(20)
    assert sim.list_builds()[0] == 1
    assert sim.read_status() == 0
    sim.close()


def test_lists_inside_a_cuda_graph_equal_eager():
    from paper_1805_05128_gb300.ensemble import GraphRun
    prob = PROBLEMS["fast_plate"]()
    eager = _sim(prob, "mixed")
    eager.eval_rates()
    eager.step(12)
    graphed = _sim(prob, "mixed")
    graphed.eval_rates()
    g = GraphRun(graphed, 6)
    g.replay()
    g.replay()
    a, b = eager.numpy(), graphed.numpy()
    for k in ("x", "z", "vz", "rho", "E", "az"):
        assert np.array_equal(a[k], b[k]), k
    assert eager.list_builds()[0] == graphed.list_builds()[0] >= 2
    eager.close()
    graphed.close()


def test_lists_with_work_units_and_rebalancing():
    """Rebalancing renumbers the particles into slot order under the lists;
    the run stays within the one-step tolerance and conserves mass."""
    from paper_1805_05128_gb300 import Simulation
    prob = synth.plate_impact(6, (16, 16, 5), a=1e-4, v=3000.0, units=8, seed=7, jitter=0.05)
    gen = synth.problem_generators(prob)
    sim = Simulation(prob, precision="mixed", generators=gen, n_upd=5, cell_beta=0.3)
    sim.assign()
    sim.build_cells()
    m0 = float(sim.conservation().cpu().numpy()[0][0])
    sim.step(12)
    assert sim.list_builds()[0] >= 2
    g0 = sim.numpy()
    p, _ = O.from_problem(prob)
    s = O.State(prob.dim, {k: g0[k] for k in O.State.FIELDS + O.State.DERIVED if k in g0}, None)
    dt = torch.zeros(1, dtype=torch.float64, device=sim.device)
    sim.step(1)
    sim.last_dt(dt)
    O.step_replay(p, s, [float(dt[0])], rates_valid=True)
    g = sim.numpy()
    for k in ("vz", "rho", "E", "az", "drho"):
        assert _rel(g[k], getattr(s, k)) <= 1e-4, (k, _rel(g[k], getattr(s, k)))
    assert float(sim.conservation().cpu().numpy()[0][0]) == pytest.approx(m0, rel=1e-15)
    assert sim.read_status() == 0
    sim.close()


def test_lists_follow_a_body_in_uniform_motion():
    """The validity criterion bounds each particle's displacement since the
    build relative to one common displacement U (the bulk motion), which
    leaves every pair separation's bound unchanged: a lattice translating at
    3 km/s keeps its first build, where the displacements themselves exceed
    the per-particle buffer beta kh d many times; the FP64 run agrees with
    the oracle every step."""
    import dataclasses
    prob = synth.plate_impact(5, (14, 14, 4), a=1e-4, v=0.0, units=0, seed=3, jitter=0.05)
    arr = dict(prob.arrays)
    vz = np.full_like(arr["vz"], -3000.0)
    arr["E"] = arr["E"] - 0.5 * arr["vz"] ** 2 + 0.5 * vz ** 2
    arr["vz"] = vz
    prob = dataclasses.replace(prob, arrays=arr)
    beta = 0.3
    sim = _sim(prob, "fp64", beta=beta)
    p, s = O.from_problem(prob)
    z0 = arr["z"].copy()
    t = 0.0
    for step in range(20):
        sim.step(1)
        t, _ = O.step(p, s, 1, rates_valid=step > 0, t=t)
        g = sim.numpy()
        # (the rates themselves are rounding noise around zero here)
        for k in ("x", "z", "vz", "rho", "E"):
            assert _rel(g[k], getattr(s, k)) <= 1e-10, (step, k)
    kh = 0.5 * prob.kappa * prob.eta
    d = prob.arrays["m"][0] / prob.arrays["rho"][0]
    d = d ** (1.0 / 3.0)
    moved = float(np.max(np.abs(s.z - z0)))
    assert moved > 5 * beta * kh * d                  # the lab-frame bound would have rebuilt
    assert sim.list_builds()[0] == 1
    assert sim.read_status() == 0
    sim.close()


def test_lists_survive_the_renumbering_of_a_rebalance():
    """A rebalance (Alg. 1: shift the generators, reassign, renumber in cell
    order) permutes the particles into the slot order of the current mesh,
    so the lists, the mesh and the slots stay valid: a slow flow keeps its
    first build through four rebalances, and every FP64 step agrees with the
    oracle (which never renumbers) particle by particle to 1e-10."""
    from paper_1805_05128_gb300 import Simulation
    prob = synth.plate_impact(5, (14, 14, 4), a=1e-4, v=20.0, units=8, seed=3, jitter=0.05)
    gen = synth.problem_generators(prob)
    sim = Simulation(prob, precision="fp64", generators=gen, n_upd=3, cell_beta=0.4)
    sim.assign()
    p, s = O.from_problem(prob)
    t = 0.0
    for step in range(13):
        sim.step(1)
        t, _ = O.step(p, s, 1, rates_valid=step > 0, t=t)
        g = sim.numpy()
        order = np.argsort(g["id"])
        for k in ("x", "z", "vx", "vz", "rho", "E", "az", "drho", "dE"):
            assert _rel(g[k][order], getattr(s, k)) <= 1e-10, (step, k, _rel(g[k][order], getattr(s, k)))
    assert not np.array_equal(np.argsort(g["id"]), np.arange(len(g["id"])))   # renumbered
    assert sim.list_builds()[0] == 1
    assert sim.read_status() == 0
    sim.close()


def test_mixed_lists_survive_the_renumbering_of_a_rebalance():
    """The same in mixed precision, where the packed FP32 positions are
    offsets from each particle's cell origin: after four rebalances on the
    first build, a step from the GPU's own state agrees with the oracle's
    step from that state to 1e-4 (a particle paired with the wrong cell
    would be off by a cell width)."""
    from paper_1805_05128_gb300 import Simulation
    prob = synth.plate_impact(5, (14, 14, 4), a=1e-4, v=20.0, units=8, seed=3, jitter=0.05)
    gen = synth.problem_generators(prob)
    sim = Simulation(prob, precision="mixed", generators=gen, n_upd=3, cell_beta=0.4)
    sim.assign()
    sim.step(13)
    g0 = sim.numpy()
    assert not np.array_equal(np.argsort(g0["id"]), np.arange(len(g0["id"])))   # renumbered
    p, _ = O.from_problem(prob)
    s = O.State(prob.dim, {k: g0[k] for k in O.State.FIELDS + O.State.DERIVED if k in g0}, None)
    dt = torch.zeros(1, dtype=torch.float64, device=sim.device)
    sim.step(1)
    sim.last_dt(dt)
    O.step_replay(p, s, [float(dt[0])], rates_valid=True)
    g = sim.numpy()
    for k in ("vx", "vz", "rho", "E", "ax", "az", "drho", "dE"):
        assert _rel(g[k], getattr(s, k)) <= 1e-4, (k, _rel(g[k], getattr(s, k)))
    assert sim.list_builds()[0] == 1
    assert sim.read_status() == 0
    sim.close()


def test_list_query_needs_lists():
    from paper_1805_05128_gb300 import CsphError
    prob = PROBLEMS["plate"]()
    sim = _sim(prob, "mixed", beta=0.0)
    with pytest.raises(CsphError):
        sim.list_builds()
    sim.close()


def test_mixed_lists_with_uneven_particle_sizes():
    """A jittered cloud whose particle sizes d = (m/rho)^(1/3) spread over a
    factor of two and whose velocities are random: the list build's
    candidate cull works with the largest size of each home group, so uneven
    sizes test that it keeps every pair within (1 + beta) kappa h_ij.  Each
    mixed step over the lists against one oracle step (exact pair set) from
    the same state."""
    import dataclasses
    a, rho0, nx, ny, nz = 1e-4, 2700.0, 14, 14, 6
    n = nx * ny * nz
    k = np.arange(n)
    u = synth.uniform(41, 7 * n).reshape(7, n)
    x = (k % nx + 0.25 * (u[0] - 0.5)) * a
    y = ((k // nx) % ny + 0.25 * (u[1] - 0.5)) * a
    z = (k // (nx * ny) + 0.25 * (u[2] - 0.5)) * a
    m = rho0 * a ** 3 * 8.0 ** (u[3] - 0.5)
    v = 100.0 * (u[4:7] - 0.5)
    mat = synth.stiffened(rho0, 5300.0, 2.0)
    e0 = 2.0 * mat.p_inf / rho0
    arrays = dict(x=x, y=y, z=z, vx=v[0].copy(), vy=v[1].copy(), vz=v[2].copy(), rho=np.full(n, rho0),
                  E=e0 + 0.5 * np.sum(v * v, axis=0), m=m)
    base = synth.plate_impact(2, (2, 2, 2), a=a, units=0)
    prob = dataclasses.replace(base, name="uneven_cloud", arrays=arrays, materials=[mat], units=0)
    sim = _sim(prob, "mixed", beta=0.15)
    sim.step(1)
    for step in range(6):
        g0 = sim.numpy()
        p, _ = O.from_problem(prob)
        s = O.State(prob.dim, {k: g0[k] for k in O.State.FIELDS + O.State.DERIVED if k in g0}, prob.mat)
        dt = torch.zeros(1, dtype=torch.float64, device=sim.device)
        sim.step(1)
        sim.last_dt(dt)
        O.step_replay(p, s, [float(dt[0])], rates_valid=True)
        g = sim.numpy()
        for f in ("vx", "vy", "vz", "rho", "E", "drho", "ax", "ay", "az", "dE"):
            assert _rel(g[f], getattr(s, f)) <= 1e-4, (step, f, _rel(g[f], getattr(s, f)))
    assert sim.list_builds()[0] >= 1
    assert sim.read_status() == 0
    sim.close()
