"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated for this method):
  cell indices, pair sets, Voronoi ownership   bit-exact
  FP64 path, per field, one step / evaluation  max|a-b| / max|b| <= 1e-10
  mixed path (FP32 pair fluxes), one step      max|a-b| / max|b| <= 1e-4
  mixed path after 200 Sod steps               mean|a-b| / mean|b| <= 1e-3
"""
import numpy as np
import pytest

import oracle as O
import sod_exact
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_05128_gb300 import build
    build.build()


def _sim(prob, precision, **kw):
    from paper_1805_05128_gb300 import Simulation
    gen = kw.pop("generators", None)
    if prob.units and gen is None and kw.get("units", prob.units) > 0:
        gen = synth.problem_generators(prob)
    return Simulation(prob, precision=precision, generators=gen, **kw)


def _oracle_state(prob, arrays):
    """Oracle state holding the given arrays (GPU numpy dict or problem arrays)."""
    p, _ = O.from_problem(prob)
    keys = [k for k in O.State.FIELDS + O.State.DERIVED if k in arrays]
    s = O.State(prob.dim, {k: arrays[k] for k in keys}, prob.mat)
    return p, s


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _by_id(arr, ids):
    out = np.empty_like(arr)
    out[ids] = arr
    return out


PROBLEMS = {
    "sod": lambda: synth.sod_1d(),
    "plate": lambda: synth.plate_impact(6, (16, 16, 5), a=1e-4, v=1000.0, units=8, seed=7, jitter=0.05),
    "plate_lattice": lambda: synth.plate_impact(5, (12, 12, 4), a=1e-4, v=1000.0, units=4),
}


def _contrast():
    """3D lattice with a block of particles 8x lighter (size contrast 2:1)."""
    prob = synth.plate_impact(4, (14, 14, 6), a=1e-4, v=500.0, units=4, seed=3, jitter=0.1)
    x = prob.arrays["x"]
    light = x > 0.0
    prob.arrays["m"] = np.where(light, prob.arrays["m"] / 8.0, prob.arrays["m"])
    prob.arrays["rho"] = np.where(light, prob.arrays["rho"] / 8.0, prob.arrays["rho"])
    return prob


PROBLEMS["contrast"] = _contrast


# ------------------------------------------------------------ bit-exact sets
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_cell_index_bitexact(name):
    prob = PROBLEMS[name]()
    sim = _sim(prob, "fp64", units=0)
    cells, grid = sim.cell_index()
    g = sim.numpy()
    p, s = _oracle_state(prob, g)
    og, ocells = O.cell_grid(p, s)
    assert np.array_equal(grid[0, :3], og["x0"]) and grid[0, 3] == og["dc"]
    assert np.array_equal(grid[0, 4:7].astype(np.int64), og["dims"]) and grid[0, 7] == og["ncells"]
    assert np.array_equal(cells.astype(np.int64), ocells)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_pair_set_bitexact(name, precision):
    prob = PROBLEMS[name]()
    sim = _sim(prob, precision, units=0)
    gi, gj = sim.pair_list()
    g = sim.numpy()
    p, s = _oracle_state(prob, g)        # same x and the GPU's d
    oi, oj = O.pairs(p, s, "cells")
    assert len(gi) == len(oi) > 0
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
    hp, cand, nexact = sim.pair_counts()
    assert hp == len(oi) and cand >= 2 * hp


# ------------------------------------------------------------------- rates
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_rates_parity(name, precision, tol):
    prob = PROBLEMS[name]()
    if name == "plate":   # add a velocity field so every rate is exercised
        n = prob.n
        A = prob.arrays
        e = A["E"] - 0.5 * (A["vx"] ** 2 + A["vy"] ** 2 + A["vz"] ** 2)
        u = synth.uniform(17, 3 * n)
        for a, k in enumerate(("vx", "vy", "vz")):
            A[k] = A[k] + 50.0 * (u[a::3] - 0.5)
        A["E"] = e + 0.5 * (A["vx"] ** 2 + A["vy"] ** 2 + A["vz"] ** 2)
    sim = _sim(prob, precision, units=0)
    sim.eval_rates()
    g = sim.numpy()
    p, s = O.from_problem(prob)
    O.eval_rates(p, s)
    fields = ["drho", "dE", "ax", "d", "c"] + (["ay", "az"] if prob.dim == 3 else [])
    for k in fields:
        ftol = 1e-10 if k in ("d", "c") else tol
        assert _rel(g[k], getattr(s, k)) <= ftol, (k, _rel(g[k], getattr(s, k)))
    # P may vanish (rest state of a stiffened gas); its scale is then the stiffness P_inf
    pscale = max(np.max(np.abs(s.P)), max(m.p_inf for m in prob.materials))
    assert np.max(np.abs(g["P"] - s.P)) <= 1e-10 * pscale


# -------------------------------------------------------------------- steps
@pytest.mark.parametrize("name", ["sod", "plate"])
def test_step_parity_fp64(name):
    prob = PROBLEMS[name]()
    sim = _sim(prob, "fp64", units=0)
    p, s = O.from_problem(prob)
    t = 0.0
    for step in range(5):
        sim.step(1)
        t, _ = O.step(p, s, 1, rates_valid=step > 0, t=t)
        g = sim.numpy()
        for k in ("x", "vx", "rho", "E", "drho", "ax") + (("z", "vz", "az") if prob.dim == 3 else ()):
            assert _rel(g[k], getattr(s, k)) <= 1e-10, (step, k, _rel(g[k], getattr(s, k)))
    assert float(sim.time[0]) == pytest.approx(t, rel=1e-14)


@pytest.mark.parametrize("name", ["sod", "plate"])
def test_step_parity_mixed_one_step(name):
    prob = PROBLEMS[name]()
    sim = _sim(prob, "mixed", units=0)
    p, s = O.from_problem(prob)
    sim.step(1)
    O.step(p, s, 1)
    g = sim.numpy()
    for k in ("vx", "rho", "E", "drho", "ax", "dE") + (("vz", "az") if prob.dim == 3 else ()):
        assert _rel(g[k], getattr(s, k)) <= 1e-4, (k, _rel(g[k], getattr(s, k)))


def test_sod_mixed_200_steps_l1():
    prob = synth.sod_1d()
    sim = _sim(prob, "mixed", units=0)
    p, s = O.from_problem(prob)
    sim.step(prob.n_steps)
    O.step(p, s, prob.n_steps)
    g = sim.numpy()
    for k in ("rho", "vx", "E"):
        l1 = np.mean(np.abs(g[k] - getattr(s, k))) / np.mean(np.abs(getattr(s, k)))
        assert l1 <= 1e-3, (k, l1)


def test_sod_fp64_matches_oracle_and_exact():
    prob = synth.sod_1d()
    sim = _sim(prob, "fp64", units=0)
    sim.step(prob.n_steps)
    g = sim.numpy()
    t = float(sim.time[0])
    win = (g["x"] >= 0) & (g["x"] <= 1)
    ex, _, _, _ = sod_exact.sample(g["x"][win], t, 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    l1 = np.mean(np.abs(g["rho"][win] - ex))
    p, s = O.from_problem(prob)
    to, _ = O.step(p, s, prob.n_steps)
    win_o = (s.x >= 0) & (s.x <= 1)
    exo, _, _, _ = sod_exact.sample(s.x[win_o], to, 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    assert l1 == pytest.approx(np.mean(np.abs(s.rho[win_o] - exo)), rel=1e-8)
    assert l1 < 0.035


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_conservation_gpu(precision, tol):
    prob = PROBLEMS["plate"]()
    sim = _sim(prob, precision, units=0)
    c0 = sim.conservation().cpu().numpy()[0]
    sim.step(50)
    c1 = sim.conservation().cpu().numpy()[0]
    g = sim.numpy()
    assert c1[0] == pytest.approx(c0[0], rel=1e-15)
    mom_scale = np.sum(g["m"] * np.sqrt(g["vx"] ** 2 + g["vy"] ** 2 + g["vz"] ** 2))
    for a in (1, 2, 3):
        assert abs(c1[a] - c0[a]) <= tol * mom_scale, (a, abs(c1[a] - c0[a]) / mom_scale)
    assert abs(c1[4] - c0[4]) <= tol * abs(c0[4])
    assert sim.read_status() == 0


def test_determinism_bitwise():
    prob = PROBLEMS["plate"]()
    outs = []
    for _ in range(2):
        sim = _sim(prob, "mixed", units=0)
        sim.step(20)
        outs.append(sim.numpy())
    for k in ("x", "vx", "rho", "E", "ax", "drho"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


# ------------------------------------------------------------------- VD3
@pytest.mark.parametrize("name,K,gdim", [("plate", 8, 2), ("sod", 4, 1), ("plate", 8, 3)])
def test_assign_bitexact(name, K, gdim):
    prob = PROBLEMS[name]()
    prob.unit_dim = gdim
    prob.units = K
    gen = synth.problem_generators(prob)
    sim = _sim(prob, "fp64", units=K, generators=gen)
    offs = sim.assign()
    g = sim.numpy()
    pos = [prob.arrays[k] for k in ("x", "y", "z")[:gdim]]
    ref = O.voronoi_assign(pos, gen)
    assert np.array_equal(g["unit"], ref)
    assert np.array_equal(offs.cpu().numpy(), np.concatenate([[0], np.cumsum(np.bincount(ref, minlength=K))]))


def test_assign_ties_bitexact():
    """Particles exactly equidistant from several generators go to the smallest index."""
    prob = PROBLEMS["plate_lattice"]()
    a = prob.meta["a"]
    gen = np.array([[2 * a, 0.0], [-2 * a, 0.0], [0.0, 2 * a], [0.0, -2 * a]])   # on lattice lines
    prob.units, prob.unit_dim = 4, 2
    sim = _sim(prob, "fp64", units=4, generators=gen)
    sim.assign()
    ref = O.voronoi_assign([prob.arrays["x"], prob.arrays["y"]], gen)
    assert np.array_equal(sim.numpy()["unit"], ref)


@pytest.mark.parametrize("sigma,theta", [(0.0, 0.0), (0.5, 0.25), (1.0, 0.0)])
def test_balance_parity(sigma, theta):
    prob = PROBLEMS["plate"]()
    K = prob.units
    gen = synth.problem_generators(prob) + np.array([[3e-4, -2e-4]])   # start off balance
    sim = _sim(prob, "fp64", units=K, generators=gen.copy())
    sim.assign()
    gi, gj = sim.pair_list()
    load_g, adj_g = sim.unit_stats()
    shift = sim.balance(theta=theta, sigma=sigma, gamma_b=1.0, beta_sh=0.45)
    g = sim.numpy()
    newgen = sim.gen.cpu().numpy()
    p, s = _oracle_state(prob, g)
    st = O.unit_stats(p, s, g["unit"], K, 2, gi, gj, 0.45)
    assert np.array_equal(load_g, st["load"])
    assert np.array_equal(adj_g, st["adj"])
    ref, rshift, _ = O.balance(gen, st["load"], st["adj"], st["dsh"], st["centroid"], st["count"],
                               theta, sigma, 1.0)
    scale = np.max(np.abs(gen))
    assert np.max(np.abs(newgen - ref)) <= 1e-12 * scale
    assert float(shift[0]) == pytest.approx(rshift, rel=1e-10, abs=1e-15)


@pytest.mark.parametrize("sigma", [0.0, 0.5])
def test_balance_parity_3d(sigma):
    """3D decomposition (unit_dim = 3): two-body, and the four-body terms of
    mutually adjacent quadruples (rotation on their circumsphere)."""
    prob = PROBLEMS["plate"]()
    prob.unit_dim = 3
    K = prob.units
    gen = synth.problem_generators(prob) + np.array([[3e-4, -2e-4, 1e-4]])
    sim = _sim(prob, "fp64", units=K, generators=gen.copy())
    sim.assign()
    gi, gj = sim.pair_list()
    load_g, adj_g = sim.unit_stats()
    shift = sim.balance(theta=0.25, sigma=sigma, gamma_b=1.0, beta_sh=0.45)
    g = sim.numpy()
    newgen = sim.gen.cpu().numpy()
    p, s = _oracle_state(prob, g)
    st = O.unit_stats(p, s, g["unit"], K, 3, gi, gj, 0.45)
    assert np.array_equal(adj_g, st["adj"])
    ref, rshift, _ = O.balance(gen, st["load"], st["adj"], st["dsh"], st["centroid"], st["count"], 0.25, sigma, 1.0)
    scale = np.max(np.abs(gen))
    assert np.max(np.abs(newgen - ref)) <= 1e-12 * scale
    assert float(shift[0]) == pytest.approx(rshift, rel=1e-10, abs=1e-15)
    if sigma > 0:   # the four-body terms took part
        ref0, _, _ = O.balance(gen, st["load"], st["adj"], st["dsh"], st["centroid"], st["count"], 0.25, 0.0, 1.0)
        assert np.max(np.abs(ref - ref0)) > 1e-9 * scale


def test_step_with_rebalancing_runs_and_conserves():
    prob = PROBLEMS["plate"]()
    sim = _sim(prob, "mixed", units=prob.units, n_upd=5)
    sim.assign()
    c0 = sim.conservation().cpu().numpy()[0]
    sim.step(20)
    c1 = sim.conservation().cpu().numpy()[0]
    g = sim.numpy()
    assert sim.read_status() == 0
    assert c1[0] == pytest.approx(c0[0], rel=1e-15)
    # renumbering keeps each particle's identity and the units match the generators
    assert np.array_equal(np.sort(g["id"]), np.arange(prob.n))
    ref = O.voronoi_assign([g["x"], g["y"]], sim.gen.cpu().numpy())
    # units are from the last rebalance (step 20): positions unchanged since then
    assert np.array_equal(g["unit"], ref)


# -------------------------------------------------------------- instances
def test_two_instances_equal_separate_runs():
    a = synth.plate_impact(4, (10, 10, 4), a=1e-4, v=800.0, units=0, seed=1, jitter=0.05)
    b = synth.plate_impact(5, (12, 12, 3), a=1e-4, v=1200.0, units=0, seed=2, jitter=0.05)
    from paper_1805_05128_gb300 import Simulation
    both = Simulation([a, b], precision="fp64", units=0)
    both.step(5)
    gb = both.numpy()
    for k, prob in enumerate((a, b)):
        one = Simulation(prob, precision="fp64", units=0)
        one.step(5)
        g1 = one.numpy()
        lo, hi = both.inst_offsets[k], both.inst_offsets[k + 1]
        for f in ("x", "vz", "rho", "E"):
            assert np.array_equal(gb[f][lo:hi], g1[f]), (k, f)
        assert float(both.time[k]) == float(one.time[0])


# -------------------------------------------------------------- edge cases
@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_systems(n):
    x = np.arange(n, dtype=float) * 1e-4
    prob = synth.Problem("tiny", 3, dict(x=x, y=np.zeros(n), z=np.zeros(n), vx=np.linspace(-1, 1, n),
                                         vy=np.zeros(n), vz=np.zeros(n), rho=np.full(n, 2700.0),
                                         E=np.full(n, 2.809e7), m=np.full(n, 2.7e-9)),
                         [synth.stiffened(2700.0, 5300.0, 2.0)], units=0)
    sim = _sim(prob, "fp64", units=0)
    sim.step(3)
    p, s = O.from_problem(prob)
    O.step(p, s, 3)
    g = sim.numpy()
    for k in ("x", "vx", "rho", "E"):
        assert _rel(g[k], getattr(s, k)) <= 1e-10
    assert sim.read_status() == 0


def test_nonfinite_input_rejected():
    prob = PROBLEMS["plate_lattice"]()
    prob.arrays["rho"] = prob.arrays["rho"].copy()
    prob.arrays["rho"][7] = np.nan
    from paper_1805_05128_gb300 import abi
    with pytest.raises(abi.CsphError) as e:
        _sim(prob, "mixed", units=0)
    assert e.value.code == abi.SPH_ERR_NONFINITE
