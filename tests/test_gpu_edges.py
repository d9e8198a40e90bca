"""Degenerate inputs on the GPU: a single particle, particles without
neighbours, a one-particle instance beside a full one in a batched handle,
and coincident particles (r = 0: no direction, no flux, Sec. 4.1), each with
the per-step search and with Verlet lists, FP64 and mixed precision.  Empty
inputs are rejected on the host (tests/test_abi.py)."""
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


def _free(x, y, z, v, a=1e-4, rho0=2700.0, c0=5300.0, gamma=2.0):
    """Particles of lattice mass at rest density (P = 0) with velocities v."""
    n = len(x)
    mat = synth.stiffened(rho0, c0, gamma)
    e0 = gamma * mat.p_inf / ((gamma - 1.0) * rho0)
    v = np.asarray(v, dtype=np.float64).reshape(n, 3)
    arrays = dict(x=np.asarray(x, float), y=np.asarray(y, float), z=np.asarray(z, float),
                  vx=v[:, 0].copy(), vy=v[:, 1].copy(), vz=v[:, 2].copy(), rho=np.full(n, rho0),
                  E=e0 + 0.5 * np.sum(v * v, axis=1), m=np.full(n, rho0 * a ** 3))
    base = synth.plate_impact(2, (2, 2, 2), a=a, units=0)
    return dataclasses.replace(base, name=f"free_{n}", arrays=arrays, materials=[mat], units=0)


def _sim(prob, precision, beta):
    from paper_1805_05128_gb300 import Simulation
    return Simulation(prob, precision=precision, units=0, cell_beta=beta)


@pytest.mark.parametrize("beta", [0.0, 0.15])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_particle_moves_ballistically(precision, beta):
    prob = _free([1e-3], [-2e-3], [5e-4], [[12.5, -3.0, 7.25]])
    sim = _sim(prob, precision, beta)
    x0 = np.array([1e-3, -2e-3, 5e-4])
    sim.step(5)
    g = sim.numpy()
    assert sim.read_status() == 0
    t = float(sim.time[0])
    assert t > 0.0
    for k in ("ax", "ay", "az", "drho", "dE"):
        assert g[k][0] == 0.0, k
    assert np.array_equal([g["vx"][0], g["vy"][0], g["vz"][0]], [12.5, -3.0, 7.25])
    pos = np.array([g["x"][0], g["y"][0], g["z"][0]])
    assert np.allclose(pos, x0 + t * np.array([12.5, -3.0, 7.25]), rtol=0, atol=1e-15)
    assert sim.pair_counts()[0] == 0
    sim.close()


@pytest.mark.parametrize("beta", [0.0, 0.15])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_isolated_particles_have_no_pairs(precision, beta):
    """Four particles, each farther than the kernel support from the others."""
    a = 1e-4
    prob = _free([0.0, 10 * a, 0.0, 10 * a], [0.0, 0.0, 10 * a, 10 * a], [0.0, 0.0, 0.0, 5 * a],
                 [[1.0, 0.0, 0.0], [0.0, -2.0, 0.0], [0.0, 0.0, 3.0], [-1.0, 1.0, 0.0]])
    sim = _sim(prob, precision, beta)
    sim.step(3)
    g = sim.numpy()
    assert sim.read_status() == 0
    assert sim.pair_counts()[0] == 0
    for k in ("ax", "ay", "az", "drho", "dE"):
        assert np.all(g[k] == 0.0), k
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_particle_instance_beside_a_plate(precision):
    """A batched handle whose first instance is one particle: the plate
    instance steps exactly as it does alone (bit for bit), the lone particle
    ballistically."""
    from paper_1805_05128_gb300 import Simulation
    lone = _free([0.0], [0.0], [0.0], [[4.0, 0.0, -1.0]])
    plate = synth.plate_impact(5, (12, 12, 4), a=1e-4, v=1000.0, units=0, seed=9, jitter=0.05)
    both = Simulation([lone, plate], precision=precision, units=0, cell_beta=0.15)
    alone = Simulation(plate, precision=precision, units=0, cell_beta=0.15)
    both.step(6)
    alone.step(6)
    gb, ga = both.numpy(), alone.numpy()
    assert both.read_status() == 0 and alone.read_status() == 0
    for k in ("x", "z", "vx", "vz", "rho", "E", "az", "drho"):
        assert np.array_equal(gb[k][1:], ga[k]), k
        if k in ("az", "drho"):
            assert gb[k][0] == 0.0
    assert gb["vx"][0] == 4.0 and gb["vz"][0] == -1.0
    both.close()
    alone.close()


def test_coincident_particles_match_the_oracle():
    """Two particles at the same position inside a plate: their pair has no
    direction and adds nothing; every rate equals the oracle's (FP64, 1e-10)."""
    prob = synth.plate_impact(4, (10, 10, 4), a=1e-4, v=500.0, units=0, seed=2, jitter=0.05)
    arr = {k: v.copy() for k, v in prob.arrays.items()}
    for k in ("x", "y", "z"):
        arr[k][7] = arr[k][3]                  # particle 7 onto particle 3
    prob = dataclasses.replace(prob, arrays=arr)
    from paper_1805_05128_gb300 import Simulation
    for beta in (0.0, 0.15):
        sim = Simulation(prob, precision="fp64", units=0, cell_beta=beta)
        sim.step(1)
        g = sim.numpy()
        assert sim.read_status() == 0
        p, s = O.from_problem(prob)
        O.step(p, s, 1)
        for k in ("x", "z", "vx", "vz", "rho", "E", "ax", "az", "drho", "dE"):
            assert _rel(g[k], getattr(s, k)) <= 1e-10, (beta, k)
        sim.close()
