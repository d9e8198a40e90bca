"""GPU checks of the step's side results through the C ABI:

* the FP64 conservation sums (mass, momentum, total energy; the totals whose
  invariance the pair symmetry of eqs. SPH:Conti, SPH:Pulse and SPH:Energy
  implies) against the oracle's sums of the same state, per instance;
* the stiffened gas given by (rho0, c0, gamma), whose P_inf the library
  derives, against the same gas with P_inf passed explicitly;
* the device-side error latches (failure detection without a GPU fault):
  a Verlet list longer than its capacity, a cell holding more than 2047
  particles, and a work-unit id out of range each latch their code, which
  sph_read_status reports, and the kernels return normally.  Each case was
  read first: the list build writes only below the capacity and records the
  cut length, the pair search masks the in-cell offset into the cell, and
  the operand packing clamps the unit id, so every access stays in bounds.
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


def _stirred_plate(seed, proj=5, target=(12, 12, 4), v=900.0):
    """A jittered plate impact with a random velocity field added, so that
    every momentum component and the kinetic energy are non-trivial."""
    prob = synth.plate_impact(proj, target, a=1e-4, v=v, units=0, seed=seed, jitter=0.05)
    A = prob.arrays
    e = A["E"] - 0.5 * (A["vx"] ** 2 + A["vy"] ** 2 + A["vz"] ** 2)
    u = synth.uniform(seed + 100, 3 * prob.n)
    for a, k in enumerate(("vx", "vy", "vz")):
        A[k] = A[k] + 40.0 * (u[a::3] - 0.5)
    A["E"] = e + 0.5 * (A["vx"] ** 2 + A["vy"] ** 2 + A["vz"] ** 2)
    return prob


def _oracle_totals(arrays, lo, hi):
    s = O.State(3, {k: arrays[k][lo:hi] for k in O.State.FIELDS})
    return np.asarray(O.conservation(s))


def _check_totals(gpu, ref, arrays, lo, hi):
    """Mass and energy relative to themselves, momentum relative to
    sum m |v| (the total momentum of a plate impact may be near zero)."""
    m = arrays["m"][lo:hi]
    speed = np.sqrt(arrays["vx"][lo:hi] ** 2 + arrays["vy"][lo:hi] ** 2 + arrays["vz"][lo:hi] ** 2)
    mom_scale = float(np.sum(m * speed))
    assert abs(gpu[0] - ref[0]) <= 1e-12 * abs(ref[0])
    for a in (1, 2, 3):
        assert abs(gpu[a] - ref[a]) <= 1e-12 * mom_scale, (a, gpu[a], ref[a])
    assert abs(gpu[4] - ref[4]) <= 1e-12 * abs(ref[4])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_conservation_sums_match_oracle_one_instance(precision):
    from paper_1805_05128_gb300 import Simulation
    prob = _stirred_plate(5)
    sim = Simulation(prob, precision=precision, units=0, cell_beta=0.15)
    sim.step(7)
    tot = sim.conservation().cpu().numpy()
    g = sim.numpy()
    assert tot.shape == (1, 5)
    _check_totals(tot[0], _oracle_totals(g, 0, prob.n), g, 0, prob.n)
    assert sim.read_status() == 0


def test_conservation_sums_match_oracle_two_instances():
    from paper_1805_05128_gb300 import Simulation
    a, b = _stirred_plate(8), _stirred_plate(9, proj=4, target=(10, 10, 5), v=1400.0)
    sim = Simulation([a, b], precision="fp64", units=0)
    sim.step(4)
    tot = sim.conservation().cpu().numpy()
    g = sim.numpy()
    assert tot.shape == (2, 5)
    for k in range(2):
        lo, hi = sim.inst_offsets[k], sim.inst_offsets[k + 1]
        _check_totals(tot[k], _oracle_totals(g, lo, hi), g, lo, hi)


def test_stiffened_gas_from_c0_equals_explicit_p_inf():
    """SPH_EOS_STIFFENED_C0 (P_inf derived by the library) and SPH_EOS_STIFFENED
    with P_inf = rho0 c0^2 / gamma given by the caller run the same step."""
    from paper_1805_05128_gb300 import Simulation
    out = []
    for eos in ("stiffened", "stiffened_c0"):
        prob = _stirred_plate(3)
        m = prob.materials[0]
        prob.materials = [synth.MaterialSpec(eos, m.gamma, rho0=m.rho0, c0=m.c0,
                                             p_inf=m.p_inf if eos == "stiffened" else 0.0)]
        sim = Simulation(prob, precision="mixed", units=0)
        sim.step(3)
        out.append(sim.numpy())
        sim.close()
    for k in ("x", "vz", "rho", "E", "P", "c", "drho"):
        assert np.array_equal(out[0][k], out[1][k]), k


def test_list_capacity_overflow_latches():
    """Lists of 32 entries cannot hold the ~90 listed neighbours of a plate
    particle: the build cuts them and latches SPH_ERR_CAPACITY."""
    from paper_1805_05128_gb300 import Simulation, abi
    prob = synth.plate_impact(5, (12, 12, 4), a=1e-4, v=1000.0, units=0, seed=2, jitter=0.05)
    sim = Simulation(prob, precision="mixed", units=0, cell_beta=0.15, list_cap=32)
    assert sim.list_builds()[1] == 32
    sim.step(2)
    assert sim.read_status() == abi.SPH_ERR_CAPACITY
    assert sim.read_status() == abi.SPH_OK          # reading clears the word
    ok = Simulation(prob, precision="mixed", units=0, cell_beta=0.15)
    ok.step(2)
    assert ok.read_status() == abi.SPH_OK


def _crowded_cell():
    """2548 particles (a 14 x 14 x 13 lattice of spacing a, d = a) plus two
    particles of size 30 a far away: the cell edge of eq. (Dcell) follows the
    two largest sizes (1.3 (30 a + 30 a) = 78 a), so the whole lattice lies in
    one cell.  The large particles interact with nothing (137 a from the
    lattice against 1.3 x 31 a, 200 a apart against 78 a)."""
    a, rho0 = 1e-4, 2700.0
    g = np.arange(14) * a
    X, Y, Z = np.meshgrid(g, g, np.arange(13) * a, indexing="ij")
    x = np.concatenate([X.ravel(), [150 * a, 350 * a]])
    y = np.concatenate([Y.ravel(), [0.0, 0.0]])
    z = np.concatenate([Z.ravel(), [0.0, 0.0]])
    n = len(x)
    m = np.full(n, rho0 * a ** 3)
    m[-2:] = rho0 * (30 * a) ** 3
    mat = synth.stiffened(rho0, 5300.0, 2.0)
    e0 = 2.0 * mat.p_inf / ((2.0 - 1.0) * rho0)          # P = 0 at rho0
    arrays = dict(x=x, y=y, z=z, vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n), rho=np.full(n, rho0),
                  E=np.full(n, e0), m=m)
    return synth.Problem("crowded_cell", 3, arrays, [mat], units=0)


@pytest.mark.parametrize("beta", [0.0, 0.15])
def test_cell_over_2047_particles_latches(beta):
    from paper_1805_05128_gb300 import Simulation, abi
    prob = _crowded_cell()
    sim = Simulation(prob, precision="mixed", units=0, cell_beta=beta)
    sim.eval_rates()
    assert sim.read_status() == abi.SPH_ERR_CAPACITY


def test_unit_id_out_of_range_latches():
    from paper_1805_05128_gb300 import Simulation, abi
    prob = synth.plate_impact(5, (12, 12, 4), a=1e-4, v=1000.0, units=4, seed=4, jitter=0.05)
    sim = Simulation(prob, precision="mixed", generators=synth.problem_generators(prob))
    sim.assign()
    torch.cuda.synchronize()
    assert sim.read_status() == abi.SPH_OK
    sim.t["unit"][17] = 9                       # K = 4
    sim.eval_rates()
    assert sim.read_status() == abi.SPH_ERR_INVALID
