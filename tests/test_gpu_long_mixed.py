"""Accuracy of the mixed-precision step (FP32 pair fluxes, FP64 positions
and time) over long 3D runs against the FP64 oracle from the same inputs.

Bound (the mixed path's long-run tolerance): after 200 steps, per field,
L1 = mean_i |a_i - b_i| / mean_i |b_i| <= 1e-3, particles matched by
identity.  The GPU runs its production configuration (Verlet lists with
beta = 0.15, work units rebalanced every 10 steps with renumbering); the
oracle runs its plain step (pairs found every step, no units), which
computes the same rates, so units and lists change the particle order and
the rounding but not the scheme.  The measured L1 of each field is printed
for the record.
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEPS = 200
FIELDS = ("x", "y", "z", "vx", "vy", "vz", "rho", "E")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_05128_gb300 import build
    build.build()


def _run_both(prob, K):
    from paper_1805_05128_gb300 import Simulation
    gen = synth.problem_generators(prob)
    sim = Simulation(prob, precision="mixed", generators=gen, n_upd=10, cell_beta=0.15)
    sim.assign()
    sim.step(STEPS)
    g = sim.numpy()
    assert sim.read_status() == 0
    t_gpu = float(sim.time[0])
    sim.close()
    p, s = O.from_problem(prob)
    t_orc, _ = O.step(p, s, STEPS)
    order = np.argsort(g["id"])
    l1 = {}
    for k in FIELDS:
        a, b = g[k][order], getattr(s, k)
        l1[k] = float(np.mean(np.abs(a - b)) / np.mean(np.abs(b)))
    return l1, t_gpu, t_orc


def test_plate_impact_3d_200_mixed_steps_l1():
    """A jittered 3D plate impact of 31,728 particles (12^3 projector at
    1 km/s onto a 50 x 50 x 12 slab, stiffened gas), 8 units in x-y."""
    prob = synth.plate_impact(12, (50, 50, 12), a=1e-4, v=1000.0, units=8, seed=31, jitter=0.05)
    l1, t_gpu, t_orc = _run_both(prob, 8)
    print("plate 200 steps L1:", {k: f"{v:.2e}" for k, v in l1.items()}, "time rel",
          abs(t_gpu - t_orc) / t_orc)
    assert abs(t_gpu - t_orc) <= 1e-5 * t_orc
    for k, v in l1.items():
        assert v <= 1e-3, (k, v)


def test_droplets_two_materials_200_mixed_steps_l1():
    """Two Tait water droplets approaching at 300 m/s in ideal gas at
    1:1000 density (7.7k particles), 8 units in 3D."""
    prob = synth.droplets(n_sphere=3000, n_gas=1500, units=8)
    l1, t_gpu, t_orc = _run_both(prob, 8)
    print("droplets 200 steps L1:", {k: f"{v:.2e}" for k, v in l1.items()}, "time rel",
          abs(t_gpu - t_orc) / t_orc)
    assert abs(t_gpu - t_orc) <= 1e-5 * t_orc
    for k, v in l1.items():
        assert v <= 1e-3, (k, v)
