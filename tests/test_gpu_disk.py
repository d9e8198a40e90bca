"""The three-subdomain disk test of Sec. 5 on the GPU, through the C ABI
(voronoi_assign, the rate evaluation that counts the unit loads and their
adjacency, voronoi_balance), for the four variants of the paper: two-body
only (sigma = 0, theta = 0), three-body only (sigma = 1, theta = 0), both
(sigma = 0.5, theta = 0) and both with the cumulative movement (sigma = 0.5,
theta = 0.25); gamma = 1 throughout.

The first updates equal the oracle's (generators within 1e-10 of the
disk's size).  The qualitative results of Sec. 5 are asserted as in the
oracle's own test; the iteration counts to sum_k |g^_k - g_k| < 0.01
(eq. VDConvergence) depend on the paper's initial generators, which it does
not give: parity unpinned, they are printed beside the paper's 21/21/17/11
(and reported by the benchmark), not asserted."""
import json
import os

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
G0 = np.array([[0.0, 0.1], [-0.12, -0.25], [0.12, -0.25]])     # about 0.53 / 0.24 / 0.24 of the particles
VARIANTS = {"two_body": (0.0, 0.0), "three_body": (1.0, 0.0), "both": (0.5, 0.0), "both_cumulative": (0.5, 0.25)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_05128_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def disk_problem():
    g = GOLD["disk"]
    D = synth.disk(g["particles"], g["radius"], g["height"])
    n, a = len(D["x"]), D["a"]
    arrays = dict(x=D["x"], y=D["y"], z=D["z"], vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n),
                  rho=np.ones(n), E=np.ones(n), m=np.full(n, a ** 3))
    return synth.Problem("disk", 3, arrays, [synth.MaterialSpec("ideal", 1.4)], eta=1.3, units=3, unit_dim=2,
                         meta=dict(a=a))


def _gpu_iterate(prob, sigma, theta, iters=45):
    from paper_1805_05128_gb300 import Simulation
    sim = Simulation(prob, precision="fp64", generators=G0.copy(), n_upd=0)
    imb, shifts, gens = [], [], []
    for _ in range(iters):
        sim.assign()
        sim.eval_rates()
        load, adj = sim.unit_stats()
        imb.append((load.max() - load.min()) / load.mean())
        shifts.append(float(sim.balance(theta=theta, sigma=sigma, gamma_b=1.0, beta_sh=0.45)[0]))
        gens.append(sim.gen.cpu().numpy().copy())
    assert sim.read_status() == 0
    g = gens[-1]
    A = np.array([2 * (g[1] - g[0]), 2 * (g[2] - g[0])])
    b = np.array([g[1] @ g[1] - g[0] @ g[0], g[2] @ g[2] - g[0] @ g[0]])
    o = np.linalg.solve(A, b)                 # common point of the three subdomains
    sim.close()
    return dict(imb=imb, shifts=shifts, gens=gens, o=o,
                first_balanced=next(i for i, v in enumerate(imb + [0.0]) if v < 0.02),
                first_converged=next((i + 1 for i, v in enumerate(shifts) if v < 0.01), None))


def test_disk_first_updates_match_oracle(disk_problem):
    """Three balancing updates of the 'both, cumulative' variant: GPU = oracle."""
    prob = disk_problem
    gpu = _gpu_iterate(prob, 0.5, 0.25, iters=3)
    n = prob.n
    s = O.State(3, {k: prob.arrays[k] for k in ("x", "y", "z", "rho", "E", "m")})
    p = O.Params(dim=3, eta=1.3)
    O.derive(p, s)
    pi, pj = O.pairs(p, s)
    g = G0.copy()
    for it in range(3):
        unit = O.voronoi_assign([s.x, s.y], g)
        st = O.unit_stats(p, s, unit, 3, 2, pi, pj, 0.45)
        g, shift, _ = O.balance(g, st["load"], st["adj"], st["dsh"], st["centroid"], st["count"], 0.25, 0.5, 1.0)
        assert np.max(np.abs(gpu["gens"][it] - g)) <= 1e-10 * 0.45, it
        assert gpu["shifts"][it] == pytest.approx(shift, rel=1e-9)
    assert n > 127000


def test_disk_variants_on_gpu(disk_problem):
    res = {name: _gpu_iterate(disk_problem, *sv) for name, sv in VARIANTS.items()}
    two, three, comb, best = (res[k] for k in ("two_body", "three_body", "both", "both_cumulative"))
    dsh = 1.45 * 1.3 * 2 * disk_problem.meta["a"]     # D^sh of eq. (Horizon) on the lattice: (1 + beta) kh (d + d)
    assert best["imb"][-1] < 0.02 and comb["imb"][-1] < 0.02 and two["imb"][-1] < 0.02
    assert np.linalg.norm(best["o"]) < dsh                       # common point at the centre
    assert np.linalg.norm(two["o"]) > 2 * dsh                    # two-body: initial geometry kept
    assert np.linalg.norm(three["o"]) > 2 * dsh                  # three-body: common point stuck
    assert np.linalg.norm(best["o"]) < np.linalg.norm(comb["o"]) < np.linalg.norm(two["o"])
    assert best["first_balanced"] < comb["first_balanced"] < two["first_balanced"]
    assert best["first_converged"] is not None
    paper = {"two_body": 21, "three_body": 21, "both": 17, "both_cumulative": 11}
    print("iterations to sum |g^ - g| < 0.01 (GPU; paper):",
          {k: (v["first_converged"], paper[k]) for k, v in res.items()})
