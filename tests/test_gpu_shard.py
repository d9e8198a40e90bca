"""The decomposed run's library backend (shard.LibBackend: sph_cfl_dt,
sph_hold_rates + sph_step_dt, sph_pair_list, voronoi_assign_static,
voronoi_balance_stats) on the GPU, driven by the same host logic as the
gloo test on one rank, against the oracle backend of that test (FP64 path:
1e-10 per field after the steps, rebalancing included)."""
import numpy as np
import pytest

from test_shard_gloo import OracleBackend, _problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_05128_gb300 import build
    build.build()


def _decomposed(backend, steps):
    import synth
    from paper_1805_05128_gb300 import shard
    prob = _problem()
    cfg = shard.Config(dim=3, K=prob.units, gdim=2, n_upd=3, kh=0.5 * prob.kappa * prob.eta)
    run = shard.Decomposed(cfg, dict(prob.arrays), synth.problem_generators(prob), backend, None)
    run.step(steps)
    return run


def test_library_backend_matches_oracle_backend():
    import oracle as O
    from paper_1805_05128_gb300 import shard
    prob = _problem()
    p, _ = O.from_problem(prob)
    ref = _decomposed(OracleBackend(p, 3), 5)
    gpu = _decomposed(shard.LibBackend(prob, precision="fp64"), 5)
    a, b = gpu.gather(), ref.gather()
    assert np.array_equal(a["id"], b["id"])
    assert gpu.time == pytest.approx(ref.time, rel=1e-12)
    np.testing.assert_allclose(gpu.gen, ref.gen, rtol=0, atol=1e-10 * np.max(np.abs(ref.gen)))
    for k in ("x", "y", "z", "vx", "vy", "vz", "rho", "E"):
        assert np.max(np.abs(a[k] - b[k])) <= 1e-10 * np.max(np.abs(b[k])), k
