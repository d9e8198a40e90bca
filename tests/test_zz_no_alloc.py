"""voronoi_assign_static: the allocation-free Voronoi assignment, for callers
that cannot allocate device memory (a host loop that must not call cudaMalloc,
code whose device memory belongs to another allocator or a fixed arena).  Its
scratch is a fixed device array in the library, so these checks call it
several times in a row and compare each result with the handle-based
voronoi_assign on the same inputs.  This file is
collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_05128_gb300 import build
    build.build()


def _reference(prob, K, gdim, gen):
    """Ownership and unit offsets from the existing entry point (voronoi_assign)."""
    from paper_1805_05128_gb300 import Simulation
    prob.units, prob.unit_dim = K, gdim
    sim = Simulation(prob, precision="fp64", units=K, generators=gen)
    offs = sim.assign()
    torch.cuda.synchronize()
    return sim, sim.t["unit"].clone(), offs.clone()


def _call_static(sim, gen_dev, K, gdim):
    from paper_1805_05128_gb300 import abi
    n = sim.n
    dev = sim.device
    unit = torch.full((n,), -7, dtype=torch.int32, device=dev)
    offs = torch.full((K + 1,), -7, dtype=torch.int32, device=dev)
    lst = torch.full((n,), -7, dtype=torch.int32, device=dev)
    ptr = lambda k: sim.t[k].data_ptr() if sim.t.get(k) is not None and "xyz".index(k) < gdim else None
    abi.voronoi_assign_static(n, ptr("x"), ptr("y"), ptr("z"), gen_dev.data_ptr(), K, gdim, unit.data_ptr(),
                              offs.data_ptr(), lst.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return unit, offs, lst


def _check(unit, offs, lst, ref_unit, ref_offs, K):
    assert torch.equal(unit, ref_unit)
    assert torch.equal(offs, ref_offs)
    u = unit.cpu().numpy()
    expect = np.argsort(u, kind="stable").astype(np.int32)   # grouped by unit, ascending inside a unit
    assert np.array_equal(lst.cpu().numpy(), expect)
    assert np.array_equal(offs.cpu().numpy(), np.concatenate([[0], np.cumsum(np.bincount(u, minlength=K))]))


def test_static_assign_matches_voronoi_assign_on_consecutive_calls():
    plate = synth.plate_impact(6, (16, 16, 5), a=1e-4, v=1000.0, units=8, seed=7, jitter=0.05)
    K, gdim = 8, 2
    plate.units, plate.unit_dim = K, gdim
    gen = synth.problem_generators(plate)
    sim, ref_unit, ref_offs = _reference(plate, K, gdim, gen)
    gen_dev = torch.as_tensor(gen, device=sim.device).contiguous()
    for _ in range(2):                                   # same inputs twice: the shared scratch is reset
        _check(*_call_static(sim, gen_dev, K, gdim), ref_unit, ref_offs, K)

    sod = synth.sod_1d()                                 # then a different size, K and dimension
    K2, g2 = 4, 1
    gen2 = synth.seed_generators([sod.arrays["x"]], K2)
    sim2, ref_unit2, ref_offs2 = _reference(sod, K2, g2, gen2)
    gen2_dev = torch.as_tensor(gen2, device=sim2.device).contiguous()
    _check(*_call_static(sim2, gen2_dev, K2, g2), ref_unit2, ref_offs2, K2)


def test_static_assign_rejects_sizes_beyond_its_scratch():
    from paper_1805_05128_gb300 import abi
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    with pytest.raises(abi.CsphError) as e:
        abi.voronoi_assign_static((1 << 22) + 1, dummy.data_ptr(), None, None, dummy.data_ptr(), 2, 1,
                                  out.data_ptr(), None, None, st)
    assert e.value.code == abi.SPH_ERR_CAPACITY
    with pytest.raises(abi.CsphError) as e:
        abi.voronoi_assign_static(4, dummy.data_ptr(), None, None, dummy.data_ptr(), 257, 1,
                                  out.data_ptr(), None, None, st)
    assert e.value.code == abi.SPH_ERR_CAPACITY
    with pytest.raises(abi.CsphError) as e:
        abi.voronoi_assign_static(4, dummy.data_ptr(), None, None, dummy.data_ptr(), 2, 2,
                                  out.data_ptr(), None, None, st)   # dim 2 without y
    assert e.value.code == abi.SPH_ERR_INVALID
