"""Gradients of a CSPH plate impact through the hand-written adjoint
(sph_step_adjoint behind torch.autograd): loss = mean impact-axis velocity of
the target's rear face after the last step; parameters = impact speed v and
the stiffened-gas c0 and gamma.  Checked against the FP64 CPU oracle's
reverse mode and against central finite differences (eps = 1e-4 relative)
with the recorded dt schedule replayed."""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHO0, C0, GAMMA = 2700.0, 5300.0, 2.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_05128_gb300 import build
    build.build()


def _geometry(proj, target):
    prob = synth.plate_impact(proj, target, a=1e-4, v=1000.0, rho0=RHO0, c0=C0, gamma=GAMMA, units=0)
    A = prob.arrays
    dev = "cuda"
    pos = torch.tensor(np.stack([A["x"], A["y"], A["z"]], axis=1), dtype=torch.float64, device=dev)
    proj_mask = torch.tensor(A["vz"] < 0.0, device=dev)
    rear = torch.tensor(A["z"] < 0.5e-4, device=dev)
    m = torch.tensor(A["m"], dtype=torch.float64, device=dev)
    return prob, pos, proj_mask, rear, m


def _loss_and_grads(proj, target, n_steps, every, precision, v0=1000.0, reverse="fp64"):
    from paper_1805_05128_gb300.adjoint import RunSpec, csph_run
    prob, pos, proj_mask, rear, m = _geometry(proj, target)
    v = torch.tensor(v0, dtype=torch.float64, device="cuda", requires_grad=True)
    c0 = torch.tensor(C0, dtype=torch.float64, device="cuda", requires_grad=True)
    g = torch.tensor(GAMMA, dtype=torch.float64, device="cuda", requires_grad=True)
    n = pos.shape[0]
    vel = torch.zeros(n, 3, dtype=torch.float64, device="cuda")
    vel = vel + torch.stack([torch.zeros_like(m), torch.zeros_like(m), -v * proj_mask.double()], dim=1)
    rho = torch.full((n,), RHO0, dtype=torch.float64, device="cuda")
    E = c0 * c0 / (g - 1.0) + 0.5 * vel[:, 2] ** 2          # P = 0 at rho0 for the stiffened gas
    spec = RunSpec(m=m, n_steps=n_steps, every=every, precision=precision, rho0=RHO0, reverse=reverse)
    p1, v1, r1, E1 = csph_run(pos, vel, rho, E, c0, g, spec)
    loss = v1[rear, 2].mean()
    loss.backward()
    grads = np.array([v.grad.item(), c0.grad.item(), g.grad.item()])
    return loss.item(), grads, spec.record["dts"], (prob, pos, proj_mask, rear, m)


def _replay_loss(geo, dts, precision, v0, c0, g):
    from paper_1805_05128_gb300 import Simulation
    prob, pos, proj_mask, rear, m = geo
    q = synth.plate_impact(prob.meta["proj"], prob.meta["target"], a=1e-4, v=v0, rho0=RHO0, c0=c0, gamma=g,
                           units=0)
    sim = Simulation(q, precision=precision, units=0)
    sim.step_dt(dts.reshape(-1, 1))
    return sim.t["vz"][rear].mean().item()


def test_adjoint_matches_oracle_gradient():
    """FP64 forward + FP64 adjoint on the GPU vs the oracle's reverse mode."""
    L, grads, dts, geo = _loss_and_grads(4, (10, 10, 4), 20, 5, "fp64")
    prob = geo[0]
    p, s0 = O.from_problem(prob)
    s = s0.copy()
    _, odts = O.step(p, s, 20)
    assert np.allclose(dts.cpu().numpy(), odts, rtol=1e-12)
    rear = prob.arrays["z"] < 0.5e-4
    assert L == pytest.approx(float(np.mean(s.vz[rear])), rel=1e-10)
    yf = O.zero_adjoint(s0.n)
    yf["v"][rear, 2] = 1.0 / rear.sum()
    g0, bpar = O.trajectory_vjp(p, s0, odts, yf)
    proj = prob.arrays["vz"] < 0.0
    e0 = C0 * C0 / (GAMMA - 1.0)
    ref = np.array([np.sum(-g0["v"][proj, 2]) + np.sum(g0["E"][proj] * 1000.0),
                    bpar[0] + np.sum(g0["E"]) * 2.0 * C0 / (GAMMA - 1.0),
                    bpar[1] + np.sum(g0["E"]) * (-e0 / (GAMMA - 1.0))])
    assert np.allclose(grads, ref, rtol=1e-8, atol=0), (grads, ref)


@pytest.mark.parametrize("proj,target,n_steps,every", [(4, (10, 10, 4), 20, 5), (25, (120, 120, 13), 100, 10)])
def test_adjoint_matches_central_differences(proj, target, n_steps, every):
    """eps = 1e-4 relative, dt schedule of the base run replayed; the second
    case is the 200k-particle, 100-step run with checkpoints every 10 steps."""
    L, grads, dts, geo = _loss_and_grads(proj, target, n_steps, every, "fp64")
    base = dict(v0=1000.0, c0=C0, g=GAMMA)
    for k, name in enumerate(("v0", "c0", "g")):
        h = 1e-4 * base[name]
        kp, km = dict(base), dict(base)
        kp[name] += h
        km[name] -= h
        fd = (_replay_loss(geo, dts, "fp64", **kp) - _replay_loss(geo, dts, "fp64", **km)) / (2 * h)
        assert grads[k] == pytest.approx(fd, rel=1e-5), (name, grads[k], fd)


@pytest.mark.parametrize("reverse,tol", [("fp64", 1e-4), ("fp32", 1e-3)])
def test_mixed_forward_gradient_close_to_fp64(reverse, tol):
    """FP32 pair fluxes in the forward replay; pair derivatives in FP64 (FP64
    adjoint accumulation) or in FP32 with Kahan sums."""
    _, g64, _, _ = _loss_and_grads(4, (10, 10, 4), 20, 5, "fp64")
    _, g32, _, _ = _loss_and_grads(4, (10, 10, 4), 20, 5, "mixed", reverse=reverse)
    assert np.allclose(g32, g64, rtol=tol), (g32, g64)
