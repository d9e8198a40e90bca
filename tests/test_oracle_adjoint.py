"""Pins of the oracle's hand-derived reverse mode: the vector-Jacobian
products of the CSPH rates and of one KDK step, and the gradient of a whole
run with respect to the impact velocity and the stiffened-gas (c0, gamma),
all against central finite differences (dt schedule replayed, pair set of the
unperturbed run for the rate and step checks)."""
import numpy as np
import pytest

import oracle as O
import synth

RHO0, C0, GAMMA = 2700.0, 5300.0, 2.0


def _params(c0=C0, gamma=GAMMA, dim=3):
    mat = O.Material(O.EOS_STIFFENED, gamma, RHO0, c0, RHO0 * c0 * c0 / gamma)
    return O.Params(dim=dim, eta=1.3, cfl=0.3, materials=[mat])


def _state(seed=5, side=5, a=1e-4):
    g = np.meshgrid(*[np.arange(side, dtype=float)] * 3, indexing="ij")
    n = side ** 3
    u = synth.uniform(seed, 10 * n).reshape(10, n)
    x = g[0].ravel() * a + 0.1 * a * (u[0] - 0.5)
    y = g[1].ravel() * a + 0.1 * a * (u[1] - 0.5)
    z = g[2].ravel() * a + 0.1 * a * (u[2] - 0.5)
    v = 100.0 * (u[3:6] - 0.5)
    rho = RHO0 * (1.0 + 0.02 * (u[6] - 0.5))
    e0 = C0 * C0 / (GAMMA - 1.0)
    E = e0 * (1.0 + 0.02 * (u[7] - 0.5)) + 0.5 * (v ** 2).sum(axis=0)
    return O.State(3, dict(x=x, y=y, z=z, vx=v[0], vy=v[1], vz=v[2], rho=rho, E=E, m=np.full(n, RHO0 * a ** 3)))


def _L_rates(p, s, pi, pj, ga, gr, gE):
    t = s.copy()
    O.derive(p, t)
    O.rates(p, t, pi, pj)
    _, _, acc = O.state_vectors(t)
    return float(np.sum(ga * acc) + np.sum(gr * t.drho) + np.sum(gE * t.dE))


def _perturbed(s, dvec, eps):
    t = s.copy()
    for a, k in enumerate(("x", "y", "z")):
        getattr(t, k)[:] += eps * dvec["x"][:, a]
    for a, k in enumerate(("vx", "vy", "vz")):
        getattr(t, k)[:] += eps * dvec["v"][:, a]
    t.rho[:] += eps * dvec["rho"]
    t.E[:] += eps * dvec["E"]
    return t


def test_rates_vjp_matches_central_differences():
    p = _params()
    s = _state()
    O.eval_rates(p, s)
    n = s.n
    pi, pj = O.pairs(p, s)
    rng = np.random.default_rng(2)
    _, _, acc = O.state_vectors(s)
    ga = rng.normal(size=(n, 3)) / np.abs(acc).max()
    gr = rng.normal(size=n) / np.abs(s.drho).max()
    gE = rng.normal(size=n) / np.abs(s.dE).max()
    O.derive(p, s)
    g = O.rates_vjp(p, s, pi, pj, ga, gr, gE)
    dvec = dict(x=1e-6 * rng.normal(size=(n, 3)), v=rng.normal(size=(n, 3)),
                rho=RHO0 * 1e-3 * rng.normal(size=n), E=1e4 * rng.normal(size=n))
    for part in ("x", "v", "rho", "E"):
        d = {k: (dvec[k] if k == part else np.zeros_like(dvec[k])) for k in dvec}
        eps = 1e-3
        fd = (_L_rates(p, _perturbed(s, d, eps), pi, pj, ga, gr, gE)
              - _L_rates(p, _perturbed(s, d, -eps), pi, pj, ga, gr, gE)) / (2 * eps)
        an = float(np.sum(g[{"x": "bx", "v": "bv", "rho": "brho", "E": "bE"}[part]] * d[part]))
        assert an == pytest.approx(fd, rel=1e-6), part
    # parameters: c0 and gamma enter through P_inf = rho0 c0^2 / gamma and the EOS
    for k, (c0p, gp, h) in enumerate([(C0 * (1 + 1e-6), GAMMA, C0 * 1e-6), (C0, GAMMA * (1 + 1e-6), GAMMA * 1e-6)]):
        c0m, gm = (C0 - h, GAMMA) if k == 0 else (C0, GAMMA - h)
        fd = (_L_rates(_params(c0p, gp), s, pi, pj, ga, gr, gE)
              - _L_rates(_params(c0m, gm), s, pi, pj, ga, gr, gE)) / (2 * h)
        assert g["bpar"][k] == pytest.approx(fd, rel=1e-6), k


def _state_after_step(p, s, dt):
    t = s.copy()
    O.step_replay(p, t, [dt], rates_valid=True)
    pos, vel, acc = O.state_vectors(t)
    return dict(x=pos, v=vel, rho=t.rho, E=t.E, a=acc, drho=t.drho, dE=t.dE)


def test_step_vjp_matches_central_differences():
    p = _params()
    s = _state(seed=9)
    O.eval_rates(p, s)
    dt = 5e-9
    n = s.n
    rng = np.random.default_rng(4)
    out0 = _state_after_step(p, s, dt)
    w = {k: rng.normal(size=np.shape(v)) / max(np.abs(v).max(), 1e-300) for k, v in out0.items()}
    L = lambda o: sum(float(np.sum(w[k] * o[k])) for k in w)
    y = {k: w[k].copy() for k in w}
    bpar = np.zeros(2)
    O.step_vjp(p, s, dt, y, bpar)
    dvec = dict(x=1e-6 * rng.normal(size=(n, 3)), v=rng.normal(size=(n, 3)),
                rho=RHO0 * 1e-3 * rng.normal(size=n), E=1e4 * rng.normal(size=n))
    for part in ("x", "v", "rho", "E"):
        d = {k: (dvec[k] if k == part else np.zeros_like(dvec[k])) for k in dvec}
        eps = 1e-3
        fd = (L(_state_after_step(p, _perturbed(s, d, eps), dt))
              - L(_state_after_step(p, _perturbed(s, d, -eps), dt))) / (2 * eps)
        assert float(np.sum(y[part] * d[part])) == pytest.approx(fd, rel=1e-5), part
    # the held rates a, drho, dE of the state before the step
    da = np.abs(O.state_vectors(s)[2]).max() * rng.normal(size=(n, 3))

    def with_rates(eps):
        t = s.copy()
        for a_, k in enumerate(("ax", "ay", "az")):
            getattr(t, k)[:] += eps * da[:, a_]
        return t
    eps = 1e-3
    fd = (L(_state_after_step(p, with_rates(eps), dt)) - L(_state_after_step(p, with_rates(-eps), dt))) / (2 * eps)
    assert float(np.sum(y["a"] * da)) == pytest.approx(fd, rel=1e-5)


# ------------------------------------------------------------ whole run ---
def _plate(v, c0, gamma):
    prob = synth.plate_impact(4, (10, 10, 4), a=1e-4, v=v, rho0=RHO0, c0=c0, gamma=gamma, units=0)
    return prob


def _rear(prob):
    return prob.arrays["z"] < 0.5 * prob.meta["a"]        # target layer farthest from the impact


def _run(v, c0, gamma, dts=None, steps=20):
    prob = _plate(v, c0, gamma)
    p, s = O.from_problem(prob)
    if dts is None:
        _, dts = O.step(p, s, steps)
    else:
        O.eval_rates(p, s)
        O.step_replay(p, s, dts, rates_valid=True)
    return float(np.mean(s.vz[_rear(prob)])), dts, prob


def test_trajectory_gradient_matches_central_differences():
    """d(mean v_z of the rear face after 20 steps)/d(impact speed, c0, gamma):
    the oracle's reverse mode against central differences at eps = 1e-4
    relative with the recorded dt schedule replayed."""
    v0 = 1000.0
    L0, dts, prob = _run(v0, C0, GAMMA)
    p, s0 = O.from_problem(prob)
    n = s0.n
    yf = O.zero_adjoint(n)
    rear = _rear(prob)
    yf["v"][rear, 2] = 1.0 / rear.sum()
    g0, bpar = O.trajectory_vjp(p, s0, dts, yf)
    proj = prob.arrays["vz"] < 0.0
    e0 = C0 * C0 / (GAMMA - 1.0)
    grad = {
        # v_z0 = -v on the projector, E0 = e0 + v^2/2 there
        "v": float(np.sum(-g0["v"][proj, 2]) + np.sum(g0["E"][proj] * v0)),
        # e0 = c0^2 / (gamma - 1) everywhere (P = 0 at rho0)
        "c0": float(bpar[0] + np.sum(g0["E"]) * 2.0 * C0 / (GAMMA - 1.0)),
        "gamma": float(bpar[1] + np.sum(g0["E"]) * (-e0 / (GAMMA - 1.0))),
    }
    for name, base in (("v", v0), ("c0", C0), ("gamma", GAMMA)):
        h = 1e-4 * base
        kw_p = dict(v=v0, c0=C0, gamma=GAMMA)
        kw_m = dict(kw_p)
        kw_p[name] = base + h
        kw_m[name] = base - h
        fd = (_run(kw_p["v"], kw_p["c0"], kw_p["gamma"], dts)[0]
              - _run(kw_m["v"], kw_m["c0"], kw_m["gamma"], dts)[0]) / (2 * h)
        assert grad[name] == pytest.approx(fd, rel=1e-5, abs=1e-9 * abs(L0) / base), (name, grad[name], fd)
