"""Pins of the Mie-Grueneisen closure in motion (Sec. 7 lead: rho0 = 11.35
g/cc, c_a = 2.58 km/s, s_a = 1.26, Gamma = 1.7): a 1D lead column driven at
u_p = 1 km/s onto a rigid wall (the symmetry plane of a mirror copy) carries
a steady shock whose state follows the Rankine-Hugoniot relations of the
linear u_s - u_p fit: u_s = c_a + s_a u_p, P = rho0 u_s u_p,
rho = rho0 u_s / (u_s - u_p), and the shock front moves at u_s - u_p from
the wall."""
import numpy as np
import pytest

import oracle as O
import synth


def _column(n=300, a=1e-6, up=1000.0):
    mat = synth.lead()
    x = np.arange(n) * a
    x = np.concatenate([x, -x - a])
    vx = np.concatenate([np.full(n, -up), np.full(n, up)])
    arrays = dict(x=x, vx=vx, rho=np.full(2 * n, mat.rho0), E=0.5 * vx * vx, m=np.full(2 * n, mat.rho0 * a))
    p = O.Params(dim=1, eta=1.5, cfl=0.3, materials=[O.Material(O.EOS_MIE_GRUNEISEN, mat.gamma, mat.rho0, mat.c0,
                                                                0.0, mat.s_a)])
    return p, O.State(1, arrays), mat


@pytest.mark.parametrize("order", [1, 2])
def test_lead_piston_shock_follows_the_hugoniot(order):
    up = 1000.0
    p, s, mat = _column(up=up)
    p.order = order
    t, _ = O.step(p, s, 400)
    us = mat.c0 + mat.s_a * up
    P_h = mat.rho0 * us * up
    rho_h = mat.rho0 * us / (us - up)
    front = (us - up) * t                          # shock position from the wall
    right = s.x > 0
    x, P, rho, v = s.x[right], s.P[right], s.rho[right], s.vx[right]
    plateau = (x > 0.25 * front) & (x < 0.75 * front)
    assert plateau.sum() >= 20
    assert np.median(P[plateau]) == pytest.approx(P_h, rel=0.03)
    assert np.median(rho[plateau]) == pytest.approx(rho_h, rel=0.01)
    assert np.max(np.abs(v[plateau])) <= 0.05 * up               # the shocked lead is at rest
    ahead = (x > 1.3 * front) & (x < x.max() - 20e-6)
    assert np.allclose(v[ahead], -up, rtol=1e-3) and np.allclose(rho[ahead], mat.rho0, rtol=1e-3)
    # front position: where the density crosses the midpoint between the states
    mid = 0.5 * (rho_h + mat.rho0)
    xf = x[np.argmin(np.abs(np.where(x < 2 * front, rho, 0.0) - mid))]
    assert xf == pytest.approx(front, rel=0.1)


def test_ejecta_geometry_and_mirror_symmetry():
    q = synth.ejecta(nx=16, periods=2, lam=8, nz=3, units=0)
    x, y = q.arrays["x"], q.arrays["y"]
    n1 = q.meta["n_half"]
    assert q.n == 2 * n1
    assert np.allclose(x[n1:], -x[:n1] - q.meta["a"])
    # the V-grooves remove lam/2 spacings at their centres and nothing at the ridges
    a, lam, nx = q.meta["a"], q.meta["lam"], q.meta["nx"]
    top = {}
    for xi, yi in zip(x[:n1], y[:n1]):
        top[round(yi / a, 3)] = max(top.get(round(yi / a, 3), -1), round(xi / a))
    depths = sorted(nx - 1 - v for v in top.values())
    assert depths[0] == 0 and depths[-1] == lam // 2 - 1
    p, s = O.from_problem(q)
    O.step(p, s, 10)
    # the symmetric impact keeps the mirror symmetry of the state (the wall is at rest)
    assert np.allclose(s.x[n1:], -s.x[:n1] - a, rtol=0, atol=1e-9 * a)
    assert np.allclose(s.vx[n1:], -s.vx[:n1], rtol=0, atol=1e-9 * 1000.0)
    assert np.allclose(s.rho[n1:], s.rho[:n1], rtol=1e-12)
