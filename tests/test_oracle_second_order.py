"""Pins of the oracle's order-2 variant (states reconstructed to the pair
midpoint with minmod-limited SPH gradients; a reading, the paper's scheme is
order 1):

  * Sod tube at 400 particles: L1 density error <= 2e-2 against the exact
    Riemann solution, and below the order-1 error;
  * the SPH gradient of a linear field equals M b, M = sum_j V_j (-W'_ij)
    e^R_ij (x_j - x_i)^T the discrete first moment of the kernel (within 2-3 %
    of the identity on these lattices), for P and every velocity component,
    in 1D and 3D;
  * a uniform compression (linear velocity, uniform P): the discrete
    isentropic identity de_i = (P_i / rho_i^2) drho_i, which the order-1 P*
    violates by the acoustic dissipation Z (v_j^R - v_i^R) / 2, holds in
    order 2 up to a small fraction of that dissipation;
  * conservation: mass exact, momentum and energy to rounding;
  * the Sod density stays near its data range (limited reconstruction);
  * the reverse mode refuses order 2.
"""
import numpy as np
import pytest

import oracle as O
import sod_exact
import synth


def _sod(order):
    prob = synth.sod_1d()
    p, s = O.from_problem(prob, order=order)
    t, _ = O.step(p, s, prob.n_steps)
    win = (s.x >= 0) & (s.x <= 1)
    ex, _, _, _ = sod_exact.sample(s.x[win], t, 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    return float(np.mean(np.abs(s.rho[win] - ex))), s


def test_sod_l1_order2_within_bound_and_below_order1():
    l2, _ = _sod(2)
    l1, _ = _sod(1)
    assert l2 <= 2e-2, l2
    assert l2 < 0.6 * l1, (l2, l1)


def test_sod_order2_density_stays_near_the_data_range():
    """Density is not reconstructed (it follows the continuity equation), so
    the limiter bounds it only loosely: within [0.99 * 0.125, 1.05] in the
    window (order 1 reaches 1.012, order 2 1.041; an unlimited or wrong-signed
    reconstruction oscillates far beyond)."""
    _, s = _sod(2)
    win = (s.x >= 0) & (s.x <= 1)
    assert s.rho[win].min() >= 0.99 * 0.125 and s.rho[win].max() <= 1.05


def _lattice_1d(n=200, dx=0.01, eta=1.5):
    x = np.arange(n) * dx
    arrays = dict(x=x, vx=np.zeros(n), rho=np.ones(n), E=np.full(n, 2.5), m=np.full(n, dx))
    p = O.Params(dim=1, eta=eta, cfl=0.3, materials=[O.Material(O.EOS_IDEAL, 1.4)], order=2)
    return p, O.State(1, arrays)


def _moment(p, s, X):
    """M_i = sum_j V_j (-W'_ij) e_ij (x_j - x_i)^T over the pair list."""
    pi, pj = O.pairs(p, s)
    n, D = X.shape
    M = np.zeros((n, D, D))
    for i, j in zip(pi, pj):
        d = X[j] - X[i]
        r = np.linalg.norm(d)
        h = p.eta * 0.5 * (s.d[i] + s.d[j])
        w = -O.kernel_dw(p.kernel, p.dim, p.kappa, r, h)
        e = d / r
        M[i] += s.m[j] / s.rho[j] * w * np.outer(e, d)
        M[j] += s.m[i] / s.rho[i] * w * np.outer(-e, -d)
    return M


def test_gradient_of_linear_field_1d():
    p, s = _lattice_1d()
    O.derive(p, s)
    s.P[:] = 3.0 + 7.0 * s.x          # linear pressure
    s.vx[:] = -2.0 + 5.0 * s.x        # linear velocity
    gP, gV = O.pair_gradients(p, s)
    M = _moment(p, s, s.x[:, None])[:, 0, 0]
    inner = slice(10, -10)
    assert np.allclose(gP[inner, 0], 7.0 * M[inner], rtol=1e-12)
    assert np.allclose(gV[inner, 0, 0], 5.0 * M[inner], rtol=1e-12)
    assert np.allclose(M[inner], 1.0, atol=2e-2)      # the kernel's first moment on this lattice


def test_gradient_of_linear_field_3d():
    side, a = 10, 1e-3
    g = np.meshgrid(*[np.arange(side, dtype=float)] * 3, indexing="ij")
    x, y, z = (gi.ravel() * a for gi in g)
    n = side ** 3
    u = synth.uniform(11, 3 * n).reshape(3, n)
    x, y, z = x + 0.05 * a * (u[0] - 0.5), y + 0.05 * a * (u[1] - 0.5), z + 0.05 * a * (u[2] - 0.5)
    arrays = dict(x=x, y=y, z=z, vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n), rho=np.full(n, 1000.0),
                  E=np.full(n, 1e5), m=np.full(n, 1000.0 * a ** 3))
    p = O.Params(dim=3, eta=1.3, cfl=0.3, materials=[O.Material(O.EOS_IDEAL, 1.4)], order=2)
    s = O.State(3, arrays)
    O.derive(p, s)
    bP = np.array([1.0, -2.0, 3.0])
    A = np.array([[0.5, 1.0, 0.0], [-1.0, 2.0, 0.25], [0.0, 0.0, -3.0]])
    X = np.stack([x, y, z], axis=1)
    s.P[:] = X @ bP
    V = X @ A.T
    s.vx[:], s.vy[:], s.vz[:] = V[:, 0], V[:, 1], V[:, 2]
    gP, gV = O.pair_gradients(p, s)
    M = _moment(p, s, X)
    assert np.allclose(gP, np.einsum("iab,b->ia", M, bP), rtol=1e-10, atol=1e-12)
    assert np.allclose(gV, np.einsum("ibc,ac->iab", M, A), rtol=1e-10, atol=1e-12)
    inner = np.all((X > 2.7 * a) & (X < (side - 3.7) * a), axis=1)
    assert inner.sum() > 20
    assert np.allclose(M[inner], np.eye(3), atol=3e-2)     # jittered lattice: within 3 %


def test_linear_compression_nearly_isentropic_in_order2():
    """Uniform rho, P; v = -alpha x.  de_i - (P_i/rho_i^2) drho_i vanishes when
    P* = P on every pair; order 1 makes it the positive acoustic dissipation."""
    excess = {}
    for order in (1, 2):
        p, s = _lattice_1d(eta=1.5)
        alpha = 3.0
        s.vx[:] = -alpha * (s.x - s.x.mean())
        s.E[:] = 2.5 + 0.5 * s.vx ** 2
        p.order = order
        O.eval_rates(p, s)
        de = s.dE - s.vx * s.ax
        excess[order] = (de - s.P / s.rho ** 2 * s.drho)[20:-20]
    scale = np.abs(excess[1]).max()
    assert np.all(excess[1] > 0.1 * scale)                 # order 1: dissipative everywhere inside
    assert np.abs(excess[2]).max() <= 0.05 * scale, (np.abs(excess[2]).max(), scale)


def test_conservation_order2():
    prob = synth.plate_impact(5, (12, 12, 4), a=1e-4, v=1000.0, units=0, seed=3, jitter=0.05)
    p, s = O.from_problem(prob, order=2)
    c0 = np.zeros(5)
    O.eval_rates(p, s)
    c0 = O.conservation(s)
    O.step(p, s, 20, rates_valid=True)
    c1 = O.conservation(s)
    mscale = np.sum(s.m * np.sqrt(s.vx ** 2 + s.vy ** 2 + s.vz ** 2))
    assert c1[0] == pytest.approx(c0[0], rel=1e-15)
    for a in (1, 2, 3):
        assert abs(c1[a] - c0[a]) <= 1e-12 * mscale
    assert abs(c1[4] - c0[4]) <= 1e-12 * abs(c0[4])


def test_reverse_mode_refuses_order2():
    prob = synth.plate_impact(4, (8, 8, 3), a=1e-4, v=1000.0, units=0)
    p, s = O.from_problem(prob, order=2)
    O.eval_rates(p, s)
    pi, pj = O.pairs(p, s)
    z = np.zeros((s.n, 3))
    with pytest.raises(ValueError):
        O.rates_vjp(p, s, pi, pj, z, np.zeros(s.n), np.zeros(s.n))
