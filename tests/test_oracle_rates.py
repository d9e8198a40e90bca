"""Pins of the oracle's CSPH rates, eqs. (SPH:Conti), (SPH:Pulse),
(SPH:Energy): signs on a two-particle collision, exact pairwise conservation,
Galilean invariance, and consistency with the continuum equations on a
lattice (-rho div v, -grad P / rho, and the first law de = P/rho^2 drho)."""
import numpy as np
import pytest

import oracle as O
import synth


def _lattice_state(n_side, a=1.0, jitter=0.0, seed=1):
    g = np.meshgrid(*[np.arange(n_side, dtype=float) * a] * 3, indexing="ij")
    x, y, z = [v.ravel() for v in g]
    if jitter:
        u = synth.uniform(seed, 3 * len(x))
        x = x + jitter * a * (2 * u[0::3] - 1)
        y = y + jitter * a * (2 * u[1::3] - 1)
        z = z + jitter * a * (2 * u[2::3] - 1)
    n = len(x)
    return dict(x=x, y=y, z=z, vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n),
                rho=np.ones(n), E=np.full(n, 2.5), m=np.full(n, a ** 3))


IDEAL = O.Params(dim=3, eta=1.3, materials=[O.Material(O.EOS_IDEAL, 1.4)])


def _rates(arrays, p=IDEAL):
    s = O.State(3, arrays)
    O.eval_rates(p, s)
    return s


def test_two_particles_collision_signs():
    arr = dict(x=np.array([0.0, 1.0]), y=np.zeros(2), z=np.zeros(2),
               vx=np.array([0.3, -0.1]), vy=np.zeros(2), vz=np.zeros(2),
               rho=np.ones(2), E=np.array([2.5 + 0.045, 2.5 + 0.005]), m=np.ones(2))
    s = _rates(arr)
    assert s.drho[0] > 0 and s.drho[1] > 0           # approaching: both compress
    assert s.ax[0] < 0 and s.ax[1] > 0               # repulsion along the line of centres
    assert s.ay[0] == 0 and s.az[1] == 0
    assert s.m[0] * s.ax[0] + s.m[1] * s.ax[1] == pytest.approx(0.0, abs=1e-15)
    # the contact moves right (v* > 0); the left particle does work on the right one
    assert s.dE[0] < 0 and s.dE[1] > 0
    assert s.m[0] * s.dE[0] + s.m[1] * s.dE[1] == pytest.approx(0.0, abs=1e-15)


def test_pairwise_conservation_random_state():
    arr = _lattice_state(8, jitter=0.3, seed=4)
    n = len(arr["x"])
    u = synth.uniform(99, 5 * n)
    arr["vx"], arr["vy"], arr["vz"] = u[:n] - 0.5, u[n:2 * n] - 0.5, u[2 * n:3 * n] - 0.5
    arr["rho"] = 1.0 + 0.2 * (u[3 * n:4 * n] - 0.5)
    arr["m"] = arr["rho"] * 1.0
    arr["E"] = 2.5 + 0.5 * (u[4 * n:] - 0.5) + 0.5 * (arr["vx"] ** 2 + arr["vy"] ** 2 + arr["vz"] ** 2)
    s = _rates(arr)
    for comp in (s.ax, s.ay, s.az, s.dE):
        tot = np.sum(s.m * comp)
        assert abs(tot) <= 1e-14 * np.sum(np.abs(s.m * comp))


def test_galilean_invariance():
    """Adding a uniform velocity U leaves drho/dt and dv/dt unchanged and
    shifts dE/dt by U . dv/dt (E carries the kinetic energy)."""
    arr = _lattice_state(7, jitter=0.25, seed=8)
    n = len(arr["x"])
    u = synth.uniform(7, 3 * n)
    arr["vx"], arr["vy"], arr["vz"] = 0.1 * u[:n], 0.1 * u[n:2 * n], -0.1 * u[2 * n:]
    U = np.array([0.3, -0.2, 0.5])
    b = {k: v.copy() for k, v in arr.items()}
    for k, c in zip(("vx", "vy", "vz"), U):
        b[k] = b[k] + c
    ke = lambda a: 0.5 * (a["vx"] ** 2 + a["vy"] ** 2 + a["vz"] ** 2)
    b["E"] = arr["E"] - ke(arr) + ke(b)     # same internal energy
    s0, s1 = _rates(arr), _rates(b)
    scale = np.abs(s0.ax).max()
    assert np.allclose(s1.drho, s0.drho, rtol=0, atol=1e-12 * np.abs(s0.drho).max())
    for a0, a1 in ((s0.ax, s1.ax), (s0.ay, s1.ay), (s0.az, s1.az)):
        assert np.allclose(a1, a0, rtol=0, atol=1e-12 * scale)
    shift = U[0] * s0.ax + U[1] * s0.ay + U[2] * s0.az
    assert np.allclose(s1.dE, s0.dE + shift, rtol=0, atol=1e-11 * np.abs(s1.dE).max())


def _centre(n_side):
    c = n_side // 2
    return c + n_side * c + n_side * n_side * c


def test_continuity_uniform_expansion():
    """v = alpha r on a lattice: drho/dt -> -rho div v = -3 alpha rho."""
    n = 13
    arr = _lattice_state(n)
    alpha = 1e-3
    arr["vx"], arr["vy"], arr["vz"] = alpha * arr["x"], alpha * arr["y"], alpha * arr["z"]
    arr["E"] = 2.5 + 0.5 * (arr["vx"] ** 2 + arr["vy"] ** 2 + arr["vz"] ** 2)
    s = _rates(arr)
    i = _centre(n)
    assert s.drho[i] == pytest.approx(-3.0 * alpha, rel=0.03)
    # first law for this adiabatic expansion: de/dt = (P/rho^2) drho/dt, up to the
    # acoustic solver's dissipation, which is second order in alpha
    dedt = s.dE[i] - (s.vx[i] * s.ax[i] + s.vy[i] * s.ay[i] + s.vz[i] * s.az[i])
    assert dedt == pytest.approx(s.P[i] / s.rho[i] ** 2 * s.drho[i], rel=0.01)


def test_momentum_linear_pressure():
    """P = P0 + G x at rest: dv/dt -> -grad P / rho = (-G, 0, 0)."""
    n = 13
    arr = _lattice_state(n)
    G = 1e-3
    P = 1.0 + G * arr["x"]
    arr["E"] = P / (0.4 * arr["rho"])
    s = _rates(arr)
    i = _centre(n)
    assert s.ax[i] == pytest.approx(-G, rel=0.03)
    assert abs(s.ay[i]) < 1e-12 and abs(s.az[i]) < 1e-12
    # the contact velocity v* = (P_i - P_j)/(Z_i + Z_j) feeds drho/dt only through the
    # asymmetry of Z = rho c across the gradient: second order in G
    assert abs(s.drho[i]) < 10 * G * G
