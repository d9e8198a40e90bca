"""Pins of the oracle's HLL pair solver (the alternative to the acoustic
solver; Sec. 4.1 names no solver form, the reading is the two-wave HLL state
of the linearised Lagrangian problem with Davis wave speeds +-max(Z_i, Z_j)):

  * against the general HLL flux formula (Harten, Lax and van Leer) written
    out for a linear system U_t + F(U)_m = 0, U = (v, P), F = (P, C^2 v),
    with arbitrary states: P* is its first flux component, C^2 v* its second;
  * equal impedances give the acoustic solution;
  * exchange symmetry (left/right swap with e^R reversed);
  * entropy: with converging velocities and mismatched impedances the HLL
    pressure exceeds the acoustic one (more dissipation);
  * the Sod tube with HLL pairs: order 2 within the L1 bound of 2e-2, order 1
    no worse than the acoustic solver; both conserve;
  * the reverse mode refuses it.
"""
import numpy as np
import pytest

import oracle as O
import sod_exact
import synth


def _hll_flux(UL, UR, FL, FR, SL, SR):
    """Textbook HLL numerical flux for wave-speed bounds SL < 0 < SR."""
    return (SR * FL - SL * FR + SL * SR * (UR - UL)) / (SR - SL)


@pytest.mark.parametrize("seed", range(4))
def test_hll_matches_general_hll_flux(seed):
    rng = np.random.default_rng(seed)
    for _ in range(40):
        Pi, Pj = rng.uniform(-2.0, 5.0, 2)
        Zi, Zj = rng.uniform(0.05, 7.0, 2)
        vi, vj = rng.normal(size=2) * 3
        C = max(Zi, Zj)
        UL, UR = np.array([vi, Pi]), np.array([vj, Pj])
        FL, FR = np.array([Pi, C * C * vi]), np.array([Pj, C * C * vj])
        F = _hll_flux(UL, UR, FL, FR, -C, C)
        P, v = O.riemann_hll(Pi, Pj, Zi, Zj, vi, vj)
        assert P == pytest.approx(F[0], rel=1e-12, abs=1e-12)
        assert v == pytest.approx(F[1] / (C * C), rel=1e-12, abs=1e-12)


def test_hll_equals_acoustic_for_equal_impedance():
    rng = np.random.default_rng(9)
    for _ in range(50):
        Pi, Pj, Z = rng.uniform(0.1, 5.0, 3)
        vi, vj = rng.normal(size=2)
        a = O.riemann_acoustic(Pi, Pj, Z, Z, vi, vj)
        b = O.riemann_hll(Pi, Pj, Z, Z, vi, vj)
        assert b[0] == pytest.approx(a[0], rel=1e-14) and b[1] == pytest.approx(a[1], rel=1e-13, abs=1e-15)


def test_hll_exchange_symmetry_and_uniform_state():
    P, v = O.riemann_hll(2.0, 2.0, 1.0, 4.0, 0.7, 0.7)
    assert P == 2.0 and v == pytest.approx(0.7, rel=1e-15)
    rng = np.random.default_rng(4)
    for _ in range(50):
        Pi, Pj, Zi, Zj = rng.uniform(0.1, 5.0, 4)
        vi, vj = rng.normal(size=2)
        Pa, va = O.riemann_hll(Pi, Pj, Zi, Zj, vi, vj)
        Pb, vb = O.riemann_hll(Pj, Pi, Zj, Zi, -vj, -vi)
        assert Pa == pytest.approx(Pb, rel=1e-14) and va == pytest.approx(-vb, rel=1e-13, abs=1e-15)


def test_hll_more_dissipative_than_acoustic_for_mismatched_impedance():
    """Equal pressures, converging velocities (v_i^R > v_j^R): the acoustic P*
    rises by Z_i Z_j / (Z_i + Z_j) dv, the HLL P* by max(Z) dv / 2, which is
    larger whenever Z_i != Z_j."""
    for Zi, Zj in ((1.0, 3.0), (5.0, 0.5), (2.0, 2.5)):
        dv = 0.3
        Pa, _ = O.riemann_acoustic(1.0, 1.0, Zi, Zj, dv, 0.0)
        Ph, _ = O.riemann_hll(1.0, 1.0, Zi, Zj, dv, 0.0)
        assert Pa - 1.0 == pytest.approx(Zi * Zj / (Zi + Zj) * dv, rel=1e-14)
        assert Ph - 1.0 == pytest.approx(max(Zi, Zj) * dv / 2, rel=1e-14)
        assert Ph > Pa


def _sod(solver, order):
    prob = synth.sod_1d()
    p, s = O.from_problem(prob, solver=solver, order=order)
    c0 = O.conservation(s)
    t, _ = O.step(p, s, prob.n_steps)
    win = (s.x >= 0) & (s.x <= 1)
    ex, _, _, _ = sod_exact.sample(s.x[win], t, 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    return float(np.mean(np.abs(s.rho[win] - ex))), c0, O.conservation(s)


@pytest.mark.parametrize("order", [1, 2])
def test_sod_with_hll_within_bound_and_conservative(order):
    l1, c0, c1 = _sod(O.SOLVER_HLL, order)
    l1a, _, _ = _sod(O.SOLVER_ACOUSTIC, order)
    if order == 2:
        assert l1 <= 2e-2, l1
    else:
        assert l1 <= l1a, (l1, l1a)           # the extra dissipation damps the contact ringing
    assert l1 != l1a                        # the solver choice reaches the rates
    assert c1[0] == pytest.approx(c0[0], rel=1e-15)
    assert abs(c1[1] - c0[1]) <= 1e-13 * np.sum(np.abs(c0[1:2])) + 1e-13
    assert c1[4] == pytest.approx(c0[4], rel=1e-12)


def test_hll_rates_equal_acoustic_at_uniform_impedance():
    """Uniform density and pressure (so uniform Z) with a velocity field: the
    two solvers give the same rates to rounding."""
    prob = synth.sod_1d()
    n = prob.n
    A = prob.arrays
    A["rho"] = np.ones(n)                    # uniform state, velocity field only
    A["vx"] = 0.1 * np.sin(7.0 * A["x"])
    A["E"] = 2.5 + 0.5 * A["vx"] ** 2
    A["m"] = np.full(n, A["m"].mean())
    out = {}
    for solver in (O.SOLVER_ACOUSTIC, O.SOLVER_HLL):
        p, s = O.from_problem(prob, solver=solver)
        O.eval_rates(p, s)
        out[solver] = (s.drho.copy(), s.ax.copy(), s.dE.copy())
    for a, b in zip(out[0], out[1]):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())


def test_reverse_mode_refuses_hll():
    prob = synth.plate_impact(4, (8, 8, 3), a=1e-4, v=1000.0, units=0)
    p, s = O.from_problem(prob, solver=O.SOLVER_HLL)
    O.eval_rates(p, s)
    pi, pj = O.pairs(p, s)
    z = np.zeros((s.n, 3))
    with pytest.raises(ValueError):
        O.rates_vjp(p, s, pi, pj, z, np.zeros(s.n), np.zeros(s.n))
