"""Pins of the oracle's closure: smoothing kernels, equations of state and
the acoustic pair Riemann solver, against quadrature, closed forms, the
Rankine-Hugoniot relations, numerical isentropes and the exact Riemann solver.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle as O
import sod_exact

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- kernels ---
@pytest.mark.parametrize("kernel,kappa", [(O.KERNEL_CUBIC, 2.0), (O.KERNEL_WENDLAND_C2, 1.936)])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_kernel_normalised(kernel, kappa, dim):
    """Integral of W over its support equals one (quadrature, independent of the closed form)."""
    h = 0.7
    surf = {1: 2.0, 2: 2.0 * math.pi, 3: 4.0 * math.pi}[dim]
    rmax = kappa * h if kernel == O.KERNEL_WENDLAND_C2 else 2.0 * h
    f = lambda r: surf * r ** (dim - 1) * O.kernel_w(kernel, dim, kappa, r, h)
    pts = [h] if kernel == O.KERNEL_CUBIC else None
    val, _ = integrate.quad(f, 0.0, rmax, points=pts, epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-12


@pytest.mark.parametrize("kernel,kappa", [(O.KERNEL_CUBIC, 2.0), (O.KERNEL_WENDLAND_C2, 1.936)])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_kernel_derivative_matches_fd(kernel, kappa, dim):
    h = 1.3
    for q in np.linspace(0.05, 1.9, 23):
        r = q * h
        if kernel == O.KERNEL_WENDLAND_C2 and r >= kappa * h:
            continue
        eps = 1e-6 * h
        fd = (O.kernel_w(kernel, dim, kappa, r + eps, h) - O.kernel_w(kernel, dim, kappa, r - eps, h)) / (2 * eps)
        dw = O.kernel_dw(kernel, dim, kappa, r, h)
        assert abs(dw - fd) <= 1e-7 * max(1.0, abs(fd)) / h ** (dim + 1)
        assert dw <= 0.0


def test_kernel_support_and_centre():
    # cubic spline centre values sigma_D / h^D and compact support 2h
    assert O.kernel_w(O.KERNEL_CUBIC, 3, 2.0, 0.0, 1.0) == pytest.approx(1.0 / math.pi, rel=1e-15)
    assert O.kernel_w(O.KERNEL_CUBIC, 1, 2.0, 0.0, 2.0) == pytest.approx(1.0 / 3.0, rel=1e-15)
    for kern, kap in [(O.KERNEL_CUBIC, 2.0), (O.KERNEL_WENDLAND_C2, 1.936)]:
        for dim in (1, 2, 3):
            assert O.kernel_w(kern, dim, kap, 2.0 if kern == 0 else kap, 1.0) == 0.0
            assert O.kernel_dw(kern, dim, kap, 2.0 if kern == 0 else kap, 1.0) == 0.0
    # Wendland C2: W(0) = 21/(2 pi H^3) in 3D with H = kappa h (Dehnen & Aly normalisation)
    H = 1.936 * 0.5
    assert O.kernel_w(O.KERNEL_WENDLAND_C2, 3, 1.936, 0.0, 0.5) == pytest.approx(21 / (2 * math.pi * H ** 3), rel=1e-14)
    # cubic spline W' and W'' both vanish at q = 2 (so forces switch off smoothly)
    h = 1.0
    assert abs(O.kernel_dw(0, 3, 2.0, 2.0 - 1e-6, h)) < 1e-11


# -------------------------------------------------------------------- EOS ---
def _isentropic_c2(mat, rho, e, drho=1e-6):
    """dP/drho along de = P/rho^2 drho, by central differences (independent of c)."""
    P0, _, _ = O.eos(mat, rho, e)
    h = drho * rho
    rp, rm = rho + h, rho - h
    # second-order step of the isentrope de/drho = P/rho^2
    Pp, _, _ = O.eos(mat, rp, e + P0 / rho ** 2 * h)
    Pm, _, _ = O.eos(mat, rm, e - P0 / rho ** 2 * h)
    return (Pp - Pm) / (2 * h)


def test_ideal_gas():
    m = O.Material(O.EOS_IDEAL, 1.4)
    P, c, bad = O.eos(m, 0.125, 2.0)
    assert P == pytest.approx(0.1, rel=1e-15) and not bad
    assert c * c == pytest.approx(_isentropic_c2(m, 0.125, 2.0), rel=1e-6)


def test_stiffened_gas_reference_state():
    rho0, c0, g = 2700.0, 5300.0, 2.0
    m = O.Material(O.EOS_STIFFENED, g, rho0, c0, rho0 * c0 * c0 / g)
    e0 = g * m.p_inf / ((g - 1.0) * rho0)
    P, c, bad = O.eos(m, rho0, e0)
    assert abs(P) < 1e-6 * m.p_inf and c == pytest.approx(c0, rel=1e-14) and not bad
    for rho, e in [(2900.0, e0 * 1.1), (2500.0, e0 * 0.95)]:
        _, c, _ = O.eos(m, rho, e)
        assert c * c == pytest.approx(_isentropic_c2(m, rho, e), rel=1e-6)


def test_tait():
    m = O.Material(O.EOS_TAIT, 7.0, 1000.0, 1500.0)
    P, c, _ = O.eos(m, 1000.0, 0.0)
    assert P == 0.0 and c == pytest.approx(1500.0, rel=1e-15)
    for rho in (990.0, 1010.0, 1100.0):
        _, c, _ = O.eos(m, rho, 0.0)
        assert c * c == pytest.approx(_isentropic_c2(m, rho, 0.0), rel=1e-6)


@pytest.mark.parametrize("name", ["mie_gruneisen_lead", "mie_gruneisen_aluminium"])
def test_mie_gruneisen_hugoniot(name):
    """The reference curves of eq. (mie_gruneisen_reference) lie on the shock
    Hugoniot u_s = c_a + s_a u_p: P_r = rho0 u_s u_p and e_r = u_p^2/2 at
    x = 1 - u_p/u_s (Rankine-Hugoniot jump conditions from rest)."""
    g = json.load(open(os.path.join(GOLD, "paper_constants.json")))[name]
    m = O.Material(O.EOS_MIE_GRUNEISEN, g["Gamma"], g["rho0"], g["c_a"], 0.0, g["s_a"])
    for up in (10.0, 300.0, 1000.0, 2000.0):
        us = g["c_a"] + g["s_a"] * up
        rho = g["rho0"] / (1.0 - up / us)
        P, c, bad = O.eos(m, rho, 0.5 * up * up)   # e = e_r: P reduces to P_r
        assert P == pytest.approx(g["rho0"] * us * up, rel=1e-12)
        assert not bad
        assert c * c == pytest.approx(_isentropic_c2(m, rho, 0.5 * up * up), rel=1e-5)
    P, c, _ = O.eos(m, g["rho0"], 0.0)
    assert abs(P) < 1e-9 and c == pytest.approx(g["c_a"], rel=1e-14)


# ---------------------------------------------------------------- Riemann ---
def test_sod_exact_solver_matches_textbook():
    ref = json.load(open(os.path.join(GOLD, "sod_star_state.json")))
    st = sod_exact.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    _, _, _, info = sod_exact.sample(np.array([0.5]), 1.0, 0.0, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    tol = ref["abs_tol"]
    assert abs(st["p"] - ref["p_star"]) < tol and abs(st["u"] - ref["u_star"]) < tol
    assert abs(st["rho_l"] - ref["rho_star_left"]) < tol and abs(st["rho_r"] - ref["rho_star_right"]) < tol
    assert abs(info["shock"] - ref["shock_speed"]) < tol
    assert abs(info["head"] - ref["rarefaction_head"]) < tol
    assert abs(info["tail"] - ref["rarefaction_tail"]) < tol


def test_acoustic_solver_equal_states_and_symmetry():
    P, v = O.riemann_acoustic(2.0, 2.0, 3.0, 3.0, 0.7, 0.7)
    assert P == pytest.approx(2.0, rel=1e-15) and v == pytest.approx(0.7, rel=1e-15)
    rng = np.random.default_rng(3)
    for _ in range(50):
        Pi, Pj, Zi, Zj = rng.uniform(0.1, 5.0, 4)
        vi, vj = rng.normal(size=2)
        Pa, va = O.riemann_acoustic(Pi, Pj, Zi, Zj, vi, vj)
        # seen from j the axis e^R flips: v^R -> -v^R, left/right swap
        Pb, vb = O.riemann_acoustic(Pj, Pi, Zj, Zi, -vj, -vi)
        assert Pa == pytest.approx(Pb, rel=1e-14) and va == pytest.approx(-vb, rel=1e-13, abs=1e-15)


def test_acoustic_solver_is_weak_wave_limit_of_exact_solver():
    """For small jumps the acoustic solution agrees with the exact ideal-gas
    Riemann solution with an error that falls like the square of the jump."""
    g = 1.4
    rl, pl = 1.0, 1.0
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        rr, pr, ul, ur = rl * (1 - eps), pl * (1 - 1.3 * eps), 0.2 * eps, -0.1 * eps
        ex = sod_exact.star_state(rl, ul, pl, rr, ur, pr, g)
        Zl, Zr = rl * math.sqrt(g * pl / rl), rr * math.sqrt(g * pr / rr)
        Pa, va = O.riemann_acoustic(pl, pr, Zl, Zr, ul, ur)
        errs.append(max(abs(Pa - ex["p"]) / pl, abs(va - ex["u"]) / math.sqrt(g * pl / rl)))
    assert errs[0] < 1e-4
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.3   # second order in the jump
