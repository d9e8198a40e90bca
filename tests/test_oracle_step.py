"""Pins of the oracle's whole scheme (rates + KDK leapfrog): the exact Sod
solution, exact mass conservation, momentum and energy conservation to
round-off, the sound speed of a small-amplitude pulse and the CFL formula."""
import math

import numpy as np
import pytest

import oracle as O
import sod_exact
import synth


def _sod(res: int, steps: int):
    """Equal-mass Sod set-up of the 400-particle workload at resolution res
    (res particles per unit length on the left, res/8 on the right)."""
    xl = 0.5 - (np.arange(res) + 0.5) / res
    xr = 0.5 + (np.arange(res // 4) + 0.5) / (res / 8)
    x = np.concatenate([xl[::-1], xr])
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    P = np.where(left, 1.0, 0.1)
    p = O.Params(dim=1, eta=1.5, cfl=0.3, materials=[O.Material(O.EOS_IDEAL, 1.4)])
    s = O.State(1, dict(x=x, vx=np.zeros_like(x), rho=rho, E=P / (0.4 * rho), m=np.full_like(x, 1.0 / res)))
    t, _ = O.step(p, s, steps)
    win = (s.x >= 0) & (s.x <= 1)
    ex, _, _, info = sod_exact.sample(s.x[win], t, 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    return s, t, float(np.mean(np.abs(s.rho[win] - ex))), info


def test_sod_first_order_convergence():
    """The first-order acoustic scheme converges to the exact Sod solution:
    L1 density error over [0, 1] at t ~ 0.175 falls with resolution and is
    below 2e-2 at four times the 400-particle resolution."""
    errs = {}
    for res in (320, 640, 1280):
        s, t, l1, info = _sod(res, 200 * res // 320)
        assert 0.17 < t < 0.18
        errs[res] = l1
    plateau = (s.x > 0.5 + info["tail"] * t + 0.02) & (s.x < 0.5 + info["shock"] * t - 0.02)
    assert np.median(s.vx[plateau]) == pytest.approx(info["u"], rel=0.03)
    assert errs[320] < 0.035
    assert errs[640] < 0.85 * errs[320] and errs[1280] < 0.75 * errs[640]
    assert errs[1280] < 2e-2


def test_sod_workload_waves():
    """400-particle workload: the shock, contact and rarefaction sit where the
    exact solution puts them."""
    prob = synth.sod_1d()
    p, s = O.from_problem(prob)
    t, dts = O.step(p, s, prob.n_steps)
    o = np.argsort(s.x)
    x, rho, vx = s.x[o], s.rho[o], s.vx[o]
    _, _, _, info = sod_exact.sample(np.array([0.5]), t, 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    # shock: rightmost particle with rho above the midpoint of rho*_R and rho_R
    mid = 0.5 * (info["rho_r"] + 0.125)
    xs = x[np.nonzero((rho > mid) & (x < 1.5))[0].max()]
    assert abs(xs - (0.5 + info["shock"] * t)) < 2.0 / 40 * 1.0
    # rarefaction: where the velocity first reaches u*/2, against the exact profile
    xf = np.linspace(0.0, 1.0, 20001)
    _, uf, _, _ = sod_exact.sample(xf, t, 0.5, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    x_exact = xf[np.argmax(uf >= 0.5 * info["u"])]
    sel = np.nonzero((x > 0.0) & (vx >= 0.5 * info["u"]))[0]
    assert abs(x[sel[0]] - x_exact) < 0.03
    # plateau velocity between the rarefaction tail and the shock (about 15
    # particles on the coarse right side at this resolution)
    sel = (x > 0.5 + info["tail"] * t + 0.05) & (x < 0.5 + info["shock"] * t - 0.05)
    assert np.median(vx[sel]) == pytest.approx(info["u"], rel=0.1)


def test_cfl_first_step():
    """dt = CFL min_i eta d_i / (c_i + |v_i|): at rest on the left Sod state,
    d = 1/320, c = sqrt(1.4)."""
    prob = synth.sod_1d(jitter=0.0)
    p, s = O.from_problem(prob)
    _, dts = O.step(p, s, 1)
    assert dts[0] == pytest.approx(0.3 * 1.5 / 320.0 / math.sqrt(1.4), rel=1e-14)


@pytest.mark.parametrize("case", ["sod", "plate_2d", "plate"])
def test_conservation(case):
    if case == "sod":
        prob = synth.sod_1d()
        steps = 200
    elif case == "plate_2d":
        prob = synth.plate_impact_2d(8, (24, 6), a=1e-4, v=1000.0, seed=3, jitter=0.05)
        steps = 30
    else:
        prob = synth.plate_impact(5, (14, 14, 5), a=1e-4, v=1000.0, units=4, seed=3, jitter=0.05)
        steps = 30
    p, s = O.from_problem(prob)
    c0 = O.conservation(s)
    O.step(p, s, steps)
    c1 = O.conservation(s)
    assert c1[0] == c0[0]                                    # mass: constant m, exact
    mom_scale = np.sum(s.m * np.sqrt(s.vx ** 2 + (s.vy ** 2 if s.vy is not None else 0)
                                     + (s.vz ** 2 if s.vz is not None else 0)))
    for a in (1, 2, 3):
        assert abs(c1[a] - c0[a]) <= 1e-12 * mom_scale
    assert abs(c1[4] - c0[4]) <= 1e-12 * abs(c0[4])


def test_sound_speed_of_small_pulse():
    """A small isentropic density bump in a uniform ideal gas at rest splits
    into two pulses that travel at +-c."""
    n, L = 2400, 2.0
    x = (np.arange(n) + 0.5) / n * L - 0.5 * L
    g, rho0, P0, amp, w = 1.4, 1.0, 1.0, 1e-4, 0.02
    rho = rho0 * (1.0 + amp * np.exp(-(x / w) ** 2))
    P = P0 * (rho / rho0) ** g
    m = rho / n * L          # equal spacing, mass follows the bump
    p = O.Params(dim=1, eta=1.5, cfl=0.3, materials=[O.Material(O.EOS_IDEAL, g)])
    s = O.State(1, dict(x=x, vx=np.zeros(n), rho=rho, E=P / ((g - 1) * rho), m=m))
    t, _ = O.step(p, s, 1000)
    c = math.sqrt(g * P0 / rho0)
    # window between the two pulses and the rarefaction entering from the free end
    right = (s.x > 0.5 * c * t) & (s.x < 0.5 * L - 1.5 * c * t)
    dr = s.rho[right] - rho0
    xc = np.sum(s.x[right] * dr) / np.sum(dr)
    assert xc == pytest.approx(c * t, rel=0.02)
