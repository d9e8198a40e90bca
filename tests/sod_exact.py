"""Exact solution of the Riemann problem for an ideal gas (textbook, e.g.
Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4).

Independent of the oracle: the star-region pressure is found by Newton
iteration on the pressure function f_L(p) + f_R(p) + (u_R - u_L) = 0 with the
shock (Rankine-Hugoniot) and rarefaction (isentropic) branches, then the
self-similar solution is sampled at x/t.
"""
from __future__ import annotations

import math

import numpy as np


def _f(p, rho, pk, c, g):
    if p > pk:  # shock branch
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction branch
    r = (p / pk) ** ((g - 1.0) / (2.0 * g))
    return 2.0 * c / (g - 1.0) * (r - 1.0), 1.0 / (rho * c) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


def star_state(rl, ul, pl, rr, ur, pr, g=1.4, tol=1e-14):
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = max(tol, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dl = _f(p, rl, pl, cl, g)
        fr, dr = _f(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        pn = max(p - dp, tol)
        if abs(pn - p) < tol * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, cl, g)
    fr, _ = _f(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    gm = (g - 1.0) / (g + 1.0)
    rsl = rl * ((p / pl + gm) / (gm * p / pl + 1.0)) if p > pl else rl * (p / pl) ** (1.0 / g)
    rsr = rr * ((p / pr + gm) / (gm * p / pr + 1.0)) if p > pr else rr * (p / pr) ** (1.0 / g)
    return dict(p=p, u=u, rho_l=rsl, rho_r=rsr, cl=cl, cr=cr)


def sample(x, t, x0, rl, ul, pl, rr, ur, pr, g=1.4):
    """Density, velocity and pressure at positions x and time t > 0.
    Only the waves of the Sod configuration (left rarefaction, right shock)
    are handled, which is all the tests need."""
    st = star_state(rl, ul, pl, rr, ur, pr, g)
    ps, us = st["p"], st["u"]
    cl, cr = st["cl"], st["cr"]
    assert ps <= pl and ps > pr, "only left rarefaction + right shock"
    s = (np.asarray(x, dtype=np.float64) - x0) / t
    rho = np.empty_like(s); u = np.empty_like(s); p = np.empty_like(s)
    csl = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
    head, tail = ul - cl, us - csl
    shock = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
    for i, si in enumerate(s):
        if si < head:
            rho[i], u[i], p[i] = rl, ul, pl
        elif si < tail:
            uu = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + si)
            cc = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - si))
            rho[i] = rl * (cc / cl) ** (2.0 / (g - 1.0))
            u[i] = uu
            p[i] = pl * (cc / cl) ** (2.0 * g / (g - 1.0))
        elif si < us:
            rho[i], u[i], p[i] = st["rho_l"], us, ps
        elif si < shock:
            rho[i], u[i], p[i] = st["rho_r"], us, ps
        else:
            rho[i], u[i], p[i] = rr, ur, pr
    return rho, u, p, dict(head=head, tail=tail, shock=shock, **st)
