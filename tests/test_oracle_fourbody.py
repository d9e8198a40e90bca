"""Pins of the oracle's four-body balancing term for 3D decompositions (the
paper names a rotation on the circumsphere of four generators without a
formula; the reading is in orc_balance).  What the construction fixes:

  * the rotations keep |c_k|: after a four-body-only update (sigma = 1,
    theta = 0) of one mutually adjacent quadruple every generator lies on the
    circumsphere of the old generators, whose centre (the common point) is
    unchanged;
  * equal loads give no displacement;
  * a lighter unit turns toward a heavier neighbour;
  * the update does not depend on the labels of the units;
  * on a 4-unit ball the loads balance, and adding the four-body term
    (sigma = 0.5) is not slower than the two-body term alone.
"""
import numpy as np
import pytest

import oracle as O
import synth

ADJ4 = np.ones((4, 4), np.uint8) - np.eye(4, dtype=np.uint8)


def _circumcentre(g):
    a, b, c = g[1] - g[0], g[2] - g[0], g[3] - g[0]
    M = 2 * np.array([a, b, c])
    rhs = np.array([a @ a, b @ b, c @ c])
    return g[0] + np.linalg.solve(M, rhs)


def _gens(seed=3):
    u = synth.uniform(seed, 12).reshape(4, 3)
    tet = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) / np.sqrt(3)
    return tet + 0.3 * (u - 0.5)


def _update(g, load, theta=0.0, sigma=1.0):
    dsh = np.full((4, 4), 1e3)                  # no length limit
    cnt = np.full(4, 100, dtype=np.int64)
    new, _, dg = O.balance(g, load, ADJ4, dsh, g.copy(), cnt, theta=theta, sigma=sigma, gamma_b=1.0)
    return new, dg


def test_four_body_rotation_keeps_the_circumsphere():
    g = _gens()
    o = _circumcentre(g)
    R = np.linalg.norm(g - o, axis=1)
    assert np.allclose(R, R[0], rtol=1e-12)
    new, dg = _update(g, np.array([0.1, 0.2, 0.3, 0.4]))
    assert np.max(np.abs(dg)) > 1e-3                                    # it moved
    assert np.allclose(np.linalg.norm(new - o, axis=1), R, rtol=1e-12)  # on the sphere
    assert np.allclose(_circumcentre(new), o, atol=1e-12)               # same common point


def test_equal_loads_give_no_displacement():
    g = _gens(5)
    new, dg = _update(g, np.full(4, 0.25))
    assert np.max(np.abs(dg)) == 0.0 and np.array_equal(new, g)


def test_lighter_unit_turns_toward_heavier_neighbour():
    g = _gens(7)
    o = _circumcentre(g)
    load = np.array([0.1, 0.4, 0.25, 0.25])    # unit 0 light, unit 1 heavy, 2 and 3 equal to the mean
    new, _ = _update(g, load)
    cos_old = (g[0] - o) @ (g[1] - o) / np.linalg.norm(g[0] - o) / np.linalg.norm(g[1] - o)
    cos_new = (new[0] - o) @ (g[1] - o) / np.linalg.norm(new[0] - o) / np.linalg.norm(g[1] - o)
    assert cos_new > cos_old


def test_update_is_label_independent():
    g = _gens(9)
    load = np.array([0.15, 0.35, 0.2, 0.3])
    new, _ = _update(g, load, theta=0.25, sigma=0.5)
    perm = np.array([2, 0, 3, 1])
    newp, _ = _update(g[perm], load[perm], theta=0.25, sigma=0.5)
    assert np.allclose(newp, new[perm], rtol=0, atol=1e-12)


def _ball_run(sigma, theta, iters):
    n = 20000
    u = synth.uniform(41, 3 * n).reshape(3, n)
    P = 2 * u - 1
    P = P[:, (P ** 2).sum(axis=0) <= 1]
    tet = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) / np.sqrt(3) * 0.5
    g = tet + np.array([0.25, 0.2, 0.15])         # off-centre: one unit holds far more particles
    hist = []
    for _ in range(iters):
        unit = O.voronoi_assign([P[0], P[1], P[2]], g)
        cnt = np.bincount(unit, minlength=4).astype(np.int64)
        load = cnt / cnt.sum()
        cen = np.array([P[:, unit == k].mean(axis=1) for k in range(4)])
        hist.append(load.max() / load.mean())
        g, _, _ = O.balance(g, load, ADJ4, np.full((4, 4), 0.1), cen, cnt, theta=theta, sigma=sigma)
    return np.array(hist)


def test_four_unit_ball_balances():
    h0 = _ball_run(0.0, 0.0, 21)
    h5 = _ball_run(0.5, 0.0, 21)
    assert h0[0] > 1.3
    assert h5[20] < 1.01 and h5[20] <= h0[20]
