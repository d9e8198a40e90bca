"""Pins of the oracle's Voronoi decomposition (Sec. 3): ownership against a
k-d tree and constructed ties, and the balancing displacements against the
geometry and the qualitative results the paper states for them."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle as O
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


# ------------------------------------------------------------ assignment ---
@pytest.mark.parametrize("gdim", [1, 2, 3])
def test_assign_matches_kdtree(gdim):
    n, K = 5000, 37
    u = synth.uniform(21 + gdim, n * gdim + K * gdim)
    pts = u[: n * gdim].reshape(n, gdim)
    gen = u[n * gdim:].reshape(K, gdim)
    unit = O.voronoi_assign([pts[:, a] for a in range(gdim)], gen)
    _, ref = cKDTree(gen).query(pts, k=1)
    assert np.array_equal(unit, ref)


def test_assign_ties_go_to_smaller_index():
    """Sec. 3.1: a particle on the boundary of V_k and V_l belongs to V_min(k,l).
    Integer coordinates make the equal distances exact."""
    gen = np.array([[4.0, 0.0], [0.0, 0.0], [2.0, 2.0], [2.0, -2.0]])
    pts = np.array([[2.0, 0.0],    # equidistant from all four
                    [2.0, 5.0],    # equidistant from 0 and 1, nearer 2
                    [1.0, 1.0],    # equidistant from 1 and 2
                    [3.0, -1.0]])  # equidistant from 0 and 3
    unit = O.voronoi_assign([pts[:, 0], pts[:, 1]], gen)
    assert list(unit) == [0, 2, 1, 0]
    # 3D with the z coordinate deciding nothing
    gen3 = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    unit3 = O.voronoi_assign([np.zeros(3), np.zeros(3), np.array([0.0, 0.5, -0.5])], gen3)
    assert list(unit3) == [0, 0, 1]


# ------------------------------------------------------------- balancing ---
def _three(Lh=0.5, Ll=0.25, dsh=0.03):
    gen = np.array([[0.0, 0.2], [-0.2, -0.1], [0.2, -0.1]])
    load = np.array([Lh, Ll, Ll])
    adj = np.ones((3, 3), dtype=np.uint8) - np.eye(3, dtype=np.uint8)
    D = np.full((3, 3), dsh)
    return gen, load, adj, D, np.zeros((3, 2)), np.zeros(3, dtype=np.int64)


def test_static_and_lagrangian_limits():
    """gamma = theta = 0 is the static decomposition; theta = 1 puts each
    generator on its subdomain centre (Secs. 3.4 and 7.1)."""
    gen, load, adj, D, cen, cnt = _three()
    g, shift, _ = O.balance(gen, load, adj, D, cen, cnt, theta=0.0, sigma=0.5, gamma_b=0.0)
    assert np.array_equal(g, gen) and shift == 0.0
    cen = np.array([[0.1, 0.1], [-0.3, 0.0], [0.2, -0.2]])
    cnt = np.array([5, 6, 7])
    g, shift, _ = O.balance(gen, load, adj, D, cen, cnt, theta=1.0, sigma=0.5, gamma_b=1.0)
    assert np.allclose(g, cen, rtol=0, atol=1e-15)
    assert shift == pytest.approx(np.sum(np.linalg.norm(cen - gen, axis=1)), rel=1e-14)


def test_two_body_directions():
    """Eq. (BalancingOffset) with L_0 = L_h > L_1 = L_2 = L_l (Fig. 3a,b):
    the light generators move toward the heavy one by Dsh (L_h-L_l)/(L_h+L_l),
    the heavy one moves away by that length times |u_01 + u_02| (about twice it
    when both light units lie on the same side), so a heavy worker sheds
    particles to its lighter neighbours (Sec. 3.4)."""
    gen, load, adj, D, cen, cnt = _three()
    _, _, dg = O.balance(gen, load, adj, D, cen, cnt, theta=0.0, sigma=0.0, gamma_b=1.0)
    f = 0.03 * (0.5 - 0.25) / 0.75
    u01 = (gen[0] - gen[1]) / np.linalg.norm(gen[0] - gen[1])
    u02 = (gen[0] - gen[2]) / np.linalg.norm(gen[0] - gen[2])
    assert np.allclose(dg[1], f * u01, atol=1e-16)            # toward the heavy generator
    assert np.allclose(dg[2], f * u02, atol=1e-16)
    assert np.allclose(dg[0], f * (u01 + u02), atol=1e-16)     # away from both light ones
    assert np.linalg.norm(dg[0]) / np.linalg.norm(dg[1]) == pytest.approx(np.linalg.norm(u01 + u02))
    # the displacement is linear in a small imbalance
    _, _, dg2 = O.balance(gen, np.array([0.26, 0.25, 0.25]), adj, D, cen, cnt, 0.0, 0.0, 1.0)
    _, _, dg4 = O.balance(gen, np.array([0.27, 0.25, 0.25]), adj, D, cen, cnt, 0.0, 0.0, 1.0)
    assert np.linalg.norm(dg4[1]) / np.linalg.norm(dg2[1]) == pytest.approx(2.0, rel=0.03)


def test_three_body_rotation_geometry():
    """Eq. (BalancingOffsetRot) for the configuration of Fig. 3c: the light
    generator k is rotated about the circumcentre of the triangle, toward the
    heavy one, by alpha = pi/3 (L_h - L_l)/(L_h + 2 L_l); the heavy generator's
    two rotations cancel (alpha_0 ~ 0 in the caption)."""
    gen, load, adj, D, cen, cnt = _three(dsh=10.0)   # no length limit
    _, _, dg = O.balance(gen, load, adj, D, cen, cnt, theta=0.0, sigma=1.0, gamma_b=1.0)
    assert np.linalg.norm(dg[0]) < 1e-15
    # circumcentre of the three generators, from the perpendicular bisectors
    A = np.array([2 * (gen[1] - gen[0]), 2 * (gen[2] - gen[0])])
    b = np.array([gen[1] @ gen[1] - gen[0] @ gen[0], gen[2] @ gen[2] - gen[0] @ gen[0]])
    o = np.linalg.solve(A, b)
    alpha = math.pi / 3 * (0.5 - 0.25) / 1.0
    for k in (1, 2):
        c0, c1 = gen[k] - o, gen[k] + dg[k] - o
        assert np.linalg.norm(c1) == pytest.approx(np.linalg.norm(c0), rel=1e-12)   # stays on the circle
        ang = math.atan2(c0[0] * c1[1] - c0[1] * c1[0], c0 @ c1)
        assert abs(ang) == pytest.approx(alpha, rel=1e-12)
        # toward the heavy generator: the angular distance to it shrinks
        h = gen[0] - o
        before = math.acos(c0 @ h / np.linalg.norm(c0) / np.linalg.norm(h))
        after = math.acos(c1 @ h / np.linalg.norm(c1) / np.linalg.norm(h))
        assert after == pytest.approx(before - alpha, rel=1e-10)


def test_three_body_length_limit():
    """The three-body part is limited to max_l Dsh_kl (Sec. 3.3)."""
    gen, load, adj, D, cen, cnt = _three(Lh=10.0, Ll=0.01, dsh=0.001)
    _, _, dg = O.balance(gen, load, adj, D, cen, cnt, theta=0.0, sigma=1.0, gamma_b=1.0)
    assert np.all(np.linalg.norm(dg, axis=1) <= 0.001 * (1 + 1e-12))
    assert np.linalg.norm(dg[1]) == pytest.approx(0.001, rel=1e-12)


def test_no_three_body_term_in_3d():
    """3D decompositions use four-body terms (quadruples of mutually adjacent
    units) instead of the three-body ones: with three units there is none, so
    eq. (BalancingOffsetPlusRot) leaves (1 - sigma) times the two-body sum."""
    gen = np.array([[0.0, 0.2, 0.0], [-0.2, -0.1, 0.0], [0.2, -0.1, 0.0]])
    _, load, adj, D, _, _ = _three()
    cen, cnt = np.zeros((3, 3)), np.zeros(3, dtype=np.int64)
    _, _, dg0 = O.balance(gen, load, adj, D, cen, cnt, theta=0.0, sigma=0.0, gamma_b=1.0)
    _, _, dg5 = O.balance(gen, load, adj, D, cen, cnt, theta=0.0, sigma=0.5, gamma_b=1.0)
    _, _, dg1 = O.balance(gen, load, adj, D, cen, cnt, theta=0.0, sigma=1.0, gamma_b=1.0)
    assert np.max(np.abs(dg0)) > 0
    assert np.allclose(dg5, 0.5 * dg0, rtol=1e-15, atol=0) and np.max(np.abs(dg1)) == 0.0


# ------------------------------------------------- disk test of Sec. 5 ---
@pytest.fixture(scope="module")
def disk():
    g = GOLD["disk"]
    D = synth.disk(g["particles"], g["radius"], g["height"])
    n, a = len(D["x"]), D["a"]
    s = O.State(3, dict(x=D["x"], y=D["y"], z=D["z"], rho=np.ones(n), E=np.ones(n), m=np.full(n, a ** 3)))
    s.d[:] = a
    p = O.Params(dim=3, eta=1.3)
    pi, pj = O.pairs(p, s)
    return p, s, pi, pj


def _iterate(disk, g0, sigma, theta, iters=45):
    p, s, pi, pj = disk
    g = g0.copy()
    imb, shifts = [], []
    for _ in range(iters):
        unit = O.voronoi_assign([s.x, s.y], g)
        st = O.unit_stats(p, s, unit, 3, 2, pi, pj, 0.45)
        L = st["load"]
        imb.append((L.max() - L.min()) / L.mean())
        g, shift, _ = O.balance(g, L, st["adj"], st["dsh"], st["centroid"], st["count"], theta, sigma, 1.0)
        shifts.append(shift)
    # common point of the three subdomains = circumcentre of the generators
    A = np.array([2 * (g[1] - g[0]), 2 * (g[2] - g[0])])
    b = np.array([g[1] @ g[1] - g[0] @ g[0], g[2] @ g[2] - g[0] @ g[0]])
    o = np.linalg.solve(A, b)
    return dict(imb=imb, shifts=shifts, o=o, dsh=st["dsh"][0, 1],
                first_balanced=next(i for i, v in enumerate(imb + [0.0]) if v < 0.02),
                first_converged=next((i + 1 for i, v in enumerate(shifts) if v < 0.01), None))


def test_disk_convergence(disk):
    """Three subdomains of a disk at rest from an imbalanced start (about
    0.53/0.24/0.24 of the particles, cf. L_h ~ 2 L_l in Sec. 3.3).  Sec. 5:
    two-body displacements alone balance the loads but keep the initial
    geometry; three-body terms alone cannot move the common point; the
    combination with the cumulative movement (theta = 0.25) reaches the best
    decomposition, three equal sectors meeting at the disk centre, fastest.
    The paper's iteration counts (21/21/17/11) depend on its unstated initial
    generators: parity unpinned.  The benchmark reports the GPU's counts for
    the same start (extras.disk_balancing); they are not asserted."""
    g0 = np.array([[0.0, 0.1], [-0.12, -0.25], [0.12, -0.25]])
    two = _iterate(disk, g0, 0.0, 0.0)
    three = _iterate(disk, g0, 1.0, 0.0)
    comb = _iterate(disk, g0, 0.5, 0.0)
    best = _iterate(disk, g0, 0.5, 0.25)
    assert best["imb"][-1] < 0.02 and comb["imb"][-1] < 0.02 and two["imb"][-1] < 0.02
    assert np.linalg.norm(best["o"]) < best["dsh"]            # common point at the centre
    assert np.linalg.norm(two["o"]) > 2 * best["dsh"]          # two-body: geometry kept
    assert np.linalg.norm(three["o"]) > 2 * best["dsh"]        # three-body: common point stuck
    assert np.linalg.norm(best["o"]) < np.linalg.norm(comb["o"]) < np.linalg.norm(two["o"])
    assert best["first_balanced"] < comb["first_balanced"] < two["first_balanced"]
    assert best["first_converged"] is not None


# ------------------------------------------- quadrant test of Sec. 6 ---
def test_quadrant_imbalance_balances():
    """Static plate whose quadrants hold 3/8, 1/4, 1/4 and 1/8 of the
    subdomains (Sec. 6), generators jittered slightly.  Pure balancing
    (theta = 0) brings max/mean load from about 2.1 to <= 1.05; the
    cumulative movement with theta = 0.25 trades some balance for regular
    subdomain shapes (Sec. 3.4) and settles <= 1.10."""
    P = synth.plate_static(96, 96, 2, 1.0 / 96)
    n, a = len(P["x"]), P["a"]
    s = O.State(3, dict(x=P["x"], y=P["y"], z=P["z"], rho=np.ones(n), E=np.ones(n), m=np.full(n, a ** 3)))
    s.d[:] = a
    p = O.Params(dim=3, eta=1.3)
    pi, pj = O.pairs(p, s)
    K = 32
    split = (np.array(GOLD["quadrant_split"]["value"]) * K).astype(int)      # 12, 8, 8, 4
    gens = []
    u = synth.uniform(437, 2 * K)
    for cnt, (x0, y0) in zip(split, [(0, 0), (0.5, 0), (0, 0.5), (0.5, 0.5)]):
        side = int(math.ceil(math.sqrt(cnt)))
        for i in range(cnt):
            gx = x0 + (i % side + 0.5) / side * 0.5
            gy = y0 + (i // side + 0.5) / math.ceil(cnt / side) * 0.5
            gens.append([gx, gy])
    g0 = np.array(gens) + 0.01 * (u.reshape(K, 2) - 0.5)
    for theta, bound in ((0.0, 1.05), (0.25, 1.10)):
        g = g0.copy()
        ratios = []
        for _ in range(150):
            unit = O.voronoi_assign([s.x, s.y], g)
            st = O.unit_stats(p, s, unit, K, 2, pi, pj, 0.45)
            L = st["load"]
            ratios.append(L.max() / L.mean())
            g, _, _ = O.balance(g, L, st["adj"], st["dsh"], st["centroid"], st["count"], theta, 0.5, 1.0)
        assert ratios[0] > 1.5
        assert np.mean(ratios[-30:]) <= bound
