"""Hand-worked pins of the oracle's work-unit statistics (orc_unit_stats),
which feed every balancing update: the load of each unit (Sec. 1 and
Sec. 2 name interaction counts as the load; an interacting pair inside a
unit counts 1, a pair joining two units 1/2 to each), the adjacency of
units (a pair joining them), the horizon D^sh_kl of eq. (Horizon) with
R^hrz_i = (1 + beta) kh (d_i + max_j d_j) over the interacting neighbours j
of i (Sec. 4.2-4.3; an isolated particle takes its own size), and the mean
position and particle count of each unit (the r_c,k of eq. (TotalOffset)).

Every expected value below is worked out by hand from those definitions on
a configuration small enough to check on paper; none is produced by the
code under test."""
import numpy as np

import oracle as O

BETA = 0.45


def _state(dim, pos, d, kappa, eta):
    """Particles at rest with rho = 1, an ideal gas at e = 1, and masses
    giving the sizes d (1D: d = m/rho, 2D: d = sqrt(m/rho))."""
    n = len(d)
    d = np.asarray(d, dtype=float)
    m = d if dim == 1 else d * d
    arrays = {"x": np.asarray(pos[0], float), "vx": np.zeros(n), "rho": np.ones(n), "E": np.ones(n), "m": m}
    if dim >= 2:
        arrays["y"] = np.asarray(pos[1], float)
        arrays["vy"] = np.zeros(n)
    p = O.Params(dim=dim, kappa=kappa, eta=eta, materials=[O.Material(O.EOS_IDEAL, 1.4)])
    s = O.State(dim, arrays)
    assert O.derive(p, s) >= 0
    assert np.allclose(s.d, d, rtol=1e-15, atol=0)
    return p, s


def test_unit_stats_1d_three_units_by_hand():
    """x = 0, 1, 2, 3.5, 10 with d = 1, 1.1, 1.5, 2.4, 0.5, kappa = 2,
    eta = 1.5 (kh = 1.5): particles 0-3 all interact (r < 1.5 (d_i + d_j)
    for each of the six pairs), particle 4 interacts with none.
    Units (0, 0, 1, 1, 2)."""
    p, s = _state(1, [[0.0, 1.0, 2.0, 3.5, 10.0]], [1.0, 1.1, 1.5, 2.4, 0.5], kappa=2.0, eta=1.5)
    pi, pj = O.pairs(p, s, "brute")
    assert list(zip(pi.tolist(), pj.tolist())) == [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    unit = np.array([0, 0, 1, 1, 2], dtype=np.int32)
    st = O.unit_stats(p, s, unit, 3, 1, pi, pj, BETA)

    # loads: (0,1) inside unit 0 -> 1; (2,3) inside unit 1 -> 1; the four pairs
    # (0,2), (0,3), (1,2), (1,3) join units 0 and 1 -> 1/2 to each
    assert st["load"].tolist() == [3.0, 3.0, 0.0]
    # adjacency: only units 0 and 1 share a pair; unit 2 is isolated
    assert st["adj"].tolist() == [[0, 1, 0], [1, 0, 0], [0, 0, 0]]
    # largest interacting neighbour size: p0 -> 2.4, p1 -> 2.4, p2 -> 2.4,
    # p3 -> 1.5 (p2), p4 -> none, its own 0.5; d_i + max_j d_j = 3.4, 3.5,
    # 3.9, 3.9, 1.0; R^hrz = 1.45 * 1.5 * (d_i + max_j d_j); per unit the
    # largest: 1.45 * 1.5 * 3.5 = 7.6125, 1.45 * 1.5 * 3.9 = 8.4825,
    # 1.45 * 1.5 * 1.0 = 2.175; D^sh_kl = max over both units
    r = [7.6125, 8.4825, 2.175]
    want = np.array([[max(r[k], r[l]) for l in range(3)] for k in range(3)])
    np.testing.assert_allclose(st["dsh"], want, rtol=1e-14, atol=0)
    # centroids and counts
    np.testing.assert_allclose(st["centroid"][:, 0], [0.5, 2.75, 10.0], rtol=1e-15, atol=0)
    assert st["count"].tolist() == [2, 2, 1]


def test_unit_stats_2d_isolated_particle_shares_a_unit():
    """2D, kappa = 2, eta = 1.3 (kh = 1.3): p0 (0, 0) d 1, p1 (1, 0) d 1.5,
    p2 (0, 1) d 2, p3 (5, 5) d 1.  Pairs (0,1), (0,2), (1,2) (r = 1, 1,
    sqrt 2 against 1.3 (d_i + d_j) = 3.25, 3.9, 4.55); p3 interacts with
    none (r >= 6.4 > 3.9).  Units (0, 1, 1, 0): the isolated p3 sits in
    unit 0 with p0."""
    p, s = _state(2, [[0.0, 1.0, 0.0, 5.0], [0.0, 0.0, 1.0, 5.0]], [1.0, 1.5, 2.0, 1.0], kappa=2.0, eta=1.3)
    pi, pj = O.pairs(p, s, "brute")
    assert list(zip(pi.tolist(), pj.tolist())) == [(0, 1), (0, 2), (1, 2)]
    unit = np.array([0, 1, 1, 0], dtype=np.int32)
    st = O.unit_stats(p, s, unit, 2, 2, pi, pj, BETA)
    # loads: (0,1), (0,2) join the units -> 1/2 + 1/2 to each; (1,2) inside unit 1 -> 1
    assert st["load"].tolist() == [1.0, 2.0]
    assert st["adj"].tolist() == [[0, 1], [1, 0]]
    # max neighbour size: p0 -> 2, p1 -> 2, p2 -> 1.5, p3 -> own 1;
    # d + max = 3, 3.5, 3.5, 2; unit 0: max(3, 2) = 3 -> 1.45 * 1.3 * 3 = 5.655;
    # unit 1: 3.5 -> 1.45 * 1.3 * 3.5 = 6.5975
    want = np.array([[5.655, 6.5975], [6.5975, 6.5975]])
    np.testing.assert_allclose(st["dsh"], want, rtol=1e-14, atol=0)
    np.testing.assert_allclose(st["centroid"], [[2.5, 2.5], [0.5, 0.5]], rtol=1e-15, atol=0)
    assert st["count"].tolist() == [2, 2]


def test_unit_stats_horizon_uses_the_buffer_and_the_neighbour_size():
    """The horizon scales with (1 + beta) and with the neighbour's size, not
    the particle's own twice: at beta = 0 the 1D case gives 1.5 * 3.5 and
    1.5 * 3.9, and enlarging p3 (d 2.4 -> 3.0, still interacting with
    p0-p2) raises the horizon of unit 0 through its neighbour p3."""
    p, s = _state(1, [[0.0, 1.0, 2.0, 3.5, 10.0]], [1.0, 1.1, 1.5, 2.4, 0.5], kappa=2.0, eta=1.5)
    pi, pj = O.pairs(p, s, "brute")
    unit = np.array([0, 0, 1, 1, 2], dtype=np.int32)
    st0 = O.unit_stats(p, s, unit, 3, 1, pi, pj, 0.0)
    np.testing.assert_allclose(np.diag(st0["dsh"]), [5.25, 5.85, 1.5], rtol=1e-14, atol=0)
    p, s = _state(1, [[0.0, 1.0, 2.0, 3.5, 10.0]], [1.0, 1.1, 1.5, 3.0, 0.5], kappa=2.0, eta=1.5)
    pi, pj = O.pairs(p, s, "brute")
    assert list(zip(pi.tolist(), pj.tolist())) == [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    st1 = O.unit_stats(p, s, unit, 3, 1, pi, pj, 0.0)
    # unit 0: p1 has d 1.1 and largest neighbour 3.0 -> 1.5 * 4.1 = 6.15;
    # unit 1: p3 has d 3.0 and largest neighbour 1.5 -> 1.5 * 4.5 = 6.75
    np.testing.assert_allclose(np.diag(st1["dsh"]), [6.15, 6.75, 1.5], rtol=1e-14, atol=0)
