"""Pins of the oracle's neighbour search (Sec. 4.2): the cell/linked-list
search equals the O(N^2) definition, agrees with scipy's k-d tree, gives the
lattice neighbour counts fixed by arithmetic, and the cell mesh of eq. (Dcell)
holds every particle inside its own cell."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle as O
import synth


def _state(dim, pos, d):
    n = len(pos[0])
    arrays = dict(x=pos[0], rho=np.ones(n), E=np.ones(n), m=d ** dim)
    if dim >= 2:
        arrays["y"] = pos[1]
    if dim >= 3:
        arrays["z"] = pos[2]
    s = O.State(dim, arrays)
    s.d[:] = d
    return s


def _jittered_lattice(dim, n_side, jitter, seed, contrast=False):
    g = np.meshgrid(*[np.arange(n_side, dtype=float)] * dim, indexing="ij")
    pos = [a.ravel() for a in g]
    u = synth.uniform(seed, dim * len(pos[0]))
    pos = [p + jitter * (2 * u[a::dim] - 1) for a, p in enumerate(pos)]
    d = np.ones(len(pos[0]))
    if contrast:  # a block of large particles: size contrast as in a gas/liquid mix
        d[pos[0] > 0.6 * n_side] = 3.0
    return pos, d


@pytest.mark.parametrize("dim,n_side,contrast", [(1, 300, False), (1, 300, True), (2, 30, False),
                                                 (3, 10, False), (3, 11, True)])
def test_cells_equal_brute_force(dim, n_side, contrast):
    pos, d = _jittered_lattice(dim, n_side, 0.3, 11 + dim, contrast)
    s = _state(dim, pos, d)
    p = O.Params(dim=dim, eta=1.3)
    a = O.pairs(p, s, "cells")
    b = O.pairs(p, s, "brute")
    assert len(a[0]) > 0
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("dim", [1, 3])
def test_brute_force_matches_kdtree(dim):
    """scipy's k-d tree finds every candidate within the largest radius; the
    interacting pairs are those closer than kappa eta (d_i+d_j)/2."""
    pos, d = _jittered_lattice(dim, 200 if dim == 1 else 9, 0.35, 5, contrast=True)
    s = _state(dim, pos, d)
    p = O.Params(dim=dim, eta=1.3, kappa=2.0)
    pi, pj = O.pairs(p, s, "brute")
    pts = np.stack(pos, axis=1)
    kh = 0.5 * 2.0 * 1.3
    cand = cKDTree(pts).query_pairs(kh * 2 * d.max() * 1.0001, output_type="ndarray")
    dist = np.linalg.norm(pts[cand[:, 0]] - pts[cand[:, 1]], axis=1)
    R = kh * (d[cand[:, 0]] + d[cand[:, 1]])
    sel = cand[dist < R]
    sel = np.sort(sel, axis=1)
    sel = sel[np.lexsort((sel[:, 1], sel[:, 0]))]
    assert np.array_equal(sel[:, 0], pi) and np.array_equal(sel[:, 1], pj)


def test_lattice_neighbour_counts():
    """Perfect cubic lattice, h = 1.3 a, support 2h: lattice points with
    0 < r^2 < 6.76 a^2 are the shells r^2 = 1, 2, 3, 4, 5, 6 with 6, 12, 8, 6,
    24, 24 points: 80 neighbours.  Square lattice, same h: r^2 = 1, 2, 4, 5
    with 4, 4, 4, 8 points: 20 neighbours.  1D with h = 1.5 a: 4 neighbours."""
    n = 9
    pos, d = _jittered_lattice(3, n, 0.0, 0)
    s = _state(3, pos, d)
    pi, pj = O.pairs(O.Params(dim=3, eta=1.3), s)
    cnt = np.bincount(np.concatenate([pi, pj]), minlength=s.n)
    centre = (n // 2) + n * (n // 2) + n * n * (n // 2)
    assert cnt[centre] == 80
    pos, d = _jittered_lattice(2, n, 0.0, 0)
    s = _state(2, pos, d)
    pi, pj = O.pairs(O.Params(dim=2, eta=1.3), s)
    cnt = np.bincount(np.concatenate([pi, pj]), minlength=s.n)
    assert cnt[(n // 2) + n * (n // 2)] == 20
    pos, d = _jittered_lattice(1, 50, 0.0, 0)
    s = _state(1, pos, d)
    pi, pj = O.pairs(O.Params(dim=1, eta=1.5), s)
    cnt = np.bincount(np.concatenate([pi, pj]), minlength=s.n)
    assert cnt[25] == 4


def test_cell_grid_contains_particles_and_support():
    pos, d = _jittered_lattice(3, 12, 0.4, 9, contrast=True)
    s = _state(3, pos, d)
    p = O.Params(dim=3, eta=1.3)
    g, cell = O.cell_grid(p, s)
    # eq. (Dcell): D^c covers the largest interaction radius
    dmax2 = np.sort(d)[-2:].sum()
    assert g["dc"] >= 0.5 * 2.0 * 1.3 * dmax2
    nx, ny, nz = g["dims"]
    cx, cy, cz = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    for c, x, x0 in ((cx, pos[0], g["x0"][0]), (cy, pos[1], g["x0"][1]), (cz, pos[2], g["x0"][2])):
        lo = x0 + c * g["dc"]
        assert np.all(lo <= x + 1e-12) and np.all(x < lo + g["dc"] + 1e-12)
    assert cell.max() < g["ncells"] and cell.min() >= 0


def test_cell_grid_capacity_doubling():
    pos, d = _jittered_lattice(3, 12, 0.4, 9)
    s = _state(3, pos, d)
    g_big, _ = O.cell_grid(O.Params(dim=3, eta=1.3), s)
    g_small, _ = O.cell_grid(O.Params(dim=3, eta=1.3, cell_cap=20), s)
    assert g_small["ncells"] <= 20
    ratio = g_small["dc"] / g_big["dc"]
    assert ratio > 1 and np.log2(ratio) == int(np.log2(ratio))
    # the pair set does not depend on the cell size
    a = O.pairs(O.Params(dim=3, eta=1.3, cell_cap=20), s)
    b = O.pairs(O.Params(dim=3, eta=1.3), s)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
