"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it lays particles on lattices,
sets the initial states of each test problem, seeds Voronoi generators and
draws random numbers.  Both the oracle and the CUDA path take their inputs
from here, as plain numpy arrays.

Random numbers come from splitmix64 (Steele, Lea, Flood 2014; the public
reference mixer): state advances by 0x9E3779B97F4A7C15 and each output is
mixed by the two multiply/xor-shift rounds below, then mapped to [0, 1) by
its top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of splitmix64 started from ``seed``, skipping ``offset``."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ---------------------------------------------------------------------------
# Problem descriptions
# ---------------------------------------------------------------------------
@dataclass
class MaterialSpec:
    eos: str            # "ideal" | "stiffened" | "tait" | "mie_gruneisen"
    gamma: float
    rho0: float = 1.0
    c0: float = 1.0
    p_inf: float = 0.0
    s_a: float = 0.0


@dataclass
class Problem:
    """A particle set with its physical parameters (host float64 arrays)."""
    name: str
    dim: int
    arrays: dict                      # x, y, z, vx, vy, vz, rho, E, m (float64)
    materials: list
    mat: np.ndarray | None = None     # int32 material index per particle
    kernel: str = "cubic"             # "cubic" | "wendland_c2"
    kappa: float = 2.0
    eta: float = 1.3
    cfl: float = 0.3
    n_steps: int = 100
    units: int = 1                    # Voronoi work units K
    unit_dim: int = 1                 # dimension of the Voronoi decomposition
    n_upd: int = 10                   # steps between rebalancing
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.arrays["x"])


# ---------------------------------------------------------------------------
# 1D Sod shock tube (ideal gas gamma = 1.4, 400 equal-mass particles)
# ---------------------------------------------------------------------------
def sod_1d(seed: int = 1805, jitter: float = 1e-6) -> Problem:
    """Left state rho=1, p=1 on spacing 1/320 (320 particles covering
    [-0.5, 0.5]); right state rho=0.125, p=0.1 on spacing 1/40 (80 particles
    covering [0.5, 2.5]); mass 1/320 each; diaphragm at x = 0.5; positions
    jittered uniformly by +-jitter.  Free ends lie beyond the wave fan so the
    window [0, 1] sees only the Sod waves up to t ~ 0.25."""
    g = 1.4
    xl = 0.5 - (np.arange(320) + 0.5) / 320.0
    xr = 0.5 + (np.arange(80) + 0.5) / 40.0
    x = np.concatenate([xl[::-1], xr])
    x = x + jitter * (2.0 * uniform(seed, len(x)) - 1.0)
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    e = p / ((g - 1.0) * rho)          # initial internal energy from the stated pressure
    n = len(x)
    arrays = dict(x=x, vx=np.zeros(n), rho=rho, E=e.copy(), m=np.full(n, 1.0 / 320.0))
    return Problem("sod_1d_400", 1, arrays, [MaterialSpec("ideal", g)], kernel="cubic",
                   kappa=2.0, eta=1.5, cfl=0.3, n_steps=200, units=4, unit_dim=1, n_upd=10,
                   meta=dict(gamma=g, diaphragm=0.5, window=(0.0, 1.0)))


# ---------------------------------------------------------------------------
# 3D plate impact (stiffened gas), projector cube onto a target slab
# ---------------------------------------------------------------------------
def stiffened(rho0: float, c0: float, gamma: float) -> MaterialSpec:
    """Stiffened gas whose reference state (rho0, P=0) has sound speed c0:
    P_inf = rho0 c0^2 / gamma."""
    return MaterialSpec("stiffened", gamma, rho0=rho0, c0=c0, p_inf=rho0 * c0 * c0 / gamma)


def plate_impact(proj: int = 50, target=(200, 200, 25), a: float = 1e-4, v: float = 1000.0,
                 rho0: float = 2700.0, c0: float = 5300.0, gamma: float = 2.0,
                 units: int = 64, n_steps: int = 500, seed: int | None = None,
                 jitter: float = 0.0) -> Problem:
    """Cubic lattices of spacing a: target slab tx*ty*tz with layers z = k a
    (k = 0..tz-1), projector cube proj^3 centred above it with its lowest
    layer at z = (tz + 1) a (a surface gap of one spacing), moving at -v along
    z.  Both at rho0 and P = 0 (internal energy gamma P_inf / ((gamma-1) rho0)),
    mass rho0 a^3."""
    tx, ty, tz = target
    i, j, k = np.meshgrid(np.arange(tx), np.arange(ty), np.arange(tz), indexing="ij")
    xt = ((i - (tx - 1) / 2.0) * a).ravel()
    yt = ((j - (ty - 1) / 2.0) * a).ravel()
    zt = (k * a).ravel().astype(np.float64)
    i, j, k = np.meshgrid(np.arange(proj), np.arange(proj), np.arange(proj), indexing="ij")
    xp = ((i - (proj - 1) / 2.0) * a).ravel()
    yp = ((j - (proj - 1) / 2.0) * a).ravel()
    zp = ((k + tz + 1) * a).ravel().astype(np.float64)
    x = np.concatenate([xt, xp]); y = np.concatenate([yt, yp]); z = np.concatenate([zt, zp])
    n = len(x)
    if seed is not None and jitter > 0.0:
        r = uniform(seed, 3 * n)
        x = x + jitter * a * (2.0 * r[0::3] - 1.0)
        y = y + jitter * a * (2.0 * r[1::3] - 1.0)
        z = z + jitter * a * (2.0 * r[2::3] - 1.0)
    vz = np.concatenate([np.zeros(len(xt)), np.full(len(xp), -v)])
    mat = stiffened(rho0, c0, gamma)
    e0 = gamma * mat.p_inf / ((gamma - 1.0) * rho0)
    arrays = dict(x=x, y=y, z=z, vx=np.zeros(n), vy=np.zeros(n), vz=vz,
                  rho=np.full(n, rho0), E=e0 + 0.5 * vz * vz, m=np.full(n, rho0 * a ** 3))
    return Problem(f"plate_impact_{n}", 3, arrays, [mat], kernel="cubic", kappa=2.0, eta=1.3,
                   cfl=0.3, n_steps=n_steps, units=units, unit_dim=2, n_upd=10,
                   meta=dict(a=a, v=v, target=target, proj=proj, n_target=len(xt)))


def plate_impact_2d(proj: int = 20, target=(80, 12), a: float = 1e-4, v: float = 1000.0,
                    rho0: float = 2700.0, c0: float = 5300.0, gamma: float = 2.0, units: int = 0,
                    n_steps: int = 100, seed: int | None = None, jitter: float = 0.0) -> Problem:
    """The plate impact in a plane (x, y), y the impact axis: square lattices of
    spacing a, target tx*ty with rows y = k a (k = 0..ty-1), projector square
    proj^2 centred above it with its lowest row at y = (ty + 1) a, moving at -v
    along y; both at rho0 and P = 0; mass rho0 a^2 (so d = a)."""
    tx, ty = target
    i, k = np.meshgrid(np.arange(tx), np.arange(ty), indexing="ij")
    xt = ((i - (tx - 1) / 2.0) * a).ravel()
    yt = (k * a).ravel().astype(np.float64)
    i, k = np.meshgrid(np.arange(proj), np.arange(proj), indexing="ij")
    xp = ((i - (proj - 1) / 2.0) * a).ravel()
    yp = ((k + ty + 1) * a).ravel().astype(np.float64)
    x = np.concatenate([xt, xp]); y = np.concatenate([yt, yp])
    n = len(x)
    if seed is not None and jitter > 0.0:
        r = uniform(seed, 2 * n)
        x = x + jitter * a * (2.0 * r[0::2] - 1.0)
        y = y + jitter * a * (2.0 * r[1::2] - 1.0)
    vy = np.concatenate([np.zeros(len(xt)), np.full(len(xp), -v)])
    mat = stiffened(rho0, c0, gamma)
    e0 = gamma * mat.p_inf / ((gamma - 1.0) * rho0)
    arrays = dict(x=x, y=y, vx=np.zeros(n), vy=vy, rho=np.full(n, rho0), E=e0 + 0.5 * vy * vy,
                  m=np.full(n, rho0 * a ** 2))
    return Problem(f"plate_impact_2d_{n}", 2, arrays, [mat], kernel="cubic", kappa=2.0, eta=1.3,
                   cfl=0.3, n_steps=n_steps, units=units, unit_dim=2, n_upd=10,
                   meta=dict(a=a, v=v, target=target, proj=proj, n_target=len(xt)))


def plate_impact_full() -> Problem:
    """1.125M particles: 50^3 projector at 1 km/s onto a 200x200x25 slab."""
    return plate_impact(50, (200, 200, 25), units=64, n_steps=500)


def plate_impact_small() -> Problem:
    """~203k particles: 25^3 projector onto a 120x120x13 slab, 100 steps."""
    return plate_impact(25, (120, 120, 13), units=64, n_steps=100)


def ensemble(n_inst: int = 256, seed: int = 2018, n_min: int = 5000, n_max: int = 200000,
             v_range=(500.0, 2000.0), gamma_range=(1.5, 3.0), a: float = 1e-4) -> list:
    """Independent plate impacts of uneven size: instance b has about N_b
    particles, N_b log-uniform in [n_min, n_max]; impact speed uniform in
    v_range, stiffened-gas gamma uniform in gamma_range (rho0 = 2700,
    c0 = 5300).  Each has the shape of the 1.125M plate (projector p^3 on a
    4p x 4p x p/2 slab, N = 9 p^3)."""
    u = uniform(seed, 3 * n_inst).reshape(n_inst, 3)
    probs = []
    for b in range(n_inst):
        nb = n_min * (n_max / n_min) ** u[b, 0]
        p = max(int(round((nb / 9.0) ** (1.0 / 3.0))), 4)
        v = v_range[0] + (v_range[1] - v_range[0]) * u[b, 1]
        g = gamma_range[0] + (gamma_range[1] - gamma_range[0]) * u[b, 2]
        probs.append(plate_impact(p, (4 * p, 4 * p, max(p // 2, 2)), a=a, v=v, gamma=g, units=0, n_steps=100))
    return probs


def lead() -> MaterialSpec:
    """Lead as in the ejecta test of Sec. 7: Mie-Grueneisen with rho0 = 11.35
    g/cc, c_a = 2.58 km/s, s_a = 1.26, Gamma = 1.7 (SI units)."""
    return MaterialSpec("mie_gruneisen", 1.7, rho0=11350.0, c0=2580.0, s_a=1.26)


def ejecta(nx: int = 100, periods: int = 2, lam: int = 40, nz: int = 10, a: float = 1e-7,
           up: float = 1000.0, units: int = 64, n_steps: int = 200) -> Problem:
    """Grooved lead sample driven onto a rigid wall (the ejecta test of Sec. 7,
    synthetic): a cubic lattice of spacing a, nx layers along x, `periods`
    grooves of period lam spacings along y, nz layers along z; the free face
    at x = nx a carries 90-degree V-grooves (depth lam/2 spacings at the
    groove centre, none at the ridges).  The rigid wall is the symmetry plane
    of a mirror copy: the sample at x >= 0 moves at -up, its mirror image
    (x -> -x - a) at +up, so the plane x = -a/2 stays at rest as a wall
    would.  Lead at rho0 and e = 0 (P = 0), mass rho0 a^3.  The lateral faces
    are free (no periodic images)."""
    ny = periods * lam
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    ym = (j % lam) + 0.5 - lam / 2.0                      # offset from the groove centre, in spacings
    depth = lam / 2.0 - np.abs(ym)                        # V-groove: lam/2 at the centre, 0 at the ridges
    keep = i < nx - depth
    i, j, k = i[keep], j[keep], k[keep]
    x = i * a
    y = (j - (ny - 1) / 2.0) * a
    z = (k - (nz - 1) / 2.0) * a
    n1 = len(x)
    x = np.concatenate([x, -x - a]); y = np.concatenate([y, y]); z = np.concatenate([z, z])
    vx = np.concatenate([np.full(n1, -up), np.full(n1, up)])
    mat = lead()
    n = 2 * n1
    arrays = dict(x=x, y=y, z=z, vx=vx, vy=np.zeros(n), vz=np.zeros(n), rho=np.full(n, mat.rho0),
                  E=0.5 * vx * vx, m=np.full(n, mat.rho0 * a ** 3))
    return Problem(f"ejecta_{n}", 3, arrays, [mat], kernel="cubic", kappa=2.0, eta=1.3, cfl=0.3,
                   n_steps=n_steps, units=units, unit_dim=2, n_upd=10,
                   meta=dict(a=a, up=up, lam=lam, nx=nx, n_half=n1))


def water_block(side: int = 8, a: float = 1e-3, seed: int = 29) -> Problem:
    """A cube of Tait water (rho0 = 1000, c0 = 1500, exponent 7) with a
    seeded random velocity field and +-1 % density perturbations."""
    g = np.meshgrid(*[np.arange(side, dtype=float)] * 3, indexing="ij")
    n = side ** 3
    u = uniform(seed, 4 * n).reshape(4, n)
    x, y, z = (gi.ravel() * a for gi in g)
    rho = 1000.0 * (1.0 + 0.02 * (u[3] - 0.5))
    v = 5.0 * (u[:3] - 0.5)
    arrays = dict(x=x, y=y, z=z, vx=v[0], vy=v[1], vz=v[2], rho=rho,
                  E=2.0e3 + 0.5 * (v ** 2).sum(axis=0), m=np.full(n, 1000.0 * a ** 3))
    mat = MaterialSpec("tait", 7.0, rho0=1000.0, c0=1500.0)
    return Problem(f"water_{n}", 3, arrays, [mat], kernel="cubic", kappa=2.0, eta=1.3, cfl=0.3,
                   n_steps=20, units=0, unit_dim=2, n_upd=10)


def droplets(n_sphere: int = 4_000_000, n_gas: int = 2_000_000, radius: float = 1e-3,
             speed: float = 300.0, gap: float = 5.0, jitter: float = 0.05, seed: int = 2019,
             units: int = 256, n_steps: int = 100) -> Problem:
    """Two Tait water droplets (rho0 = 1000, c0 = 1500, exponent 7) of
    n_sphere particles each and radius `radius`, approaching at relative
    speed `speed`, in an ambient ideal gas (gamma = 1.4) at 1/1000 of the
    water density.  All particles sit on one cubic lattice of spacing
    a = (4/3 pi radius^3 / n_sphere)^(1/3) with seeded +-jitter a offsets, so
    the density contrast is carried by the particle masses (1:1000) and the
    particle sizes d = (m / rho)^(1/3) agree across the interface.  The gas
    fills a shell around each droplet, thick enough for about n_gas gas
    particles in all.  The spheres' surfaces are `gap` spacings apart along x.
    Pressure equilibrium: the gas at 1e5 Pa, the water compressed to the
    same Tait pressure."""
    a = (4.0 / 3.0 * np.pi * radius ** 3 / n_sphere) ** (1.0 / 3.0)
    shell = (n_gas / 2.0) * a ** 3 / (4.0 * np.pi * radius ** 2)      # gas thickness around each sphere
    cx = radius + 0.5 * gap * a
    ext = radius + shell + 2 * a
    nx = int(np.ceil((cx + ext) / a)); ny = int(np.ceil(ext / a))
    i = np.arange(-nx, nx + 1) * a
    j = np.arange(-ny, ny + 1) * a
    X, Y, Z = np.meshgrid(i, j, j, indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    r1 = np.sqrt((X + cx) ** 2 + Y ** 2 + Z ** 2)
    r2 = np.sqrt((X - cx) ** 2 + Y ** 2 + Z ** 2)
    water = (r1 <= radius) | (r2 <= radius)
    gas = ~water & ((r1 <= radius + shell) | (r2 <= radius + shell))
    keep = water | gas
    X, Y, Z, water = X[keep], Y[keep], Z[keep], water[keep]
    n = len(X)
    u = uniform(seed, 3 * n)
    X = X + jitter * a * (2 * u[0::3] - 1)
    Y = Y + jitter * a * (2 * u[1::3] - 1)
    Z = Z + jitter * a * (2 * u[2::3] - 1)
    w_mat = MaterialSpec("tait", 7.0, rho0=1000.0, c0=1500.0)
    g_mat = MaterialSpec("ideal", 1.4)
    p0 = 1e5
    B = w_mat.rho0 * w_mat.c0 ** 2 / w_mat.gamma
    rho_w = w_mat.rho0 * (1.0 + p0 / B) ** (1.0 / w_mat.gamma)
    rho_g = w_mat.rho0 / 1000.0
    e_g = p0 / ((g_mat.gamma - 1.0) * rho_g)
    rho = np.where(water, rho_w, rho_g)
    vx = np.where(water, np.where(X < 0, 0.5 * speed, -0.5 * speed), 0.0)
    e = np.where(water, 0.0, e_g)
    arrays = dict(x=X, y=Y, z=Z, vx=vx, vy=np.zeros(n), vz=np.zeros(n), rho=rho, E=e + 0.5 * vx * vx,
                  m=rho * a ** 3)
    mat = np.where(water, 0, 1).astype(np.int32)
    return Problem(f"droplets_{n}", 3, arrays, [w_mat, g_mat], mat=mat, kernel="cubic", kappa=2.0, eta=1.3,
                   cfl=0.3, n_steps=n_steps, units=units, unit_dim=3, n_upd=10,
                   meta=dict(a=a, radius=radius, shell=shell, n_water=int(water.sum()), n_gas=int((~water).sum())))


# ---------------------------------------------------------------------------
# Voronoi generator seeding
# ---------------------------------------------------------------------------
def _morton_key(q: list) -> np.ndarray:
    """Interleave the bits of 1..3 arrays of 16-bit integers."""
    key = np.zeros(len(q[0]), dtype=np.uint64)
    nd = len(q)
    for b in range(16):
        for a in range(nd):
            bit = (q[a].astype(np.uint64) >> np.uint64(b)) & np.uint64(1)
            key |= bit << np.uint64(b * nd + a)
    return key


def seed_generators(pos: list, K: int) -> np.ndarray:
    """K generators in the space of the given coordinate arrays: particles
    sorted along a Morton curve are cut into K runs of equal count, and each
    generator is placed at the mean position of its run."""
    n = len(pos[0])
    if len(pos) == 1:
        order = np.argsort(pos[0], kind="stable")
    else:
        q = []
        for a in pos:
            lo, hi = float(a.min()), float(a.max())
            span = hi - lo if hi > lo else 1.0
            q.append(np.minimum(((a - lo) / span * 65535.0).astype(np.int64), 65535))
        order = np.argsort(_morton_key(q), kind="stable")
    cuts = np.linspace(0, n, K + 1).astype(np.int64)
    gen = np.zeros((K, len(pos)))
    for k in range(K):
        sel = order[cuts[k]:max(cuts[k + 1], cuts[k] + 1)]
        for a in range(len(pos)):
            gen[k, a] = pos[a][sel].mean()
    return gen


def problem_generators(prob: Problem) -> np.ndarray:
    keys = ("x", "y", "z")[: prob.unit_dim]
    return seed_generators([prob.arrays[k] for k in keys], prob.units)


# ---------------------------------------------------------------------------
# Balancing test geometries (Secs. 5 and 6 of the paper)
# ---------------------------------------------------------------------------
def disk(n_target: int = 127230, radius: float = 0.45, height: float = 0.1) -> dict:
    """Particles on a cubic lattice filling a disk of the given radius and
    height at rest (the three-subdomain convergence test of Sec. 5); the
    lattice spacing is chosen so the count is close to n_target."""
    vol = math.pi * radius ** 2 * height
    a = (vol / n_target) ** (1.0 / 3.0)
    nr = int(math.ceil(radius / a)) + 1
    nz = max(int(round(height / a)), 1)
    g = (np.arange(-nr, nr + 1) + 0.5) * a
    X, Y, Z = np.meshgrid(g, g, (np.arange(nz) + 0.5) * a, indexing="ij")
    keep = X ** 2 + Y ** 2 < radius ** 2
    return dict(x=X[keep].ravel(), y=Y[keep].ravel(), z=Z[keep].ravel(), a=a)


def plate_static(nx: int = 128, ny: int = 128, nz: int = 2, a: float = 1.0 / 128) -> dict:
    """A thin square plate at rest on a cubic lattice (the static test of Sec. 6)."""
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    return dict(x=((i + 0.5) * a).ravel(), y=((j + 0.5) * a).ravel(), z=((k + 0.5) * a).ravel(), a=a)
