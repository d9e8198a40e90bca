"""Plain FP64 CPU oracle for the CSPH + VD3 hot path (arXiv 1805.05128).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product package never does.  The arithmetic lives in
``csph_oracle.c`` (single-threaded FP64, ``-ffp-contract=off``); this module
only builds it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csph_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")

KERNEL_CUBIC, KERNEL_WENDLAND_C2 = 0, 1
EOS_IDEAL, EOS_STIFFENED, EOS_TAIT, EOS_MIE_GRUNEISEN = 0, 1, 2, 3
SOLVER_ACOUSTIC, SOLVER_HLL = 0, 1
MAX_MAT = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, FP64, no contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    hdr = os.path.join(_HERE, "csph_oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Material(C.Structure):
    _fields_ = [("eos", C.c_int), ("gamma", C.c_double), ("rho0", C.c_double),
                ("c0", C.c_double), ("p_inf", C.c_double), ("s_a", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("dim", C.c_int), ("kernel", C.c_int), ("kappa", C.c_double),
                ("eta", C.c_double), ("cfl", C.c_double), ("cell_beta", C.c_double),
                ("cell_cap", C.c_int64), ("n_mat", C.c_int), ("mat", _Material * MAX_MAT),
                ("order", C.c_int), ("solver", C.c_int)]


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)


class _State(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, _DP) for k in
                                     ("x", "y", "z", "vx", "vy", "vz", "rho", "E", "m")] + \
               [("mat", _IP)] + [(k, _DP) for k in ("ax", "ay", "az", "drho", "dE", "d", "P", "c")]


class _Grid(C.Structure):
    _fields_ = [("x0", C.c_double * 3), ("dc", C.c_double), ("inv_dc", C.c_double),
                ("dims", C.c_int64 * 3), ("ncells", C.c_int64)]


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_kernel_w.restype = C.c_double
        L.orc_kernel_w.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]
        L.orc_kernel_dw.restype = C.c_double
        L.orc_kernel_dw.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]
        L.orc_eos.restype = C.c_int
        L.orc_eos.argtypes = [C.POINTER(_Material), C.c_double, C.c_double, _DP, _DP]
        L.orc_riemann_acoustic.restype = None
        L.orc_riemann_acoustic.argtypes = [C.c_double] * 6 + [_DP, _DP]
        L.orc_derive.restype = C.c_int64
        L.orc_derive.argtypes = [C.POINTER(_Params), C.POINTER(_State)]
        L.orc_dt.restype = C.c_double
        L.orc_dt.argtypes = [C.POINTER(_Params), C.POINTER(_State)]
        L.orc_cell_grid.restype = C.c_int
        L.orc_cell_grid.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.POINTER(_Grid),
                                    C.POINTER(C.c_int64)]
        for f in (L.orc_pairs_brute, L.orc_pairs_cells):
            f.restype = C.c_int64
            f.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.c_int64, _IP, _IP]
        L.orc_rates.restype = None
        L.orc_rates.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.c_int64, _IP, _IP]
        L.orc_eval_rates.restype = C.c_int64
        L.orc_eval_rates.argtypes = [C.POINTER(_Params), C.POINTER(_State)]
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.c_int, C.c_int, _DP, _DP]
        L.orc_conservation.restype = None
        L.orc_conservation.argtypes = [C.POINTER(_State), _DP]
        L.orc_voronoi_assign.restype = None
        L.orc_voronoi_assign.argtypes = [C.c_int64, C.c_int, _DP, _DP, _DP, C.c_int, _DP, _IP]
        L.orc_unit_stats.restype = C.c_int
        L.orc_unit_stats.argtypes = [C.POINTER(_Params), C.POINTER(_State), _IP, C.c_int, C.c_int,
                                     C.c_int64, _IP, _IP, C.c_double, _DP,
                                     C.POINTER(C.c_uint8), _DP, _DP, C.POINTER(C.c_int64)]
        L.orc_balance.restype = C.c_double
        L.orc_balance.argtypes = [C.c_int, C.c_int, _DP, _DP, C.POINTER(C.c_uint8), _DP, _DP,
                                  C.POINTER(C.c_int64), C.c_double, C.c_double, C.c_double, _DP]
    return _lib


# --------------------------------------------------------------------------
# numpy-facing wrappers
# --------------------------------------------------------------------------
@dataclass
class Material:
    eos: int = EOS_IDEAL
    gamma: float = 1.4
    rho0: float = 1.0
    c0: float = 1.0
    p_inf: float = 0.0
    s_a: float = 0.0


@dataclass
class Params:
    dim: int = 3
    kernel: int = KERNEL_CUBIC
    kappa: float = 2.0
    eta: float = 1.3
    cfl: float = 0.3
    cell_beta: float = 0.0
    cell_cap: int = 1 << 26
    materials: list = field(default_factory=lambda: [Material()])
    order: int = 1              # 2: states reconstructed to the pair midpoint (see orc_rates)
    solver: int = 0             # 0: acoustic, 1: HLL with Davis wave speeds (see orc_riemann_hll)

    def cs(self) -> _Params:
        p = _Params()
        p.dim, p.kernel, p.kappa, p.eta, p.cfl = self.dim, self.kernel, self.kappa, self.eta, self.cfl
        p.cell_beta, p.cell_cap, p.n_mat = self.cell_beta, self.cell_cap, len(self.materials)
        p.order = self.order
        p.solver = self.solver
        for i, m in enumerate(self.materials):
            p.mat[i].eos, p.mat[i].gamma, p.mat[i].rho0 = m.eos, m.gamma, m.rho0
            p.mat[i].c0, p.mat[i].p_inf, p.mat[i].s_a = m.c0, m.p_inf, m.s_a
        return p


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


class State:
    """Host SoA particle state (float64 numpy arrays) viewed by the oracle."""

    FIELDS = ("x", "y", "z", "vx", "vy", "vz", "rho", "E", "m")
    DERIVED = ("ax", "ay", "az", "drho", "dE", "d", "P", "c")

    def __init__(self, dim: int, arrays: dict, mat=None):
        self.dim = dim
        n = len(arrays["x"])
        self.n = n
        for k in self.FIELDS:
            a = arrays.get(k)
            if a is None and k in ("y", "z", "vy", "vz"):
                axis = "xyz".index(k[-1])
                if axis >= dim:
                    setattr(self, k, None)
                    continue
                a = np.zeros(n)
            setattr(self, k, np.ascontiguousarray(np.asarray(a, dtype=np.float64)).copy())
        self.mat = None if mat is None else np.ascontiguousarray(np.asarray(mat, dtype=np.int32))
        for k in self.DERIVED:
            if k in ("ay", "az") and "xyz".index(k[-1]) >= dim:
                setattr(self, k, None)
            else:
                src = arrays.get(k)
                setattr(self, k, np.zeros(n) if src is None
                        else np.ascontiguousarray(np.asarray(src, dtype=np.float64)).copy())

    def cs(self) -> _State:
        s = _State()
        s.n = self.n
        for k in self.FIELDS + self.DERIVED:
            setattr(s, k, _dp(getattr(self, k)))
        s.mat = None if self.mat is None else self.mat.ctypes.data_as(_IP)
        return s

    def copy(self) -> "State":
        arrays = {k: getattr(self, k) for k in self.FIELDS + self.DERIVED if getattr(self, k) is not None}
        return State(self.dim, arrays, self.mat)

    def pos(self):
        return [getattr(self, k) for k in ("x", "y", "z")[: self.dim]]


def kernel_w(kernel, dim, kappa, r, h):
    return lib().orc_kernel_w(kernel, dim, kappa, r, h)


def kernel_dw(kernel, dim, kappa, r, h):
    return lib().orc_kernel_dw(kernel, dim, kappa, r, h)


def eos(mat: Material, rho: float, e: float):
    m = Params(materials=[mat]).cs().mat[0]
    P, c = C.c_double(), C.c_double()
    bad = lib().orc_eos(C.byref(m), rho, e, C.byref(P), C.byref(c))
    return P.value, c.value, bad


def riemann_acoustic(Pi, Pj, Zi, Zj, vRi, vRj):
    P, v = C.c_double(), C.c_double()
    lib().orc_riemann_acoustic(Pi, Pj, Zi, Zj, vRi, vRj, C.byref(P), C.byref(v))
    return P.value, v.value


def riemann_hll(Pi, Pj, Zi, Zj, vRi, vRj):
    L = lib()
    L.orc_riemann_hll.restype = None
    L.orc_riemann_hll.argtypes = [C.c_double] * 6 + [_DP, _DP]
    P, v = C.c_double(), C.c_double()
    L.orc_riemann_hll(Pi, Pj, Zi, Zj, vRi, vRj, C.byref(P), C.byref(v))
    return P.value, v.value


def derive(p: Params, s: State) -> int:
    pc, sc = p.cs(), s.cs()
    return lib().orc_derive(C.byref(pc), C.byref(sc))


def dt(p: Params, s: State) -> float:
    pc, sc = p.cs(), s.cs()
    return lib().orc_dt(C.byref(pc), C.byref(sc))


def cell_grid(p: Params, s: State):
    pc, sc, g = p.cs(), s.cs(), _Grid()
    cells = np.zeros(max(s.n, 1), dtype=np.int64)
    rc = lib().orc_cell_grid(C.byref(pc), C.byref(sc), C.byref(g), cells.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc != 0:
        raise ValueError("oracle cell grid failed")
    return dict(x0=np.array(g.x0[:]), dc=g.dc, inv_dc=g.inv_dc, dims=np.array(g.dims[:]),
                ncells=g.ncells), cells[: s.n]


def pairs(p: Params, s: State, method: str = "cells"):
    """Unordered interacting pairs (i < j) as two int32 arrays, sorted."""
    f = lib().orc_pairs_cells if method == "cells" else lib().orc_pairs_brute
    pc, sc = p.cs(), s.cs()
    n = f(C.byref(pc), C.byref(sc), 0, None, None)
    if n < 0:
        raise ValueError("oracle pair search failed")
    pi = np.zeros(max(n, 1), dtype=np.int32)
    pj = np.zeros(max(n, 1), dtype=np.int32)
    f(C.byref(pc), C.byref(sc), n, pi.ctypes.data_as(_IP), pj.ctypes.data_as(_IP))
    pi, pj = pi[:n], pj[:n]
    order = np.lexsort((pj, pi))
    return pi[order], pj[order]


def rates(p: Params, s: State, pi, pj):
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    pc, sc = p.cs(), s.cs()
    lib().orc_rates(C.byref(pc), C.byref(sc), len(pi), pi.ctypes.data_as(_IP), pj.ctypes.data_as(_IP))


def pair_gradients(p: Params, s: State):
    """SPH gradients of P and v used by the order-2 reconstruction, at the
    state's d and P (call derive first): (n, 3) and (n, 3, 3) arrays,
    gV[i, a, b] = d v_a / d x_b."""
    pi, pj = pairs(p, s)
    n = s.n
    gP = np.zeros(3 * n)
    gV = np.zeros(9 * n)
    pc, sc = p.cs(), s.cs()
    L = lib()
    L.orc_pair_gradients.restype = None
    L.orc_pair_gradients(C.byref(pc), C.byref(sc), C.c_int64(len(pi)), pi.ctypes.data_as(_IP),
                         pj.ctypes.data_as(_IP), _dp(gP), _dp(gV))
    return gP.reshape(n, 3), gV.reshape(n, 3, 3)


def eval_rates(p: Params, s: State) -> int:
    pc, sc = p.cs(), s.cs()
    n = lib().orc_eval_rates(C.byref(pc), C.byref(sc))
    if n < 0:
        raise ValueError("oracle rate evaluation failed")
    return n


def step(p: Params, s: State, n_steps: int, rates_valid: bool = False, t: float = 0.0):
    """Advance ``s`` in place by n_steps KDK steps; returns (t, dt per step)."""
    pc, sc = p.cs(), s.cs()
    tt = C.c_double(t)
    dts = np.zeros(max(n_steps, 1))
    rc = lib().orc_step(C.byref(pc), C.byref(sc), n_steps, int(rates_valid), C.byref(tt), _dp(dts))
    if rc != 0:
        raise ValueError("oracle step failed")
    return tt.value, dts[:n_steps]


def conservation(s: State):
    out = np.zeros(5)
    sc = s.cs()
    lib().orc_conservation(C.byref(sc), _dp(out))
    return out


def voronoi_assign(pos, gen):
    """pos: list of gdim coordinate arrays; gen: (K, gdim) array."""
    gen = np.ascontiguousarray(gen, dtype=np.float64)
    K, gdim = gen.shape
    n = len(pos[0])
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in pos]
    while len(arrs) < 3:
        arrs.append(None)
    unit = np.zeros(max(n, 1), dtype=np.int32)
    lib().orc_voronoi_assign(n, gdim, _dp(arrs[0]), _dp(arrs[1]), _dp(arrs[2]), K, _dp(gen),
                             unit.ctypes.data_as(_IP))
    return unit[:n]


def unit_stats(p: Params, s: State, unit, K: int, gdim: int, pi, pj, beta: float):
    unit = np.ascontiguousarray(unit, dtype=np.int32)
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    load = np.zeros(K)
    adj = np.zeros((K, K), dtype=np.uint8)
    dsh = np.zeros((K, K))
    cen = np.zeros((K, gdim))
    cnt = np.zeros(K, dtype=np.int64)
    pc, sc = p.cs(), s.cs()
    lib().orc_unit_stats(C.byref(pc), C.byref(sc), unit.ctypes.data_as(_IP), K, gdim, len(pi),
                         pi.ctypes.data_as(_IP), pj.ctypes.data_as(_IP), beta, _dp(load),
                         adj.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(dsh), _dp(cen),
                         cnt.ctypes.data_as(C.POINTER(C.c_int64)))
    return dict(load=load, adj=adj, dsh=dsh, centroid=cen, count=cnt)


def balance(gen, load, adj, dsh, centroid, count, theta=0.25, sigma=0.5, gamma_b=1.0):
    """One VD3 generator update; returns (new generators, shift sum, dg)."""
    g = np.ascontiguousarray(gen, dtype=np.float64).copy()
    K, gdim = g.shape
    load = np.ascontiguousarray(load, dtype=np.float64)
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    dsh = np.ascontiguousarray(dsh, dtype=np.float64)
    cen = np.ascontiguousarray(centroid, dtype=np.float64)
    cnt = np.ascontiguousarray(count, dtype=np.int64)
    dg = np.zeros_like(g)
    shift = lib().orc_balance(K, gdim, _dp(g), _dp(load), adj.ctypes.data_as(C.POINTER(C.c_uint8)),
                              _dp(dsh), _dp(cen), cnt.ctypes.data_as(C.POINTER(C.c_int64)),
                              theta, sigma, gamma_b, _dp(dg))
    return g, shift, dg


# --------------------------------------------------------------------------
# Problem (synthetic input) -> oracle parameters and state
# --------------------------------------------------------------------------
_EOS_IDS = {"ideal": EOS_IDEAL, "stiffened": EOS_STIFFENED, "tait": EOS_TAIT,
            "mie_gruneisen": EOS_MIE_GRUNEISEN}
_KERNEL_IDS = {"cubic": KERNEL_CUBIC, "wendland_c2": KERNEL_WENDLAND_C2}


def from_problem(prob, cell_cap: int = 1 << 26, order: int = 1, solver: int = 0):
    """Oracle Params and State for a ``synth.Problem``."""
    mats = [Material(_EOS_IDS[m.eos], m.gamma, m.rho0, m.c0, m.p_inf, m.s_a) for m in prob.materials]
    p = Params(dim=prob.dim, kernel=_KERNEL_IDS[prob.kernel], kappa=prob.kappa, eta=prob.eta,
               cfl=prob.cfl, cell_beta=0.0, cell_cap=cell_cap, materials=mats, order=order, solver=solver)
    return p, State(prob.dim, prob.arrays, prob.mat)


# --------------------------------------------------------------------------
# Reverse mode (hand-derived adjoint, pair set and dt held fixed)
# --------------------------------------------------------------------------
def _bind_adjoint():
    L = lib()
    if getattr(L, "_adj_bound", False):
        return L
    L.orc_rates_vjp.restype = C.c_int
    L.orc_rates_vjp.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.c_int64, _IP, _IP,
                                _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP]
    L.orc_step_replay.restype = C.c_int
    L.orc_step_replay.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.c_int, C.c_int, _DP]
    L.orc_step_vjp.restype = C.c_int
    L.orc_step_vjp.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.c_double] + [_DP] * 8
    L._adj_bound = True
    return L


def rates_vjp(p: Params, s: State, pi, pj, ga, gr, gE):
    """dL/d(x, v, rho, E, c0, gamma) for L = <ga, a> + <gr, drho> + <gE, dE> of
    the rates over the pair list (s carries d, P, c from derive)."""
    L = _bind_adjoint()
    n = s.n
    ga = np.ascontiguousarray(ga, dtype=np.float64).reshape(n, 3)
    out = dict(bx=np.zeros((n, 3)), bv=np.zeros((n, 3)), brho=np.zeros(n), bE=np.zeros(n), bpar=np.zeros(2))
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    pc, sc = p.cs(), s.cs()
    gr = np.ascontiguousarray(gr, dtype=np.float64)
    gE = np.ascontiguousarray(gE, dtype=np.float64)
    rc = L.orc_rates_vjp(C.byref(pc), C.byref(sc), len(pi), pi.ctypes.data_as(_IP), pj.ctypes.data_as(_IP),
                         _dp(ga), _dp(gr), _dp(gE), _dp(out["bx"]), _dp(out["bv"]), _dp(out["brho"]),
                         _dp(out["bE"]), _dp(out["bpar"]))
    if rc != 0:
        raise ValueError("oracle rates VJP supports the first-order scheme, cubic kernel, ideal/stiffened gas")
    return out


def step_replay(p: Params, s: State, dts, rates_valid: bool = True):
    L = _bind_adjoint()
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    pc, sc = p.cs(), s.cs()
    if L.orc_step_replay(C.byref(pc), C.byref(sc), len(dts), int(rates_valid), _dp(dts)) != 0:
        raise ValueError("oracle replay failed")


ADJ_KEYS = ("x", "v", "rho", "E", "a", "drho", "dE")


def zero_adjoint(n: int) -> dict:
    return dict(x=np.zeros((n, 3)), v=np.zeros((n, 3)), rho=np.zeros(n), E=np.zeros(n),
                a=np.zeros((n, 3)), drho=np.zeros(n), dE=np.zeros(n))


def step_vjp(p: Params, s: State, dt: float, y: dict, bpar) -> None:
    """In place: y (adjoint of the state after one step from s with this dt)
    becomes the adjoint of s; bpar (2) accumulates dL/d(c0, gamma)."""
    L = _bind_adjoint()
    for k in ADJ_KEYS:
        y[k] = np.ascontiguousarray(y[k], dtype=np.float64)
    pc, sc = p.cs(), s.cs()
    rc = L.orc_step_vjp(C.byref(pc), C.byref(sc), dt, _dp(y["x"]), _dp(y["v"]), _dp(y["rho"]), _dp(y["E"]),
                        _dp(y["a"]), _dp(y["drho"]), _dp(y["dE"]), _dp(bpar))
    if rc != 0:
        raise ValueError("oracle step VJP failed")


def state_vectors(s: State):
    """(n, 3) views of positions, velocities and accelerations (zeros for unused axes)."""
    n = s.n
    z = np.zeros(n)
    pos = np.stack([s.x, s.y if s.y is not None else z, s.z if s.z is not None else z], axis=1)
    vel = np.stack([s.vx, s.vy if s.vy is not None else z, s.vz if s.vz is not None else z], axis=1)
    acc = np.stack([s.ax, s.ay if s.ay is not None else z, s.az if s.az is not None else z], axis=1)
    return pos, vel, acc


def trajectory_vjp(p: Params, s0: State, dts, y_final: dict):
    """Adjoint of a whole run from s0 with the recorded dt sequence: returns
    (adjoint of the initial state before its first rate evaluation, i.e. of
    x, v, rho, E, and dL/d(c0, gamma) through the EOS).  Stores every state."""
    states = []
    s = s0.copy()
    eval_rates(p, s)
    for dt in dts:
        states.append(s.copy())
        step_replay(p, s, [dt], rates_valid=True)
    y = {k: np.array(v, dtype=np.float64, copy=True) for k, v in y_final.items()}
    bpar = np.zeros(2)
    for st, dt in zip(reversed(states), reversed(list(dts))):
        step_vjp(p, st, dt, y, bpar)
    # the first held rates were evaluated at s0: push their adjoint into s0
    s = s0.copy()
    derive(p, s)
    pi, pj = pairs(p, s)
    r = rates_vjp(p, s, pi, pj, y["a"], y["drho"], y["dE"])
    out = dict(x=y["x"] + r["bx"], v=y["v"] + r["bv"], rho=y["rho"] + r["brho"], E=y["E"] + r["bE"])
    return out, bpar + r["bpar"]
