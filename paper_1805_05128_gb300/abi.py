"""ctypes view of the C ABI declared in include/csph.h (argument marshalling only).

Every function here has the name of the C entry point it calls and forwards
its arguments unchanged; all computation happens in libcsph.so.  Loading
fails loudly if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_PKG, "libcsph.so")

SPH_OK, SPH_ERR_INVALID, SPH_ERR_CAPACITY, SPH_ERR_NONFINITE, SPH_ERR_CUDA, SPH_ERR_TIMEOUT = range(6)
SPH_KERNEL_CUBIC, SPH_KERNEL_WENDLAND_C2 = 0, 1
SPH_EOS_IDEAL, SPH_EOS_STIFFENED, SPH_EOS_TAIT, SPH_EOS_MIE_GRUNEISEN, SPH_EOS_STIFFENED_C0 = 0, 1, 2, 3, 4
SPH_PREC_FP64, SPH_PREC_MIXED = 0, 1
SPH_SOLVER_ACOUSTIC, SPH_SOLVER_HLL = 0, 1
SPH_LOAD_PAIRS, SPH_LOAD_TIME = 0, 1
SPH_SCHED_GLOBAL, SPH_SCHED_UNITS, SPH_SCHED_UNITS_OWNED = 0, 1, 2
SPH_MAX_MAT, SPH_MAX_UNITS = 4, 256

ERROR_NAMES = {0: "SPH_OK", 1: "SPH_ERR_INVALID", 2: "SPH_ERR_CAPACITY", 3: "SPH_ERR_NONFINITE",
               4: "SPH_ERR_CUDA", 5: "SPH_ERR_TIMEOUT"}

# every symbol include/csph.h declares
EXPORTS = ("sph_init", "sph_build_cells", "sph_eval_rates", "sph_step", "voronoi_assign", "voronoi_balance",
           "sph_conservation", "sph_unit_stats", "sph_read_status", "sph_last_error", "sph_pair_counts",
           "sph_cell_index", "sph_pair_list", "voronoi_assign_static", "sph_profile", "sph_profile_read",
           "sph_step_adjoint", "sph_last_dt", "sph_step_dt", "sph_list_builds", "sph_unit_times", "sph_cfl_dt", "sph_hold_rates",
           "voronoi_balance_stats", "sph_destroy")


class sph_material(C.Structure):
    _fields_ = [("eos", C.c_int32), ("pad_", C.c_int32), ("gamma", C.c_double), ("rho0", C.c_double),
                ("c0", C.c_double), ("p_inf", C.c_double), ("s_a", C.c_double)]


class sph_params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("kernel", C.c_int32), ("precision", C.c_int32), ("n_mat", C.c_int32),
                ("kappa", C.c_double), ("eta", C.c_double), ("cfl", C.c_double), ("cell_beta", C.c_double),
                ("cell_cap", C.c_int64), ("mat", sph_material * SPH_MAX_MAT),
                ("n_units", C.c_int32), ("unit_dim", C.c_int32), ("n_upd", C.c_int32), ("pair_blocks_per_sm", C.c_int32),
                ("theta", C.c_double), ("sigma", C.c_double), ("gamma_b", C.c_double), ("beta_sh", C.c_double),
                ("generators", C.c_void_p), ("materials", C.c_void_p),
                ("order", C.c_int32), ("solver", C.c_int32),
                ("load_measure", C.c_int32), ("list_cap", C.c_int32),
                ("unit_sched", C.c_int32), ("list_staging", C.c_int32)]


STATE_F64 = ("x", "y", "z", "vx", "vy", "vz", "rho", "E", "m")
STATE_RATES = ("ax", "ay", "az", "drho", "dE")
STATE_DERIVED = ("d", "P", "c")


class sph_state(C.Structure):
    _fields_ = ([("n", C.c_int64)] + [(k, C.c_void_p) for k in STATE_F64] + [("mat", C.c_void_p)]
                + [(k, C.c_void_p) for k in STATE_RATES + STATE_DERIVED] + [("id", C.c_void_p),
                                                                              ("unit", C.c_void_p)])


class sph_ckpt(C.Structure):
    _fields_ = [("state", sph_state), ("dt", C.c_void_p), ("rates_from_state", C.c_int32), ("reverse_fp64", C.c_int32)]


class sph_balance_params(C.Structure):
    _fields_ = [("theta", C.c_double), ("sigma", C.c_double), ("gamma_b", C.c_double), ("beta_sh", C.c_double)]


_lib = None


def lib() -> C.CDLL:
    """Load libcsph.so.  Raises if it is missing (build it with
    ``python -c "import __graft_entry__ as g; g.build()"``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(SO_PATH):
        raise RuntimeError(f"libcsph.so not built ({SO_PATH}); run paper_1805_05128_gb300.build.build()")
    L = C.CDLL(SO_PATH)
    vp, i32, i64 = C.c_void_p, C.c_int, C.c_int64
    L.sph_init.argtypes = [C.POINTER(vp), C.POINTER(sph_params), i32, C.POINTER(C.c_int64),
                           C.POINTER(sph_state), vp]
    L.sph_build_cells.argtypes = [vp, C.POINTER(sph_state), vp]
    L.sph_eval_rates.argtypes = [vp, C.POINTER(sph_state), vp]
    L.sph_step.argtypes = [vp, C.POINTER(sph_state), i32, vp, vp]
    L.voronoi_assign.argtypes = [vp, C.POINTER(sph_state), vp, i32, i32, vp, vp, vp]
    L.voronoi_balance.argtypes = [vp, C.POINTER(sph_state), vp, i32, i32, vp, C.POINTER(sph_balance_params),
                                  vp, vp]
    L.sph_conservation.argtypes = [vp, C.POINTER(sph_state), vp, vp]
    L.sph_unit_stats.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_uint8), vp]
    L.sph_read_status.argtypes = [vp, C.POINTER(C.c_int)]
    L.sph_last_error.argtypes = [vp]
    L.sph_last_error.restype = C.c_char_p
    L.sph_pair_counts.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64), vp]
    L.sph_cell_index.argtypes = [vp, C.POINTER(sph_state), vp, C.POINTER(C.c_double), vp]
    L.sph_pair_list.argtypes = [vp, C.POINTER(sph_state), i64, vp, vp, C.POINTER(C.c_int64), vp]
    L.voronoi_assign_static.argtypes = [i64, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp]
    L.sph_step_adjoint.argtypes = [vp, C.POINTER(sph_ckpt), i32, C.POINTER(sph_state), C.POINTER(sph_state), vp, vp]
    L.sph_last_dt.argtypes = [vp, vp, vp]
    L.sph_step_dt.argtypes = [vp, C.POINTER(sph_state), i32, vp, vp, vp]
    L.sph_list_builds.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32), vp]
    L.sph_unit_times.argtypes = [vp, C.POINTER(C.c_double), vp]
    L.sph_cfl_dt.argtypes = [vp, C.POINTER(sph_state), vp, vp]
    L.sph_hold_rates.argtypes = [vp]
    dp = C.POINTER(C.c_double)
    L.voronoi_balance_stats.argtypes = [vp, vp, i32, i32, dp, C.POINTER(C.c_uint8), dp, dp, C.POINTER(C.c_int64),
                                        C.POINTER(sph_balance_params), vp, vp]
    L.sph_profile.argtypes = [vp, i32]
    L.sph_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.sph_destroy.argtypes = [vp]
    L.sph_destroy.restype = None
    for name in EXPORTS:
        if name not in ("sph_last_error", "sph_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


class CsphError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code: int, handle=None):
    if code != SPH_OK:
        msg = lib().sph_last_error(handle)
        raise CsphError(code, msg.decode() if msg else "")


# thin same-name wrappers ----------------------------------------------------
def sph_init(params: sph_params, n_instances: int, inst_offsets, state: sph_state, stream: int):
    h = C.c_void_p()
    offs = (C.c_int64 * (n_instances + 1))(*inst_offsets)
    check(lib().sph_init(C.byref(h), C.byref(params), n_instances, offs, C.byref(state), C.c_void_p(stream)))
    return h


def sph_build_cells(h, state, stream):
    check(lib().sph_build_cells(h, C.byref(state), C.c_void_p(stream)), h)


def sph_eval_rates(h, state, stream):
    check(lib().sph_eval_rates(h, C.byref(state), C.c_void_p(stream)), h)


def sph_step(h, state, n_steps, t_dev_ptr, stream):
    check(lib().sph_step(h, C.byref(state), n_steps, C.c_void_p(t_dev_ptr), C.c_void_p(stream)), h)


def voronoi_assign(h, state, gen_ptr, K, dim, unit_out_ptr, unit_offsets_ptr, stream):
    check(lib().voronoi_assign(h, C.byref(state), C.c_void_p(gen_ptr), K, dim, C.c_void_p(unit_out_ptr),
                               C.c_void_p(unit_offsets_ptr), C.c_void_p(stream)), h)


def voronoi_balance(h, state, gen_ptr, K, dim, load_ptr, bp: sph_balance_params, shift_ptr, stream):
    check(lib().voronoi_balance(h, C.byref(state), C.c_void_p(gen_ptr), K, dim, C.c_void_p(load_ptr),
                                C.byref(bp), C.c_void_p(shift_ptr), C.c_void_p(stream)), h)


def sph_conservation(h, state, out_ptr, stream):
    check(lib().sph_conservation(h, C.byref(state), C.c_void_p(out_ptr), C.c_void_p(stream)), h)


def sph_unit_stats(h, load_out, adj_out, stream):
    check(lib().sph_unit_stats(h, load_out, adj_out, C.c_void_p(stream)), h)


def sph_read_status(h) -> int:
    st = C.c_int(0)
    check(lib().sph_read_status(h, C.byref(st)), h)
    return st.value


def sph_last_error(h) -> str:
    m = lib().sph_last_error(h)
    return m.decode() if m else ""


def sph_pair_counts(h, stream):
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    check(lib().sph_pair_counts(h, C.byref(a), C.byref(b), C.byref(c), C.c_void_p(stream)), h)
    return a.value, b.value, c.value


def sph_list_builds(h, stream):
    """(Verlet-list builds since sph_init, list capacity per particle)."""
    b, c = C.c_int64(), C.c_int32()
    check(lib().sph_list_builds(h, C.byref(b), C.byref(c), C.c_void_p(stream)), h)
    return b.value, c.value


def sph_unit_times(h, out, stream):
    """out: host float64 array of 2 K (start, end per unit, ns)."""
    check(lib().sph_unit_times(h, out.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(stream)), h)


def sph_hold_rates(h):
    check(lib().sph_hold_rates(h), h)


def sph_cfl_dt(h, state, dt_out_ptr, stream):
    check(lib().sph_cfl_dt(h, C.byref(state), C.c_void_p(dt_out_ptr), C.c_void_p(stream)), h)


def voronoi_balance_stats(h, gen_ptr, K, dim, load, adj, rmax, centroid, count, bp: sph_balance_params,
                          shift_ptr, stream):
    """load, rmax (K), centroid (K x dim) float64, adj (K x K) uint8, count (K) int64: host numpy arrays."""
    dp = C.POINTER(C.c_double)
    check(lib().voronoi_balance_stats(h, C.c_void_p(gen_ptr), K, dim, load.ctypes.data_as(dp),
                                      adj.ctypes.data_as(C.POINTER(C.c_uint8)), rmax.ctypes.data_as(dp),
                                      centroid.ctypes.data_as(dp), count.ctypes.data_as(C.POINTER(C.c_int64)),
                                      C.byref(bp), C.c_void_p(shift_ptr), C.c_void_p(stream)), h)


def sph_cell_index(h, state, cell_out_ptr, grid_out, stream):
    check(lib().sph_cell_index(h, C.byref(state), C.c_void_p(cell_out_ptr), grid_out, C.c_void_p(stream)), h)


def sph_pair_list(h, state, cap, pi_ptr, pj_ptr, stream) -> int:
    cnt = C.c_int64(0)
    check(lib().sph_pair_list(h, C.byref(state), cap, C.c_void_p(pi_ptr), C.c_void_p(pj_ptr), C.byref(cnt),
                              C.c_void_p(stream)), h)
    return cnt.value


def voronoi_assign_static(n, x_ptr, y_ptr, z_ptr, gen_ptr, K, dim, unit_out_ptr, unit_offsets_ptr,
                          unit_list_ptr, stream):
    """Allocation-free voronoi_assign (no handle); see include/csph.h."""
    check(lib().voronoi_assign_static(n, C.c_void_p(x_ptr), C.c_void_p(y_ptr), C.c_void_p(z_ptr),
                                      C.c_void_p(gen_ptr), K, dim, C.c_void_p(unit_out_ptr),
                                      C.c_void_p(unit_offsets_ptr), C.c_void_p(unit_list_ptr),
                                      C.c_void_p(stream)))


def sph_step_adjoint(h, ckpt: sph_ckpt, n_steps, adj_out: sph_state, adj_in: sph_state, params_ptr, stream):
    check(lib().sph_step_adjoint(h, C.byref(ckpt), n_steps, C.byref(adj_out), C.byref(adj_in),
                                 C.c_void_p(params_ptr), C.c_void_p(stream)), h)


def sph_last_dt(h, dt_out_ptr, stream):
    check(lib().sph_last_dt(h, C.c_void_p(dt_out_ptr), C.c_void_p(stream)), h)


def sph_step_dt(h, state, n_steps, dt_ptr, t_dev_ptr, stream):
    check(lib().sph_step_dt(h, C.byref(state), n_steps, C.c_void_p(dt_ptr), C.c_void_p(t_dev_ptr),
                            C.c_void_p(stream)), h)


def sph_profile(h, enable: bool):
    check(lib().sph_profile(h, int(enable)), h)


def sph_profile_read(h):
    ms, npair, nk = C.c_double(), C.c_int64(), C.c_int64()
    check(lib().sph_profile_read(h, C.byref(ms), C.byref(npair), C.byref(nk)), h)
    return ms.value, npair.value, nk.value


def sph_destroy(h):
    lib().sph_destroy(h)
