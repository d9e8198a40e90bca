"""Simulation: torch device tensors for the particle state plus a libcsph
handle.  Torch provides device memory and the stream; every step of the hot
path runs in the CUDA kernels behind the C ABI."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import abi

_EOS = {"ideal": abi.SPH_EOS_IDEAL, "stiffened": abi.SPH_EOS_STIFFENED, "tait": abi.SPH_EOS_TAIT,
        "mie_gruneisen": abi.SPH_EOS_MIE_GRUNEISEN, "stiffened_c0": abi.SPH_EOS_STIFFENED_C0}
_KERNEL = {"cubic": abi.SPH_KERNEL_CUBIC, "wendland_c2": abi.SPH_KERNEL_WENDLAND_C2}
_PREC = {"fp64": abi.SPH_PREC_FP64, "mixed": abi.SPH_PREC_MIXED}
_SOLVER = {"acoustic": abi.SPH_SOLVER_ACOUSTIC, "hll": abi.SPH_SOLVER_HLL}
_LOAD = {"pairs": abi.SPH_LOAD_PAIRS, "time": abi.SPH_LOAD_TIME}
_SCHED = {"global": abi.SPH_SCHED_GLOBAL, "units": abi.SPH_SCHED_UNITS, "units_owned": abi.SPH_SCHED_UNITS_OWNED}


def _stream_ptr() -> int:
    return torch.cuda.current_stream().cuda_stream


class Simulation:
    """One or more independent CSPH instances on one GPU.

    ``problems``: objects with the attributes of ``synth.Problem`` (dim,
    arrays, materials, mat, kernel, kappa, eta, cfl, units, unit_dim, n_upd);
    several problems become instances of one handle (same parameters)."""

    def __init__(self, problems, precision: str = "mixed", units: int | None = None,
                 generators=None, n_upd: int | None = None, theta: float = 0.25, sigma: float = 0.5,
                 gamma_b: float = 1.0, beta_sh: float = 0.45, cell_cap: int = 1 << 24, cell_beta: float = 0.0,
                 pair_blocks_per_sm: int = 0, order: int = 1, solver: str = "acoustic",
                 load_measure: str = "pairs", list_cap: int = 0, unit_sched: str = "global",
                 list_staging: bool = False,
                 device: str | torch.device = "cuda:0"):
        if not isinstance(problems, (list, tuple)):
            problems = [problems]
        self.device = torch.device(device)
        p0 = problems[0]
        self.dim = p0.dim
        self.n_inst = len(problems)
        sizes = [len(q.arrays["x"]) for q in problems]
        self.inst_offsets = [0] + list(np.cumsum(sizes))
        self.n = int(self.inst_offsets[-1])
        dev = self.device
        f64 = dict(dtype=torch.float64, device=dev)
        self.t = {}
        for k in abi.STATE_F64 + abi.STATE_RATES + abi.STATE_DERIVED:
            axis = "xyz".index(k[-1]) if k in ("y", "z", "vy", "vz", "ay", "az") else -1
            if axis >= self.dim:
                self.t[k] = None
                continue
            if k in abi.STATE_F64:
                vals = [np.asarray(q.arrays.get(k, np.zeros(len(q.arrays["x"]))), dtype=np.float64) for q in problems]
                self.t[k] = torch.from_numpy(np.concatenate(vals)).to(**f64).contiguous()
            else:
                self.t[k] = torch.zeros(self.n, **f64)
        # material table: the problems' materials in order; each particle's index is offset
        # by the materials of the problems before it (one table even when every instance has
        # its own EOS parameters)
        self.materials, mats = [], []
        for q in problems:
            base = len(self.materials)
            self.materials.extend(q.materials)
            local = q.mat if q.mat is not None else np.zeros(len(q.arrays["x"]), dtype=np.int32)
            mats.append(np.asarray(local, dtype=np.int32) + base)
        self.t["mat"] = torch.from_numpy(np.concatenate(mats).astype(np.int32)).to(dev)
        self.t["id"] = torch.arange(self.n, dtype=torch.int64, device=dev)
        K = p0.units if units is None else units
        self.K = int(K) if self.n_inst == 1 else 0
        self.unit_dim = p0.unit_dim
        self.t["unit"] = torch.zeros(self.n, dtype=torch.int32, device=dev)
        self.gen = None
        if self.K > 0:
            if generators is None:
                raise ValueError("work units need initial generators")
            self.gen = torch.as_tensor(np.asarray(generators, dtype=np.float64), device=dev).contiguous()
            assert self.gen.shape == (self.K, self.unit_dim)
        self.time = torch.zeros(self.n_inst, **f64)

        prm = abi.sph_params()
        prm.dim, prm.kernel, prm.precision = self.dim, _KERNEL[p0.kernel], _PREC[precision]
        prm.n_mat = len(self.materials)
        prm.kappa, prm.eta, prm.cfl, prm.cell_beta, prm.cell_cap = p0.kappa, p0.eta, p0.cfl, cell_beta, cell_cap
        self._mat_arr = (abi.sph_material * len(self.materials))()
        for i, m in enumerate(self.materials):
            dst = self._mat_arr[i]
            dst.eos, dst.gamma, dst.rho0, dst.c0, dst.p_inf, dst.s_a = _EOS[m.eos], m.gamma, m.rho0, m.c0, m.p_inf, m.s_a
            if i < abi.SPH_MAX_MAT:
                prm.mat[i] = dst
        prm.materials = C.cast(self._mat_arr, C.c_void_p) if len(self.materials) > abi.SPH_MAX_MAT else None
        prm.n_units, prm.unit_dim = self.K, self.unit_dim
        prm.n_upd = (p0.n_upd if n_upd is None else n_upd) if self.K > 0 else 0
        prm.theta, prm.sigma, prm.gamma_b, prm.beta_sh = theta, sigma, gamma_b, beta_sh
        prm.pair_blocks_per_sm = pair_blocks_per_sm
        prm.order = order
        prm.solver = _SOLVER[solver]
        prm.load_measure = _LOAD[load_measure]
        prm.list_cap = list_cap
        prm.unit_sched = _SCHED[unit_sched]
        prm.list_staging = int(list_staging)
        prm.generators = self.gen.data_ptr() if self.gen is not None else None
        self.params = prm
        self.precision = precision
        self.handle = abi.sph_init(prm, self.n_inst, [int(v) for v in self.inst_offsets], self.state(),
                                   _stream_ptr())

    # ---------------------------------------------------------------- state
    def state(self) -> abi.sph_state:
        s = abi.sph_state()
        s.n = self.n
        for k in abi.STATE_F64 + abi.STATE_RATES + abi.STATE_DERIVED + ("mat", "id", "unit"):
            v = self.t[k]
            setattr(s, k, v.data_ptr() if v is not None else None)
        return s

    def numpy(self) -> dict:
        torch.cuda.synchronize(self.device)
        return {k: v.cpu().numpy() for k, v in self.t.items() if v is not None}

    # ---------------------------------------------------------------- calls
    def build_cells(self):
        abi.sph_build_cells(self.handle, self.state(), _stream_ptr())

    def eval_rates(self):
        abi.sph_eval_rates(self.handle, self.state(), _stream_ptr())

    def step(self, n_steps: int = 1):
        abi.sph_step(self.handle, self.state(), n_steps, self.time.data_ptr(), _stream_ptr())

    def step_dt(self, dts: torch.Tensor):
        """Steps with prescribed time steps (device tensor, n_steps x n_instances)."""
        dts = dts.contiguous()
        abi.sph_step_dt(self.handle, self.state(), dts.shape[0], dts.data_ptr(), self.time.data_ptr(),
                        _stream_ptr())

    def last_dt(self, out: torch.Tensor):
        abi.sph_last_dt(self.handle, out.data_ptr(), _stream_ptr())

    def assign(self, gen=None) -> torch.Tensor:
        g = self.gen if gen is None else gen
        offs = torch.zeros(self.K + 1, dtype=torch.int32, device=self.device)
        abi.voronoi_assign(self.handle, self.state(), g.data_ptr(), self.K, self.unit_dim,
                           self.t["unit"].data_ptr(), offs.data_ptr(), _stream_ptr())
        return offs

    def balance(self, gen=None, load=None, theta=0.25, sigma=0.5, gamma_b=1.0, beta_sh=0.45) -> torch.Tensor:
        g = self.gen if gen is None else gen
        bp = abi.sph_balance_params(theta, sigma, gamma_b, beta_sh)
        shift = torch.zeros(1, dtype=torch.float64, device=self.device)
        abi.voronoi_balance(self.handle, self.state(), g.data_ptr(), self.K, self.unit_dim,
                            None if load is None else load.data_ptr(), bp, shift.data_ptr(), _stream_ptr())
        return shift

    def conservation(self) -> torch.Tensor:
        out = torch.zeros(self.n_inst, 5, dtype=torch.float64, device=self.device)
        abi.sph_conservation(self.handle, self.state(), out.data_ptr(), _stream_ptr())
        return out

    def unit_stats(self):
        load = np.zeros(self.K)
        adj = np.zeros((self.K, self.K), dtype=np.uint8)
        abi.sph_unit_stats(self.handle, load.ctypes.data_as(C.POINTER(C.c_double)),
                           adj.ctypes.data_as(C.POINTER(C.c_uint8)), _stream_ptr())
        return load, adj

    def cell_index(self):
        cells = torch.zeros(self.n, dtype=torch.int32, device=self.device)
        grid = np.zeros(8 * self.n_inst)
        abi.sph_cell_index(self.handle, self.state(), cells.data_ptr(),
                           grid.ctypes.data_as(C.POINTER(C.c_double)), _stream_ptr())
        return cells.cpu().numpy(), grid.reshape(self.n_inst, 8)

    def pair_list(self, cap: int | None = None):
        """Interacting pairs (i < j, particle indices), sorted; also evaluates the rates."""
        cap = cap or max(64, 64 * self.n)
        pi = torch.zeros(cap, dtype=torch.int32, device=self.device)
        pj = torch.zeros(cap, dtype=torch.int32, device=self.device)
        cnt = abi.sph_pair_list(self.handle, self.state(), cap, pi.data_ptr(), pj.data_ptr(), _stream_ptr())
        a, b = pi[:cnt].cpu().numpy(), pj[:cnt].cpu().numpy()
        o = np.lexsort((b, a))
        return a[o], b[o]

    def profile(self, enable: bool = True):
        abi.sph_profile(self.handle, enable)

    def profile_read(self):
        """(pair-kernel ms summed, pair launches, kernel launches) since the last call."""
        return abi.sph_profile_read(self.handle)

    def list_builds(self):
        """(Verlet-list builds so far, list capacity per particle); needs cell_beta > 0."""
        return abi.sph_list_builds(self.handle, _stream_ptr())

    def unit_times(self):
        """(start, end) in ns of each unit's work in the last list evaluation (K x 2)."""
        out = np.zeros(2 * self.K)
        abi.sph_unit_times(self.handle, out, _stream_ptr())
        return out.reshape(self.K, 2)

    def read_status(self) -> int:
        return abi.sph_read_status(self.handle)

    def pair_counts(self):
        return abi.sph_pair_counts(self.handle, _stream_ptr())

    def close(self):
        if getattr(self, "handle", None) is not None:
            torch.cuda.synchronize(self.device)
            abi.sph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
