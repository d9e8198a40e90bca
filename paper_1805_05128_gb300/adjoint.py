"""Differentiable CSPH runs: a torch.autograd.Function whose backward is the
hand-written adjoint of libcsph.so (sph_step_adjoint), with checkpoint and
recompute every `every` steps so memory stays bounded by one segment.

CSPHRun.apply(pos, vel, rho, E, c0, gamma, spec) -> (pos, vel, rho, E)
  pos, vel: (n, dim) device float64 tensors; rho, E: (n,) device float64;
  c0, gamma: 0-d float64 tensors, the stiffened-gas (or ideal-gas gamma)
  parameters of material 0; spec: RunSpec (fixed problem data).
The time steps of the forward run are recorded and held fixed in the
backward pass (dt is a stop-gradient), as is the pair set of each step.
spec.precision sets the forward replay ("mixed": FP32 pair fluxes, "fp64");
spec.reverse sets the pair derivatives of a mixed run ("fp64": FP32 forward
with FP64 adjoint accumulation; "fp32": FP32 with Kahan sums, several times
faster); the chain through the EOS and the kick-drift-kick algebra is FP64
in all cases.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import torch

from . import abi

_PREC = {"fp64": abi.SPH_PREC_FP64, "mixed": abi.SPH_PREC_MIXED}


@dataclass
class RunSpec:
    m: torch.Tensor                  # (n,) masses, device float64
    n_steps: int
    every: int = 10                  # checkpoint interval
    dim: int = 3
    eos: str = "stiffened"           # "stiffened" | "ideal"
    rho0: float = 2700.0
    eta: float = 1.3
    kappa: float = 2.0
    cfl: float = 0.3
    precision: str = "mixed"
    reverse: str = "fp64"            # mixed precision: pair derivatives in "fp64" or "fp32" (Kahan sums)
    cell_cap: int = 1 << 24
    record: dict = field(default_factory=dict)   # filled by forward: dts, loss bookkeeping


def _params(spec: RunSpec, c0: float, gamma: float) -> abi.sph_params:
    p = abi.sph_params()
    p.dim, p.kernel, p.precision, p.n_mat = spec.dim, abi.SPH_KERNEL_CUBIC, _PREC[spec.precision], 1
    p.kappa, p.eta, p.cfl, p.cell_beta, p.cell_cap = spec.kappa, spec.eta, spec.cfl, 0.0, spec.cell_cap
    # the stiffened gas given by (rho0, c0, gamma): the library derives P_inf
    p.mat[0].eos = abi.SPH_EOS_STIFFENED_C0 if spec.eos == "stiffened" else abi.SPH_EOS_IDEAL
    p.mat[0].gamma, p.mat[0].rho0, p.mat[0].c0 = gamma, spec.rho0, c0
    return p


class _Run:
    """A handle with its state tensors (positions and velocities split per axis)."""

    FIELDS = ("x", "y", "z", "vx", "vy", "vz", "rho", "E", "ax", "ay", "az", "drho", "dE", "d", "P", "c")

    def __init__(self, spec: RunSpec, pos, vel, rho, E, c0, gamma):
        n, dim = pos.shape
        dev = pos.device
        self.n, self.dim, self.dev = n, dim, dev
        self.t = {}
        for a, k in enumerate(("x", "y", "z")):
            self.t[k] = pos[:, a].contiguous().clone() if a < dim else None
        for a, k in enumerate(("vx", "vy", "vz")):
            self.t[k] = vel[:, a].contiguous().clone() if a < dim else None
        self.t["rho"], self.t["E"] = rho.contiguous().clone(), E.contiguous().clone()
        for k in ("ax", "ay", "az"):
            self.t[k] = torch.zeros(n, dtype=torch.float64, device=dev) if "xyz".index(k[1]) < dim else None
        for k in ("drho", "dE", "d", "P", "c"):
            self.t[k] = torch.zeros(n, dtype=torch.float64, device=dev)
        self.t["m"] = spec.m.contiguous()
        self.params = _params(spec, c0, gamma)
        self.handle = abi.sph_init(self.params, 1, [0, n], self.state(), torch.cuda.current_stream().cuda_stream)

    def state(self, t=None) -> abi.sph_state:
        t = self.t if t is None else t
        s = abi.sph_state()
        s.n = self.n
        for k in self.FIELDS + ("m",):
            v = t.get(k)
            setattr(s, k, v.data_ptr() if v is not None else None)
        return s

    def snapshot(self) -> dict:
        keep = ("x", "y", "z", "vx", "vy", "vz", "rho", "E", "ax", "ay", "az", "drho", "dE")
        snap = {k: (self.t[k].clone() if self.t[k] is not None else None) for k in keep}
        snap["m"] = self.t["m"]
        for k in ("d", "P", "c"):
            snap[k] = torch.zeros_like(self.t["rho"])
        return snap

    def close(self):
        if self.handle is not None:
            torch.cuda.synchronize(self.dev)
            abi.sph_destroy(self.handle)
            self.handle = None


class CSPHRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, vel, rho, E, c0, gamma, spec: RunSpec):
        st = torch.cuda.current_stream().cuda_stream
        run = _Run(spec, pos.detach(), vel.detach(), rho.detach(), E.detach(), float(c0), float(gamma))
        abi.sph_eval_rates(run.handle, run.state(), st)
        dts = torch.zeros(max(spec.n_steps, 1), dtype=torch.float64, device=pos.device)
        ckpts = []
        for k in range(spec.n_steps):
            if k % spec.every == 0:
                ckpts.append((k, run.snapshot()))
            abi.sph_step(run.handle, run.state(), 1, None, st)
            abi.sph_last_dt(run.handle, dts[k:].data_ptr(), st)
        spec.record["dts"] = dts[: spec.n_steps]
        ctx.run, ctx.ckpts, ctx.dts, ctx.spec = run, ckpts, dts, spec
        dim = run.dim
        out_pos = torch.stack([run.t[k] for k in ("x", "y", "z")[:dim]], dim=1).clone()
        out_vel = torch.stack([run.t[k] for k in ("vx", "vy", "vz")[:dim]], dim=1).clone()
        return out_pos, out_vel, run.t["rho"].clone(), run.t["E"].clone()

    @staticmethod
    def backward(ctx, g_pos, g_vel, g_rho, g_E):
        run, spec = ctx.run, ctx.spec
        n, dim, dev = run.n, run.dim, run.dev
        st = torch.cuda.current_stream().cuda_stream
        z = lambda: torch.zeros(n, dtype=torch.float64, device=dev)
        adj = {}
        for a, k in enumerate(("x", "y", "z")):
            adj[k] = (g_pos[:, a].contiguous().clone() if g_pos is not None else z()) if a < dim else None
        for a, k in enumerate(("vx", "vy", "vz")):
            adj[k] = (g_vel[:, a].contiguous().clone() if g_vel is not None else z()) if a < dim else None
        adj["rho"] = g_rho.contiguous().clone() if g_rho is not None else z()
        adj["E"] = g_E.contiguous().clone() if g_E is not None else z()
        for k in ("ax", "ay", "az"):
            adj[k] = z() if "xyz".index(k[1]) < dim else None
        adj["drho"], adj["dE"] = z(), z()
        adj_s = run.state(adj)
        par = torch.zeros(2, dtype=torch.float64, device=dev)
        bounds = [k for k, _ in ctx.ckpts] + [spec.n_steps]
        for idx in range(len(ctx.ckpts) - 1, -1, -1):
            k0, snap = ctx.ckpts[idx]
            length = bounds[idx + 1] - k0
            ck = abi.sph_ckpt()
            ck.state = run.state(snap)
            ck.dt = ctx.dts[k0:].data_ptr()
            ck.rates_from_state = 1 if k0 == 0 else 0
            ck.reverse_fp64 = 1 if spec.reverse == "fp64" else 0
            abi.sph_step_adjoint(run.handle, ck, length, adj_s, adj_s, par.data_ptr(), st)
        gpos = torch.stack([adj[k] for k in ("x", "y", "z")[:dim]], dim=1)
        gvel = torch.stack([adj[k] for k in ("vx", "vy", "vz")[:dim]], dim=1)
        run.close()
        return gpos, gvel, adj["rho"], adj["E"], par[0], par[1], None


def csph_run(pos, vel, rho, E, c0, gamma, spec: RunSpec):
    """Run spec.n_steps CSPH steps differentiably; returns the final (pos, vel, rho, E)."""
    return CSPHRun.apply(pos, vel, rho, E, c0, gamma, spec)
