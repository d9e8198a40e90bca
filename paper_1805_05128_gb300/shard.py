"""The Voronoi decomposition spread over processes, one rank per GPU (the
paper's parallel scheme, Secs. 3-4 and Alg. 1, with ranks in place of its
one-subdomain-per-core MPI processes).

* Units to ranks: unit k belongs to rank k * world // K.  The units are
  numbered along a Morton curve by the generator seeding, so each rank's
  units form a compact region.
* Alien layers (Sec. 4.3): before every step a rank sends to every other
  rank the particles of its own units that lie within D^sh_kl of the bisector
  between their unit l and a unit k of the other rank (D^sh_kl = max(rmax_k,
  rmax_l), eq. Horizon).  Any particle that can interact with a particle of
  V_k lies within that distance of the bisector, so the layer holds every
  neighbour the other rank needs; the step runs on owned + alien particles
  and keeps the owned ones.
* The time step (Alg. 1, "global synchronization of SPH time step"): each
  rank's CFL bound on its local set, reduced to the minimum over the ranks;
  every rank steps with that dt.
* Every n_upd steps (Alg. 1, outer loop): the unit statistics (loads with
  1/2 per crossing pair end, adjacency, rmax, centroids, counts) are summed or
  maximised over the ranks, every rank applies the same balancing update to
  the generators, reassigns its particles, and sends those whose new unit
  belongs to another rank to their new owner.

This module is the host orchestration only.  The computation of a rank (its
CFL bound, a step with a prescribed dt, the rates and pair list of its local
set, the Voronoi assignment, the balancing update) is a backend's:
LibBackend runs it in libcsph on the rank's GPU.  Communication is
torch.distributed: point-to-point sends of the alien layers and of migrating
particles, all-reduce for dt and the statistics (NCCL between GPUs, with
remote data copied into local memory first; gloo on CPUs).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

# per-particle arrays carried between ranks (float64), then the integer ones
F64 = ("x", "y", "z", "vx", "vy", "vz", "rho", "E", "m", "ax", "ay", "az", "drho", "dE", "d")
I64 = ("id", "mat", "unit")


def rank_of_unit(K: int, world: int) -> np.ndarray:
    """Owner rank of each unit: contiguous blocks of unit indices."""
    return (np.arange(K) * world) // K


@dataclass
class Config:
    dim: int
    K: int
    gdim: int
    n_upd: int
    kh: float              # (kappa / 2) eta
    beta_sh: float = 0.45
    theta: float = 0.25
    sigma: float = 0.5
    gamma_b: float = 1.0


def take(st: dict, sel) -> dict:
    return {k: (v[sel] if v is not None else None) for k, v in st.items()}


def concat(parts: list) -> dict:
    keys = parts[0].keys()
    return {k: (np.concatenate([p[k] for p in parts]) if parts[0][k] is not None else None) for k in keys}


def alien_selection(st: dict, owner_units, dest_units, gen, rmax, gdim: int) -> np.ndarray:
    """Mask of the particles of `st` (all in units owner_units) within D^sh_kl
    of the bisector between their unit l and a unit k in dest_units."""
    pos = np.stack([st[a] for a in ("x", "y", "z")[:gdim]], axis=1)
    sel = np.zeros(len(pos), dtype=bool)
    for l in owner_units:
        mine = st["unit"] == l
        if not mine.any():
            continue
        p = pos[mine]
        hit = np.zeros(len(p), dtype=bool)
        for k in dest_units:
            n = gen[k] - gen[l]
            nn = np.linalg.norm(n)
            if nn == 0.0:
                hit[:] = True
                continue
            D = max(rmax[k], rmax[l])
            s = (p - 0.5 * (gen[k] + gen[l])) @ (n / nn)     # signed distance towards unit k
            hit |= s > -D
        idx = np.flatnonzero(mine)
        sel[idx[hit]] = True
    return sel


def unit_stats_from_pairs(pi, pj, st: dict, owned: int, K: int, gdim: int, kh: float, beta: float):
    """A rank's share of the unit statistics from the interacting pairs of its
    local set (indices < owned are its own particles): 1/2 load per pair end
    it owns, adjacency of every pair with an owned end, R^hrz_i = (1 + beta)
    kh (d_i + max_j d_j) of its own particles (own size if isolated), position
    sums and counts of its own particles."""
    unit, d = st["unit"], st["d"]
    load = np.zeros(K)
    adj = np.zeros((K, K), dtype=np.uint8)
    dmax = np.full(len(d), -1.0)
    for a, b in ((pi, pj), (pj, pi)):
        np.maximum.at(dmax, a, d[b])
        own = a < owned
        np.add.at(load, unit[a[own]], 0.5)
    cross = (unit[pi] != unit[pj]) & ((pi < owned) | (pj < owned))
    adj[unit[pi[cross]], unit[pj[cross]]] = 1
    adj[unit[pj[cross]], unit[pi[cross]]] = 1
    o = slice(0, owned)
    dm = np.where(dmax[o] < 0.0, d[o], dmax[o])
    rh = (1.0 + beta) * (kh * (d[o] + dm))
    rmax = np.zeros(K)
    np.maximum.at(rmax, unit[o], rh)
    pos_sum = np.zeros((K, gdim))
    for a, ax in enumerate(("x", "y", "z")[:gdim]):
        np.add.at(pos_sum[:, a], unit[o], st[ax][o])
    count = np.bincount(unit[o], minlength=K).astype(np.int64)
    return load, adj, rmax, pos_sum, count


class Decomposed:
    """One rank's share of a decomposed run.  `state` holds every particle of
    the problem on every rank at construction (seeded synthetic input); the
    rank keeps those of its units."""

    def __init__(self, cfg: Config, state: dict, gen, backend, dist=None, comm_device="cpu"):
        self.cfg, self.be, self.dist = cfg, backend, dist
        self.rank = dist.get_rank() if dist else 0
        self.world = dist.get_world_size() if dist else 1
        self.dev = torch.device(comm_device)
        self.owner = rank_of_unit(cfg.K, self.world)
        self.my_units = np.flatnonzero(self.owner == self.rank)
        self.gen = np.array(gen, dtype=np.float64)
        full = {k: (np.array(state[k]) if state.get(k) is not None else None) for k in F64 + I64}
        n = len(full["x"])
        unused = {"y", "vy", "ay"} if cfg.dim < 2 else set()
        unused |= {"z", "vz", "az"} if cfg.dim < 3 else set()
        for k in F64:                            # rates, size: written by the first evaluation
            if full[k] is None and k not in unused:
                full[k] = np.zeros(n)
        if full["id"] is None:
            full["id"] = np.arange(n, dtype=np.int64)
        if full["mat"] is None:
            full["mat"] = np.zeros(n, dtype=np.int64)
        full["unit"] = self.be.assign(self._pos(full), self.gen).astype(np.int64)
        self.st = take(full, np.isin(full["unit"], self.my_units))
        self.rmax = np.zeros(cfg.K)
        self.steps = 0
        self.time = 0.0
        # held rates and horizon at the start: rates of the whole local set, statistics reduced
        local, n_own = self._with_aliens(initial=True)
        self.be.eval_rates(local)
        self.st = take(local, slice(0, n_own))
        self._reduce_stats(local, n_own)

    # ------------------------------------------------------------ helpers
    def _pos(self, st):
        return [st[a] for a in ("x", "y", "z")[: self.cfg.gdim]]

    def _t(self, a):
        return torch.as_tensor(a, device=self.dev)

    def _all_reduce(self, arr, op):
        if self.dist is None:
            return arr
        t = self._t(np.ascontiguousarray(arr))
        self.dist.all_reduce(t, op=op)
        return t.cpu().numpy()

    def _exchange(self, outgoing: dict) -> list:
        """Point-to-point exchange of particle sets: outgoing[q] is sent to rank q;
        returns the sets received from every other rank (rank order)."""
        if self.dist is None:
            return []
        d = self.dist
        keys = [k for k in F64 + I64 if self.st[k] is not None]
        sends, recvs, bufs = [], [], {}
        counts = {}
        for q in range(self.world):
            if q == self.rank:
                continue
            n = torch.tensor([len(outgoing[q]["x"])], dtype=torch.int64, device=self.dev)
            r = torch.zeros(1, dtype=torch.int64, device=self.dev)
            # lower rank sends first: a deadlock-free order for blocking calls
            if self.rank < q:
                d.send(n, q)
                d.recv(r, q)
            else:
                d.recv(r, q)
                d.send(n, q)
            counts[q] = int(r.item())
        for q in range(self.world):
            if q == self.rank:
                continue
            out = outgoing[q]
            f = np.stack([out[k] for k in keys if k in F64], axis=1) if len(out["x"]) else \
                np.zeros((0, sum(k in F64 for k in keys)))
            i = np.stack([out[k] for k in keys if k in I64], axis=1).astype(np.int64) if len(out["x"]) else \
                np.zeros((0, sum(k in I64 for k in keys)), dtype=np.int64)
            bufs[q] = (torch.zeros((counts[q], f.shape[1]), dtype=torch.float64, device=self.dev),
                       torch.zeros((counts[q], i.shape[1]), dtype=torch.int64, device=self.dev))
            sends += [d.isend(self._t(np.ascontiguousarray(f)), q), d.isend(self._t(np.ascontiguousarray(i)), q)]
            recvs += [d.irecv(bufs[q][0], q), d.irecv(bufs[q][1], q)]
        for w in sends + recvs:
            w.wait()
        got = []
        for q in sorted(bufs):
            f, i = bufs[q][0].cpu().numpy(), bufs[q][1].cpu().numpy()
            s, fi, ii = {}, 0, 0
            for k in F64 + I64:
                if k not in keys:
                    s[k] = None
                elif k in F64:
                    s[k] = f[:, fi].copy()
                    fi += 1
                else:
                    s[k] = i[:, ii].copy()
                    ii += 1
            got.append(s)
        return got

    def _with_aliens(self, initial=False):
        """The local set: own particles, then the alien layers of the other ranks."""
        out = {}
        for q in range(self.world):
            if q == self.rank:
                continue
            dest = np.flatnonzero(self.owner == q)
            if initial:        # no horizon yet: send everything within the largest plausible layer
                sel = np.ones(len(self.st["x"]), dtype=bool)
            else:
                sel = alien_selection(self.st, self.my_units, dest, self.gen, self.rmax, self.cfg.gdim)
            out[q] = take(self.st, sel)
        parts = [self.st] + self._exchange(out)
        return concat(parts), len(self.st["x"])

    def _reduce_stats(self, local, n_own):
        pi, pj = self.be.pairs(local)
        load, adj, rmax, pos_sum, count = unit_stats_from_pairs(pi, pj, local, n_own, self.cfg.K, self.cfg.gdim,
                                                                self.cfg.kh, self.cfg.beta_sh)
        d = self.dist
        SUM = d.ReduceOp.SUM if d else None
        MAX = d.ReduceOp.MAX if d else None
        load = self._all_reduce(load, SUM)
        pos_sum = self._all_reduce(pos_sum, SUM)
        count = self._all_reduce(count, SUM)
        adj = self._all_reduce(adj.astype(np.int64), MAX).astype(np.uint8)
        self.rmax = self._all_reduce(rmax, MAX)
        cen = np.where(count[:, None] > 0, pos_sum / np.maximum(count, 1)[:, None], self.gen)
        return load, adj, self.rmax, cen, count

    # --------------------------------------------------------------- step
    def step(self, n_steps: int = 1):
        cfg = self.cfg
        for _ in range(n_steps):
            local, n_own = self._with_aliens()
            dt = self.be.cfl_dt(local)
            if self.dist is not None:
                dt = float(self._all_reduce(np.array([dt]), self.dist.ReduceOp.MIN)[0])
            self.be.step_dt(local, dt)
            self.time += dt
            self.steps += 1
            self.st = take(local, slice(0, n_own))
            if cfg.n_upd > 0 and self.steps % cfg.n_upd == 0:
                # statistics of the new state: its own alien layers first (the aliens
                # of the step's local set were advanced with incomplete neighbourhoods)
                fresh, n_fresh = self._with_aliens()
                load, adj, rmax, cen, count = self._reduce_stats(fresh, n_fresh)
                self.gen, _ = self.be.balance(self.gen, load, adj, rmax, cen, count, cfg)
                mine = self.st
                mine["unit"] = self.be.assign(self._pos(mine), self.gen).astype(np.int64)
                stay = np.isin(mine["unit"], self.my_units)
                out = {q: take(mine, np.isin(mine["unit"], np.flatnonzero(self.owner == q)))
                       for q in range(self.world) if q != self.rank}
                self.st = concat([take(mine, stay)] + self._exchange(out))

    def gather(self) -> dict:
        """Every particle of the run on every rank, ordered by id (for checks)."""
        parts = [self.st]
        if self.dist is not None:
            objs = [None] * self.world
            self.dist.all_gather_object(objs, self.st)
            parts = objs
        allp = concat(parts)
        return take(allp, np.argsort(allp["id"]))


class LibBackend:
    """A rank's computation in libcsph on its GPU: the rates and pair list of
    the local set, its CFL bound (sph_cfl_dt), one step with the reduced dt
    (sph_step_dt), the Voronoi assignment (voronoi_assign_static) and the
    balancing update from the reduced statistics (voronoi_balance_stats).
    A handle is created for each local set (its size changes every step)."""

    def __init__(self, problem_like, precision="mixed", device="cuda"):
        self.like, self.precision, self.device = problem_like, precision, torch.device(device)

    def _sim(self, st, units=0, gen=None):
        import synth
        from .sim import Simulation
        arrays = {k: st[k] for k in ("x", "y", "z", "vx", "vy", "vz", "rho", "E", "m") if st.get(k) is not None}
        q = synth.Problem("local", self.like.dim, arrays, self.like.materials,
                          mat=st["mat"].astype(np.int32) if st.get("mat") is not None else None,
                          kernel=self.like.kernel, kappa=self.like.kappa, eta=self.like.eta, cfl=self.like.cfl,
                          units=units, unit_dim=self.like.unit_dim)
        sim = Simulation(q, precision=self.precision, units=units, generators=gen, n_upd=0, device=self.device)
        for k in ("ax", "ay", "az", "drho", "dE"):
            if sim.t.get(k) is not None and st.get(k) is not None:
                sim.t[k].copy_(torch.as_tensor(st[k], device=self.device))
        return sim

    @staticmethod
    def _back(sim, st):
        g = sim.numpy()
        for k in ("x", "y", "z", "vx", "vy", "vz", "rho", "E", "ax", "ay", "az", "drho", "dE", "d"):
            if st.get(k) is not None and k in g:
                st[k][:] = g[k]

    def eval_rates(self, st):
        sim = self._sim(st)
        sim.eval_rates()
        self._back(sim, st)
        sim.close()

    def cfl_dt(self, st) -> float:
        from . import abi
        sim = self._sim(st)
        out = torch.zeros(1, dtype=torch.float64, device=self.device)
        abi.sph_cfl_dt(sim.handle, sim.state(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        dt = float(out.item())
        sim.close()
        return dt

    def step_dt(self, st, dt: float):
        from . import abi
        sim = self._sim(st)
        abi.sph_hold_rates(sim.handle)           # the rates in st are the scheme's held rates
        abi_dt = torch.tensor([[dt]], dtype=torch.float64, device=self.device)
        abi.sph_step_dt(sim.handle, sim.state(), 1, abi_dt.data_ptr(), sim.time.data_ptr(),
                        torch.cuda.current_stream().cuda_stream)
        self._back(sim, st)
        sim.close()

    def pairs(self, st):
        sim = self._sim(st)
        pi, pj = sim.pair_list()
        st["d"][:] = sim.numpy()["d"]
        sim.close()
        return pi.astype(np.int64), pj.astype(np.int64)

    def assign(self, pos, gen):
        from . import abi
        n = len(pos[0])
        K, dim = np.asarray(gen).shape
        dev = self.device
        P = [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev) for a in pos]
        g = torch.as_tensor(np.ascontiguousarray(gen), dtype=torch.float64, device=dev)
        unit = torch.zeros(n, dtype=torch.int32, device=dev)
        ptr = [t.data_ptr() for t in P] + [None] * (3 - len(P))
        abi.voronoi_assign_static(n, ptr[0], ptr[1], ptr[2], g.data_ptr(), K, dim, unit.data_ptr(), None, None,
                                  torch.cuda.current_stream().cuda_stream)
        return unit.cpu().numpy()

    def balance(self, gen, load, adj, rmax, cen, count, cfg):
        from . import abi
        K, dim = gen.shape
        st = {k: np.asarray(self.like.arrays[k][:1]) for k in ("x", "y", "z", "vx", "vy", "vz", "rho", "E", "m")
              if k in self.like.arrays}
        st["mat"] = None
        g = torch.as_tensor(gen, dtype=torch.float64, device=self.device).contiguous()
        sim = self._sim(st, units=K, gen=gen)
        shift = torch.zeros(1, dtype=torch.float64, device=self.device)
        bp = abi.sph_balance_params(cfg.theta, cfg.sigma, cfg.gamma_b, cfg.beta_sh)
        abi.voronoi_balance_stats(sim.handle, g.data_ptr(), K, dim, np.ascontiguousarray(load, dtype=np.float64),
                                  np.ascontiguousarray(adj, dtype=np.uint8),
                                  np.ascontiguousarray(rmax, dtype=np.float64),
                                  np.ascontiguousarray(cen, dtype=np.float64),
                                  np.ascontiguousarray(count, dtype=np.int64), bp, shift.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
        out = g.cpu().numpy()
        sim.close()
        return out, float(shift.item())
