"""The Voronoi decomposition spread over ranks (paper_1805_05128_gb300.shard):
units to ranks, alien layers of width D^sh exchanged every step (Sec. 4.3),
the time step reduced to the minimum over the ranks (Alg. 1), rebalancing
every n_upd steps with the statistics reduced over the ranks and the
particles that change rank moved to their owner.  Two gloo ranks on the CPU,
the ranks' computation done by the oracle (a test backend), against the same
run on one rank.  The GPU data plane (NCCL point-to-point and all-reduce,
LibBackend) is not run on hardware here."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp       # noqa: E402

STEPS = 7


class OracleBackend:
    """A rank's computation by the FP64 oracle (test infrastructure only)."""

    def __init__(self, p, dim):
        self.p, self.dim = p, dim

    def _state(self, st):
        import oracle as O
        keys = [k for k in O.State.FIELDS + O.State.DERIVED if st.get(k) is not None]
        return O.State(self.dim, {k: st[k] for k in keys}, st["mat"].astype(np.int32))

    @staticmethod
    def _back(s, st):
        for k in ("x", "y", "z", "vx", "vy", "vz", "rho", "E", "ax", "ay", "az", "drho", "dE", "d"):
            if st.get(k) is not None:
                st[k][:] = getattr(s, k)

    def eval_rates(self, st):
        import oracle as O
        s = self._state(st)
        O.eval_rates(self.p, s)
        self._back(s, st)

    def cfl_dt(self, st):
        import oracle as O
        s = self._state(st)
        O.derive(self.p, s)
        return O.dt(self.p, s)

    def step_dt(self, st, dt):
        import oracle as O
        s = self._state(st)
        O.step_replay(self.p, s, [dt], rates_valid=True)
        self._back(s, st)

    def pairs(self, st):
        import oracle as O
        s = self._state(st)
        O.derive(self.p, s)
        pi, pj = O.pairs(self.p, s)
        st["d"][:] = s.d
        return pi.astype(np.int64), pj.astype(np.int64)

    def assign(self, pos, gen):
        import oracle as O
        return O.voronoi_assign(pos, gen)

    def balance(self, gen, load, adj, rmax, cen, count, cfg):
        import oracle as O
        dsh = np.maximum(rmax[:, None], rmax[None, :])
        g, shift, _ = O.balance(gen, load, adj, dsh, cen, count, cfg.theta, cfg.sigma, cfg.gamma_b)
        return g, shift


def _problem():
    import synth
    return synth.plate_impact(5, (16, 16, 4), a=1e-4, v=1000.0, units=6, seed=5, jitter=0.05)


def _run(rank, world, port, out, steps):
    import oracle as O
    import synth
    from paper_1805_05128_gb300 import shard
    if world > 1:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = _problem()
    p, _ = O.from_problem(prob)
    cfg = shard.Config(dim=3, K=prob.units, gdim=2, n_upd=3, kh=0.5 * prob.kappa * prob.eta)
    gen = synth.problem_generators(prob)
    run = shard.Decomposed(cfg, dict(prob.arrays), gen, OracleBackend(p, 3), dist if world > 1 else None)
    n0 = len(run.st["x"])
    ids0 = run.st["id"].copy()
    run.step(steps)
    g = run.gather()
    res = {k: g[k] for k in ("id", "x", "y", "z", "vx", "vy", "vz", "rho", "E")}
    res["gen"] = run.gen
    res["time"] = run.time
    res["owned0"] = n0
    res["moved_in"] = int(np.setdiff1d(run.st["id"], ids0).size)   # particles received from the other rank
    if world > 1:
        out.put((rank, res))
        dist.barrier()
        dist.destroy_process_group()
    return res


def _free_port() -> int:
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def test_two_gloo_ranks_equal_one_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_run, args=(r, world, port, q, STEPS)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    ref = _run(0, 1, 0, None, STEPS)
    n = len(ref["id"])
    assert got[0]["owned0"] > 0 and got[1]["owned0"] > 0 and got[0]["owned0"] + got[1]["owned0"] == n
    assert got[0]["moved_in"] + got[1]["moved_in"] > 0            # the rebalancing moved particles between ranks
    for r in range(world):
        a = got[r]
        assert np.array_equal(a["id"], ref["id"])                 # every particle once, none lost
        assert a["time"] == pytest.approx(ref["time"], rel=1e-14)  # the same reduced dt sequence
        np.testing.assert_allclose(a["gen"], ref["gen"], rtol=0, atol=1e-12 * np.max(np.abs(ref["gen"])))
        for k in ("x", "y", "z", "vx", "vy", "vz", "rho", "E"):
            scale = np.max(np.abs(ref[k]))
            assert np.max(np.abs(a[k] - ref[k])) <= 1e-12 * scale, (r, k)


def test_alien_layer_holds_every_interacting_neighbour():
    """Every interacting pair that joins units of two ranks has its other end
    in the alien layer sent to the rank (the bisector distance bound)."""
    import oracle as O
    import synth
    from paper_1805_05128_gb300 import shard
    prob = _problem()
    p, s = O.from_problem(prob)
    O.derive(p, s)
    pi, pj = O.pairs(p, s)
    gen = synth.problem_generators(prob)
    unit = O.voronoi_assign([s.x, s.y], gen)
    K, world = prob.units, 2
    owner = shard.rank_of_unit(K, world)
    st = {"x": s.x, "y": s.y, "z": s.z, "d": s.d, "unit": unit.astype(np.int64)}
    kh = 0.5 * prob.kappa * prob.eta
    _, _, rmax, _, _ = shard.unit_stats_from_pairs(pi, pj, st, len(s.x), K, 2, kh, 0.45)
    for r in range(world):
        q = 1 - r
        mine = owner[unit] == r
        layer = np.zeros(len(s.x), dtype=bool)
        sub = {k: v[mine] for k, v in st.items()}
        layer[np.flatnonzero(mine)] = shard.alien_selection(sub, np.flatnonzero(owner == r),
                                                            np.flatnonzero(owner == q), gen, rmax, 2)
        cross = (owner[unit[pi]] != owner[unit[pj]])
        for a, b in ((pi[cross], pj[cross]), (pj[cross], pi[cross])):
            need = owner[unit[a]] == r            # r's particle a interacts with q's particle b
            assert np.all(layer[a[need]])
        assert layer.sum() < mine.sum()           # a layer, not the whole subdomain
