"""Host-side logic of the multi-rank path on CPU (gloo, world size 2): k-point shards, the final
gather of eigenvalues and the max-over-ranks time.  No GPU is used."""
import os
import socket

import numpy as np
import pytest

from paper_1211_1446_gb300 import shard


def test_kpoint_shards_cover_balance_and_order():
    rng = np.random.default_rng(3)
    for nk, world in ((16, 2), (16, 8), (4, 8), (1, 2), (7, 3), (0, 2)):
        costs = rng.uniform(0.8, 1.2, nk) * 40 * 40000
        sh = shard.kpoint_shards(costs, world)
        assert len(sh) == world
        flat = [k for s in sh for k in s]
        assert flat == list(range(nk))                       # disjoint, complete, contiguous, in order
        if nk:
            loads = [costs[s].sum() if s else 0.0 for s in sh]
            assert max(loads) <= costs.sum() / world + costs.max() + 1e-6
    assert shard.kpoint_shards([0.0, 0.0, 0.0], 2) == [[0], [1, 2]]
    with pytest.raises(ValueError):
        shard.kpoint_shards([1.0], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, costs, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.kpoint_shards(costs, world)[rank]
        # stand-in for the per-rank solves: eigenvalues that identify the k-point
        local = {k: np.arange(4, dtype=np.float64) + 10.0 * k for k in mine}
        merged = shard.gather_eigenvalues(local)
        tmax = shard.max_over_ranks(1.5 + rank)
        q.put((rank, sorted(merged), {k: v.tolist() for k, v in merged.items()}, tmax))
    finally:
        dist.destroy_process_group()


def test_two_rank_gather_and_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    costs = [3.0, 1.0, 1.0, 2.0, 2.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, keys, vals, tmax in res:
        assert keys == list(range(len(costs)))               # every k-point, on every rank
        for k in keys:
            assert vals[k] == (np.arange(4) + 10.0 * k).tolist()
        assert tmax == 2.5                                    # the slower rank's time


# ---------------------------------------------------------------- SCF over k-point shards

class _OracleSteps:
    """The SCF steps of shard.scf_sharded() computed by the oracle (dense solves on the CPU), for
    the k-points `kidx` of a workload; grids are CPU tensors so that gloo can reduce them."""

    def __init__(self, wl, kidx, nocc, nev, nk_total):
        from oracle import basis as obasis, scf as oscf
        self.wl, self.nocc, self.nev, self.w = wl, nocc, nev, 1.0 / nk_total
        self.basis = [obasis.sphere(wl.lattice, wl.grid, wl.kfrac[ik], wl.ecut_k[ik]) for ik in kidx]
        self.v = wl.v_r
        self.mixer = oscf.AndersonMixer(wl.lattice, 0.5, 1.0, 8)
        self.lam = self.xs = None

    def update_potential(self, rho):
        from oracle import scf as oscf
        if rho is None:
            self.v = self.wl.v_r
            return 0.0, 0.0
        vhxc, eh, exc = oscf.hxc(rho.numpy(), self.wl.lattice, self.wl.volume)
        self.v = self.wl.v_r + vhxc
        return eh, exc

    def solve(self, n_init):
        import dataclasses
        from oracle import lobpcgf as olb, operator as oop
        w = dataclasses.replace(self.wl, v_r=self.v)
        self.lam, self.xs = [], []
        for m, q in self.basis:
            lam, u, _ = olb.dense_eigs(oop.dense_hamiltonian(w, m, q), w.c, self.nev)
            self.lam.append(lam)
            self.xs.append(u.T.reshape(-1, 4, len(q)))

    def new_grid(self):
        import torch
        return torch.zeros(self.wl.grid, dtype=torch.float64)

    def density(self, rho):
        import torch
        from oracle import scf as oscf
        for x, (m, _) in zip(self.xs, self.basis):
            rho += torch.from_numpy(oscf.density(x[:self.nocc], m, self.wl.grid, self.wl.volume,
                                                 np.full(self.nocc, self.w)))

    def residual(self, a, b):
        return self.wl.volume / self.wl.ng * float((a - b).abs().sum())

    def mix(self, rin, rout, rnext):
        import torch
        rnext.copy_(torch.from_numpy(self.mixer.step(rin.numpy().copy(), rout.numpy().copy())))


_SCF_CASE = dict(name="cubic", ecut=4.0, kfrac=[[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]], nocc=2, nev=8, tol=1e-9)


def _scf_workload():
    import workloads as W
    c = _SCF_CASE
    return W.make(c["name"], ecut=c["ecut"], kfrac=c["kfrac"])


def test_scf_sharded_single_rank_is_the_oracle_loop():
    """One rank holding every k-point runs exactly the oracle's SCF loop."""
    from oracle import scf as oscf
    c = _SCF_CASE
    wl = _scf_workload()
    steps = _OracleSteps(wl, range(wl.nk), c["nocc"], c["nev"], wl.nk)
    out = shard.scf_sharded(steps, tol=c["tol"])
    ref = oscf.scf(wl, c["nocc"], nev=c["nev"], tol=c["tol"])
    assert out["converged"] and ref.converged and out["iterations"] == ref.iterations
    for ik in range(wl.nk):
        assert np.abs(steps.lam[ik] - ref.lam[ik]).max() < 1e-12
    assert np.abs(out["rho"].numpy() - ref.rho).max() < 1e-12 * np.abs(ref.rho).max()
    assert abs(out["e_h"] - ref.history[-1]["eh"]) < 1e-12 * abs(ref.history[-1]["eh"])


def _scf_rank(rank, world, port, q):
    import torch.distributed as dist
    from threadpoolctl import threadpool_limits
    # two ranks whose BLAS thread pools each span every core slow the dense solves to a crawl
    threadpool_limits(max(1, (os.cpu_count() or 2) // world))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = _SCF_CASE
        wl = _scf_workload()
        mine = shard.kpoint_shards([1.0] * wl.nk, world)[rank]
        steps = _OracleSteps(wl, mine, c["nocc"], c["nev"], wl.nk)
        out = shard.scf_sharded(steps, tol=c["tol"])
        q.put((rank, mine, [l.tolist() for l in steps.lam], out["rho"].numpy().copy(), out["iterations"],
               out["converged"]))
    finally:
        dist.destroy_process_group()


def test_scf_sharded_two_ranks_match_single_process():
    """Two gloo ranks, one k-point each: the density all-reduce, rank 0's mixing and the shared
    stopping decision reproduce the single-process loop."""
    import torch.multiprocessing as mp
    pytest.importorskip("threadpoolctl")
    from oracle import scf as oscf
    c = _SCF_CASE
    wl = _scf_workload()
    ref = oscf.scf(wl, c["nocc"], nev=c["nev"], tol=c["tol"])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_scf_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    its = {r[4] for r in res}
    assert len(its) == 1 and all(r[5] for r in res)            # same branch on both ranks
    for rank, mine, lams, rho, _, _ in res:
        assert mine == [rank]
        assert np.abs(np.asarray(lams[0]) - ref.lam[rank]).max() < 1e-10
        assert np.abs(rho - ref.rho).max() < 1e-10 * np.abs(ref.rho).max()
