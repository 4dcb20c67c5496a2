"""k-point sharding over ranks (one process per GPU, launched by torch.distributed).

Every k-point is an independent problem -- its own planewave sphere, operator and LOBPCG-F
solve -- so the ranks split the k-points and exchange nothing while they solve.  The split is
contiguous and balanced by the cost of each k-point (nev_k + nbuf) * npw_k (the width of its
blocks times their height); the only collectives of a solve are the final gather of the
eigenvalues and the maximum of the per-rank times.  The GPU work itself runs through
Context.solve on each rank.

The SCF loop (Sec. 2.1 density, Sec. 4.1 mixing) couples the k-points through the density:
rho = sum_k w_k rho_k.  Sharded, each rank adds the densities of its own k-points and one
sum-all-reduce of the grid per SCF iteration forms rho on every rank (the loop's one real
exchange step); rank 0 mixes and broadcasts the next input density, and the stopping decision
uses the largest residual over the ranks, so every rank takes the same branch.  scf_sharded()
is that loop over any object with the SCF steps (ContextSCF: the library on this rank's GPU).
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np


def kpoint_shards(costs: Sequence[float], world: int) -> List[List[int]]:
    """Contiguous blocks of k-point indices, one per rank, balanced by cost: rank r takes the
    k-points whose cumulative cost midpoint falls in [r, r + 1) * total / world.  Every k-point is
    in exactly one block; a rank may get none when there are fewer k-points than ranks."""
    if world < 1:
        raise ValueError("world size must be positive")
    c = np.asarray(costs, dtype=np.float64)
    if c.ndim != 1 or np.any(c < 0):
        raise ValueError("costs must be a list of non-negative numbers")
    out: List[List[int]] = [[] for _ in range(world)]
    total = float(c.sum())
    if len(c) == 0:
        return out
    if total <= 0.0:
        c = np.ones_like(c)
        total = float(len(c))
    mid = np.cumsum(c) - 0.5 * c
    for ik, x in enumerate(mid):
        r = min(world - 1, int(x * world / total))
        out[r].append(ik)
    return out


def gather_eigenvalues(local: Dict[int, np.ndarray], group=None) -> Dict[int, np.ndarray]:
    """Every rank's {k-point: eigenvalues} merged on all ranks (one all_gather_object)."""
    import torch.distributed as dist
    parts: list = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, {int(k): np.asarray(v).tolist() for k, v in local.items()}, group=group)
    merged: Dict[int, np.ndarray] = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise RuntimeError(f"k-point {k} solved on two ranks")
            merged[k] = np.asarray(v, dtype=np.float64)
    return merged


def max_over_ranks(x: float, group=None) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    backend = dist.get_backend(group)
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def _dist_on(group=None):
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized()


def allreduce_sum_(t, group=None):
    """In-place sum of a tensor over the ranks (NCCL for device tensors, gloo for host ones)."""
    if _dist_on(group):
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def broadcast_(t, src=0, group=None):
    if _dist_on(group):
        import torch.distributed as dist
        dist.broadcast(t, src, group=group)
    return t


def scf_sharded(steps, tol=1e-8, max_iter=60, n_init=3, n_init_warm=1, group=None):
    """The SCF loop over k-point shards.  `steps` provides, for this rank's k-points:
        update_potential(rho or None) -> (E_H, E_xc)   V = V_loc + V_hxc(rho)
        solve(n_init)                                   eigenpairs of the current potential
        new_grid()                                      a zeroed density grid
        density(rho)                                    rho += sum_{local k} w_k rho_k
        residual(a, b) -> float                         int |a - b| dr
        mix(rho_in, rho_out, rho_next)                  one Anderson-Kerker step (rank 0 only)
    Returns dict(converged, iterations, residual, history, e_h, e_xc, rho) on every rank; rho is
    the last output density (identical on all ranks)."""
    import torch.distributed as dist
    rank = dist.get_rank(group) if _dist_on(group) else 0
    steps.update_potential(None)
    steps.solve(n_init)
    rho_in = steps.new_grid()
    steps.density(rho_in)
    allreduce_sum_(rho_in, group)
    out = dict(converged=False, iterations=0, residual=float("inf"), history=[], e_h=0.0, e_xc=0.0, rho=rho_in)
    for it in range(1, max_iter + 1):
        out["e_h"], out["e_xc"] = steps.update_potential(rho_in)
        steps.solve(n_init_warm)
        rho_out = steps.new_grid()
        steps.density(rho_out)
        allreduce_sum_(rho_out, group)
        res = steps.residual(rho_out, rho_in)
        if _dist_on(group):
            res = max_over_ranks(res, group)
        out.update(iterations=it, residual=res, rho=rho_out)
        out["history"].append(res)
        if res < tol:
            out["converged"] = True
            break
        if rank == 0:
            steps.mix(rho_in, rho_out, rho_in)
        broadcast_(rho_in, 0, group)
    return out


class ContextSCF:
    """The SCF steps of scf_sharded() through the library, for the k-points of one Context (the
    rank's shard).  xs: its complex128 blocks [nev + nbuf, ncomp, npw] (start block in, last
    eigenvectors out); nk_total: k-points of the whole job (weight 1 / nk_total each); nocc
    occupied states per k-point; solve_kw: options of Context.solve."""

    def __init__(self, ctx, xs, nev, nocc, nk_total, history=8, alpha=0.5, q0=1.0, stream=None, **solve_kw):
        self.ctx, self.xs, self.nev, self.nocc = ctx, xs, int(nev), int(nocc)
        self.w = 1.0 / float(nk_total)
        self.stream = stream
        self.kw = dict(solve_kw)
        self.mixer = ctx.mixer(history, alpha, q0)
        self.lam = None

    def update_potential(self, rho):
        return self.ctx.update_potential(rho, stream=self.stream)

    def solve(self, n_init):
        lam, rep, rc = self.ctx.solve(self.xs, self.nev, n_init=n_init, check=False, stream=self.stream,
                                      **self.kw)
        if rc not in (0, -4):                 # an eigensolve that ends NOT_CONVERGED does not stop the loop
            from . import DKSError
            raise DKSError(rc, rep["message"])
        self.lam = lam

    def new_grid(self):
        import torch
        return torch.zeros(self.ctx.grid, dtype=torch.float64, device="cuda")

    def density(self, rho):
        occ = [self.w] * self.nocc
        for ik in range(self.ctx.nk):
            self.ctx.density(ik, self.xs[ik], occ, rho, stream=self.stream)

    def residual(self, a, b):
        return self.ctx.density_residual(a, b, stream=self.stream)

    def mix(self, rho_in, rho_out, rho_next):
        self.mixer.step(rho_in, rho_out, rho_next, stream=self.stream)
