"""k-point sharding over ranks (one process per GPU, launched by torch.distributed).

Every k-point is an independent problem -- its own planewave sphere, operator and LOBPCG-F
solve -- so the ranks split the k-points and exchange nothing while they solve.  The split is
contiguous and balanced by the cost of each k-point (nev_k + nbuf) * npw_k (the width of its
blocks times their height); the only collectives are the final gather of the eigenvalues and the
maximum of the per-rank times.  The GPU work itself runs through Context.solve on each rank.
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
