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
