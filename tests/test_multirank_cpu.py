"""world_size-2 gloo tests on the CPU for the multi-rank pieces: the replica rate
aggregation bench.py uses, and the destination-row-sharded projection protocol (its
multipliers equal the oracle's sort-based projection on the unsharded columns)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import pdmcf as O
from paper_2501_17996_gb300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, fn, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, fn(rank, world)))
    finally:
        dist.destroy_process_group()


def _run(fn, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, fn, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def _replica(rank, world):
    # rank r "processed" 100 (r + 1) iterations in (1 + r) seconds
    return sharding.aggregate_rate(100.0 * (rank + 1), 1.0 + rank, world)


def test_replica_rate_is_total_units_over_slowest_rank():
    out = _run(_replica)
    for rank in (0, 1):
        rate, tmax = out[rank]
        assert tmax == 2.0
        assert rate == pytest.approx((100.0 + 200.0) / 2.0)


def _columns(seed=0, n=37, m=50):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(n, m))
    Q[:, :5] = -np.abs(Q[:, :5])          # columns whose multiplier is 0
    c = rng.uniform(0.2, 3.0, size=m)
    c[5:10] = np.maximum(Q[:, 5:10], 0).sum(axis=0) * 2   # within capacity
    return Q, c


def _sharded(rank, world):
    Q, c = _columns()
    lo, hi = sharding.row_shard(Q.shape[0], world, rank)
    mu = sharding.sharded_mu(torch.from_numpy(Q[lo:hi]), torch.from_numpy(c))
    return mu.numpy()


def test_row_sharded_projection_matches_unsharded_sort():
    out = _run(_sharded)
    Q, c = _columns()
    _, mu_ref = O.project_capped_simplex(Q, c)
    assert np.array_equal(out[0], out[1])            # every rank holds the same multipliers
    assert np.allclose(out[0], mu_ref, rtol=1e-13, atol=1e-14)


def test_row_shards_cover_all_rows():
    for n in (1, 7, 10, 101):
        for world in (1, 2, 3, 8):
            spans = [sharding.row_shard(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
