"""World-size-2 run of the multi-rank host logic on CPU (gloo): each rank
computes the stencils of its own target range (oracle arithmetic stands in for
the GPU work here), rank 0 gathers them and checks they equal the single-rank
result, and the step-time reduction returns the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2104_14447_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch

    import oracle
    from paper_2104_14447_gb300 import inputs

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = inputs.jittered_grid(2, 24, seed=1)
    n = x.shape[1]
    b, e = shard.shard_targets(n, rank, world)
    tg = np.arange(b, e, dtype=np.int32)
    idx, eps = oracle.knn(x, tg, 12, 1.5)
    off = np.arange(0, len(tg) * 12 + 1, 12)
    w, _, _ = oracle.stencils(x, tg, off, idx.reshape(-1), eps, "scalar", 2, "laplacian")
    parts = [None] * world
    dist.all_gather_object(parts, (b, e, w))
    slowest = shard.max_over_ranks(10.0 + rank)
    if rank == 0:
        out.put((parts, slowest, n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_equals_single_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts, slowest, n = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert slowest == 11.0
    assert parts[0][0] == 0 and parts[0][1] == parts[1][0] and parts[1][1] == n
    import oracle
    from paper_2104_14447_gb300 import inputs

    x = inputs.jittered_grid(2, 24, seed=1)
    tg = np.arange(n, dtype=np.int32)
    idx, eps = oracle.knn(x, tg, 12, 1.5)
    w, _, _ = oracle.stencils(x, tg, np.arange(0, n * 12 + 1, 12), idx.reshape(-1), eps, "scalar", 2, "laplacian")
    assert np.array_equal(np.concatenate([parts[0][2], parts[1][2]]), w)


@pytest.mark.parametrize("n,world", [(10, 3), (7, 7), (5, 8), (262144, 8)])
def test_shard_ranges_cover_exactly(n, world):
    ranges = [shard.shard_targets(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    sizes = [e - b for b, e in ranges]
    assert max(sizes) - min(sizes) <= 1
    assert shard.job_throughput(100, 2, world, 1000.0) == 200 * world
