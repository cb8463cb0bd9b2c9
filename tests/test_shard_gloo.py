"""Host logic of the multi-rank path with world_size 2 on the gloo backend (CPU): contiguous
shards of independent samples, the gather of per-sample results, and the max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest

from paper_2602_12011_gb300 import shard


def test_shard_bounds_partition():
    for n in (1, 7, 1024, 4099):
        for world in (1, 2, 3, 8):
            b = [shard.shard_bounds(n, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_bounds(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2602_12011_gb300 import workloads as W
        theta = torch.tensor(W.draw_prior(n, 5, 2.0 ** 20))
        lo, hi = shard.shard_bounds(n, rank, world)
        # stand-in per-sample result of this rank's shard (independent of the other rank's)
        local = theta[lo:hi, 0] * 1e-6 + theta[lo:hi, 10] * 1e-3
        full = shard.gather_results(local, n, world)
        t = shard.max_over_ranks(0.5 + rank)
        if rank == 0:
            q.put((full.numpy(), t))
    finally:
        dist.destroy_process_group()


def test_gather_and_max_timing_world2_gloo():
    import torch.multiprocessing as mp
    from paper_2602_12011_gb300 import workloads as W
    n, world = 101, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    full, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    theta = W.draw_prior(n, 5, 2.0 ** 20)
    np.testing.assert_array_equal(full, theta[:, 0] * 1e-6 + theta[:, 10] * 1e-3)
    assert t == 1.5
