"""Host logic of the multi-rank path with world_size 2 on the gloo backend (CPU): contiguous
shards of independent samples, each rank evaluating the log-likelihood of its own shard (the
oracle's, on a tiny grid, standing in for one GPU's batched call), the gather of the per-sample
results, and the max-over-ranks timing."""
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


def _problem(n):
    from oracle import oracle as O
    from paper_2602_12011_gb300 import workloads as W
    T = 2.0 ** 12
    k0, nb = W.grid(T)
    inj = W.theta_injection(T)
    f = (k0 + np.arange(nb)) / T
    od = O.Detector(W.LISA, T, k0, nb, O.make_data(W.LISA, inj, W.MODE_ALL, T, k0, nb, W.normals(nb, 4)),
                    O.psd(W.LISA, f))
    return O, od, W.draw_prior(n, 5, T), W.MODE_ALL


def _rank_loglike(rank, world, n):
    """log L of this rank's contiguous shard only."""
    O, od, theta, mask = _problem(n)
    lo, hi = shard.shard_bounds(n, rank, world)
    return O.loglike_batch([od], theta[lo:hi], mask, nthreads=1)[0]


def _worker(rank, world, port, n, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ll_local = _rank_loglike(rank, world, n)
        full = shard.gather_results(torch.tensor(ll_local), n, world)
        t = shard.max_over_ranks(0.5 + rank)
        if rank == 0:
            q.put((full.numpy(), t))
    finally:
        dist.destroy_process_group()


def test_gather_and_max_timing_world2_gloo():
    import torch.multiprocessing as mp
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
    O, od, theta, mask = _problem(n)
    np.testing.assert_array_equal(full, O.loglike_batch([od], theta, mask, nthreads=1)[0])
    assert t == 1.5
