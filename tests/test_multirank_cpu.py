"""The multi-GPU (replica) host logic on CPU ranks with the gloo backend.

Two processes shard a batch the way one-process-per-GPU runs do, decrypt
their slices with the oracle (the GPU kernels need a GPU), gather, and must
reproduce the single-process result; the timing reduction is a max over
ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2512_12904_gb300.shard import shard_mixed, shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from workloads import honest
        wl = honest(1, 4, 24, first_ct=90000, tag=31)
        s, e = shard_range(24, world, rank)
        m = oracle.decrypt(1, wl.u[s:e], wl.v[s:e], wl.y_rows[s:e], nthreads=1)
        parts = [None] * world
        dist.all_gather_object(parts, (s, e, m))
        t = torch.tensor([float(rank + 1)])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        if rank == 0:
            q.put((parts, float(t.item()), wl.m))
    finally:
        dist.destroy_process_group()


def test_shard_range_covers_exactly_once():
    for count in (0, 1, 7, 100, 65536):
        for world in (1, 2, 3, 8):
            got = [shard_range(count, world, r) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == count
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [e - s for s, e in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def test_shard_mixed_balances_levels():
    levels = np.array([1] * 40 + [3] * 35 + [5] * 25)
    np.random.default_rng(0).shuffle(levels)
    parts = [shard_mixed(levels, 4, r) for r in range(4)]
    assert sorted(np.concatenate(parts).tolist()) == list(range(100))
    for p in parts:
        counts = np.bincount(levels[p], minlength=6)[[1, 3, 5]]
        assert (np.abs(counts - np.array([10, 8.75, 6.25])) <= 1).all()


def test_two_gloo_ranks_reproduce_one_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts, tmax, m_all = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = np.concatenate([m for (_, _, m) in sorted(parts, key=lambda x: x[0])])
    assert (got == m_all).all()
    assert tmax == 2.0
