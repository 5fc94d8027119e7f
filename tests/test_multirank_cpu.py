"""Sharding the point set across ranks: each rank forms the unnormalised type-1 sums
of its shard; one SUM all-reduce and a division by the total n give the moments and
right-hand side of the whole set (the sums of Sec. 2.3 are additive over points).
Runs as two gloo ranks on the CPU with the oracle standing in for each rank's GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
import synthetic as S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n, m, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, y = S.wl2_sobolev_2d(n, dtype=np.float64)
    lo, hi = rank * n // world, (rank + 1) * n // world
    T = O.type1(x[:, lo:hi], np.ones(hi - lo), 2 * m)
    b = O.type1(x[:, lo:hi], y[lo:hi], m)
    buf = torch.from_numpy(np.concatenate([T, b]).view(np.float64).copy())
    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    cnt = torch.tensor([float(hi - lo)], dtype=torch.float64)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
    if rank == 0:
        allv = buf.numpy().view(np.complex128) / cnt.item()
        out.put((allv[:len(T)], allv[len(T):], cnt.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_partial_sums_equal_full_moments():
    n, m, world = 3001, 5, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, m, q)) for r in range(world)]
    for p in procs:
        p.start()
    T, b, cnt = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    x, y = S.wl2_sobolev_2d(n, dtype=np.float64)
    assert cnt == n
    assert np.max(np.abs(T - O.moments(x, m))) < 1e-13
    assert np.max(np.abs(b - O.rhs(x, y, m))) < 1e-13
