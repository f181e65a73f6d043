"""Host-side logic of the multi-rank bench (replicas, weak scaling) on CPU.

Two gloo ranks: each draws its own block of the seeded field stream, and the
step time that rank 0 reports is the maximum over ranks.  No GPU is used; the
data path has no collective (every rank transforms its own fields).
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2004_11346_gb300 import inputs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = bench.workload("fp64_N64")
    fields = bench.rank_fields(8, 2, w, rank)
    times = [10.0 + rank, 3.0 * (1 - rank), 7.0]
    got = bench.reduce_max(times, world, device="cpu")
    q.put((rank, fields, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, (f, g)) for r, f, g in (q.get(timeout=120) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # max over ranks
    assert res[0][1] == res[1][1] == [11.0, 3.0, 7.0]
    # rank r's fields are fields 2r, 2r+1 of the single-rank stream
    all4 = inputs.coefficients(8, 4, 0, real_m0=True)
    np.testing.assert_array_equal(res[0][0], all4[:2])
    np.testing.assert_array_equal(res[1][0], all4[2:])


def test_single_rank_reduce_is_identity():
    assert bench.reduce_max([1.0, 2.0], 1) == [1.0, 2.0]
