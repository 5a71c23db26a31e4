"""The benchmark's multi-rank logic on CPU with two gloo ranks: disjoint
Philox counter ranges and seeds per rank, and the whole-job reduction (the
slowest rank's time, the bunches of all ranks)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed, base = bench.shard(rank, 1000, 2)
        t_local = 1.0 + rank * 0.5            # rank 1 is slower
        b_local = 100.0 * (rank + 1)
        t, b = bench.reduce_over_ranks(t_local, b_local, world, "cpu")
        q.put((rank, seed, base, t, b))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, b0, t0, n0), (r1, s1, b1, t1, n1) = res
    assert (s0, s1) == (2, 3)                     # independent showers
    assert (b0, b1) == (0, 1000)                  # disjoint Philox counters
    assert t0 == t1 == pytest.approx(1.5)         # max over ranks
    assert n0 == n1 == pytest.approx(300.0)       # sum over ranks


def test_single_rank_is_identity():
    assert bench.reduce_over_ranks(2.0, 7.0, 1, "cpu") == (2.0, 7.0)
