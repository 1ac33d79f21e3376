"""Multi-rank host logic of bench.py on the CPU (gloo, world size 2).

The solve does not shard across GPUs: at N > 1 every rank solves its own replica and the step
time is the maximum over ranks. These tests run that reduction and the rank handling as two gloo
processes on 127.0.0.1, with no GPU.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    try:
        w, r, local = bench.dist_setup(None)
        dist.init_process_group("gloo", rank=r, world_size=w)
        # rank-dependent timings: rank 1 is slower on the first entry, rank 0 on the second
        got = bench.max_over_ranks([10.0 + rank, 5.0 - rank, 7.25], w)
        dist.barrier()
        # the reference arm: only rank 0 runs the oracle; the others return at once without work
        ref = bench.run_reference(None, w, r) if r != 0 else "rank0"
        dist.destroy_process_group()
        q.put((rank, (w, r, local), got, ref))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, "error", repr(e), None))


def test_max_over_ranks_and_rank_handling_with_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    for rank, env, got, ref in res:
        assert env != "error", got
        assert env == (world, rank, rank)
        assert got == [11.0, 5.0, 7.25]  # the same maximum on every rank
        assert ref == ("rank0" if rank == 0 else None)
    assert all(p.exitcode == 0 for p in procs)


def test_max_over_ranks_is_the_identity_at_world_size_one():
    import bench
    assert bench.max_over_ranks([3, 1.5], 1) == [3.0, 1.5]
