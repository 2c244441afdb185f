"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): replicas report the slowest
rank's time and the units of all ranks, and the reference arm runs on rank 0 alone."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as tdist
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        # rank r: 10 + 5 r ms for 100 (r + 1) cell-iterations
        t, u = bench.combine_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1), "cpu", world)
        w, rk, _ = bench.dist_env()
        # the reference arm: every rank but 0 leaves at once with status 0
        ref = bench.run_reference(None) if rank != 0 else None
        tdist.barrier()
        q.put((rank, t, u, w, rk, ref))
    finally:
        tdist.destroy_process_group()


def test_replicas_combine_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, t, u, w, rk, ref in out:
        assert (t, u) == (15.0, 300.0)       # max of 10, 15 ms; sum of 100, 200 units
        assert (w, rk) == (2, rank)
        assert ref == (0 if rank == 1 else None)


def test_single_rank_is_unchanged():
    import bench
    assert bench.combine_ranks(12.5, 7.0, "cpu", 1) == (12.5, 7.0)
