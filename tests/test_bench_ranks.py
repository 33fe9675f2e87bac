"""The multi-rank bookkeeping of bench.py on CPU (gloo, world size 2).

Under torchrun every rank runs its own replica of the workload; the job's
time is the slowest rank's and its throughput counts the units of all ranks.
Two gloo ranks on 127.0.0.1 check both reductions and the environment parsing.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(HERE))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, w)
    u = bench.sum_over_ranks(100.0 * (rank + 1), w)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, t, u))


def test_slowest_rank_and_summed_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    assert all(o[3] == 15.0 and o[4] == 300.0 for o in out)


def test_single_rank_is_identity():
    import sys

    sys.path.insert(0, os.path.dirname(HERE))
    import bench

    assert bench.max_over_ranks(12.5, 1) == 12.5 and bench.sum_over_ranks(7.0, 1) == 7.0
