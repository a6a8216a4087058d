"""The benchmark's multi-rank path on CPU (gloo, world size 2): each rank runs
an independent replica ("replicas only"), the timed region is bracketed by
barriers, the job time is the maximum over ranks, and only rank 0 reports;
the reference arm does its work on rank 0 alone."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup("gloo")
    bench.rank_barrier(w)
    elapsed = 1.0 + rank * 0.5                     # rank 1 is the slow one
    t_max = bench.reduce_max(elapsed, w, "cpu")
    value = bench.job_value(10, w, t_max)
    bench.rank_barrier(w)

    class A:
        gpus, steps, warmup, sample = 2, 1, 3, 8
    if r != 0:
        bench.run_reference(A())                    # must return at once on rank != 0
    q.put((r, w, t_max, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_and_weak_scale():
    port = _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == 1.5 for r in res)                 # max over ranks
    assert all(abs(r[3] - 20 / 1.5) < 1e-12 for r in res)   # steps of all ranks / slowest rank
