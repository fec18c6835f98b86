"""The replicas-only multi-GPU path of bench.py on CPU: designs are
independent, so each rank solves its own designs and the ranks only meet for
the barrier and the max-over-ranks of the timings and errors (no data-path
collective).  Two gloo ranks, rendezvous on 127.0.0.1 as under torchrun."""
import multiprocessing as mp
import os
import socket

import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist
    r, w, local = bench.dist_setup(world)
    # rank r's "timings" and "error": the job reports the largest of each
    got = bench.max_over_ranks(w, 1.0 + r, 10.0 - r, 0.5 * r)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, got, bench.rank_seeds(r, 5)))


def test_two_gloo_ranks_take_the_max_and_use_disjoint_designs():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(i, 2, port, q)) for i in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for r, w, local, got, _ in res:
        assert w == 2 and local == r
        assert got == (2.0, 10.0, 0.5)
    assert not set(res[0][4]) & set(res[1][4])


def test_single_rank_needs_no_process_group():
    os.environ.pop("WORLD_SIZE", None)
    assert bench.dist_setup(1)[1] == 1
    assert bench.max_over_ranks(1, 3.0, 4.0) == (3.0, 4.0)


def test_job_rate_is_the_whole_job():
    # 2 ranks x 5 steps x 16 designs in 2 s (the slower rank's time)
    assert bench.job_rate(2, 5, 16, 2.0) == 80.0
