"""The N > 1 host logic of bench.py on two gloo ranks (CPU): process-group set-up from the
launcher's environment, the barrier, the max-over-ranks step time and the whole-job
throughput; and the reference arm's rank rule (rank 0 alone does the work)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup(world)
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    # rank k took 10 (k + 1) ms for a step of 3 GB of its own work
    gbs, ms = bench.job_throughput(w, 3e9, 10.0 * (rank + 1))
    bench.barrier(w)
    q.put((rank, gbs, ms))
    dist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_and_sum_the_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, gbs, ms in got:
        assert ms == 20.0                       # max over ranks
        assert abs(gbs - 2 * 3e9 / 20e-3 / 1e9) < 1e-9   # both ranks' bytes / slowest time


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    gbs, ms = bench.job_throughput(1, 1e9, 4.0)
    assert ms == 4.0 and abs(gbs - 250.0) < 1e-9


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 3
    # a non-zero rank returns at once without touching the oracle or a GPU
    assert bench.run_reference(A(), 2, 1) == 0
