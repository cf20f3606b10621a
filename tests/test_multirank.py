"""The multi-rank side of bench.py on CPU ranks (gloo, world size 2): every rank evaluates its own
replica (the path has no data exchange), the job's time per step is the slowest rank's, and the
whole-job value counts every rank's units over that time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_max = bench.slowest_rank_ms(times[rank], world, "cpu")
        value = bench.job_value(2000, world, t_max)
        dist.barrier()
        q.put((rank, t_max, value))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_report_the_slowest_time_and_the_whole_job_value():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [2.5, 3.25]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in results] == [0, 1]
    for _, t_max, value in results:
        assert t_max == 3.25
        assert value == pytest.approx(2 * 2000 / 3.25e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(4.0, 1, "cpu") == 4.0
    assert bench.job_value(2000, 1, 4.0) == pytest.approx(5e5)
