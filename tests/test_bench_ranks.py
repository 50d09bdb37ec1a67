"""The replica path of bench.py on CPU: two processes over the gloo backend
(127.0.0.1) reduce their step times to the slowest rank's, and the job's
throughput counts every rank's replica."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        dist.barrier()
        out.put((rank, ms, bench.job_throughput(world, 3, 72, 1000, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank_and_the_job_throughput():
    import torch.multiprocessing as mp
    if not dist.is_gloo_available():
        pytest.skip("gloo backend not built")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [7.5, 9.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [9.0, 9.0]
    # 2 replicas x 3 solves x 72 cycles x 1000 updates in 9 ms
    assert res[0][2] == pytest.approx(2 * 3 * 72 * 1000 / 9e-3)


def test_one_process_needs_no_reduction():
    import bench
    assert bench.max_over_ranks(4.25, None, "cpu") == 4.25
    assert bench.job_throughput(1, 10, 72, 14702584, 70.2) == pytest.approx(
        10 * 72 * 14702584 / 0.0702)
