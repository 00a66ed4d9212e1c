"""Host logic of the benchmark's multi-process path on CPU: world_size-2 gloo
ranks agree on the job time (the slowest rank's) and on the whole-job value."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, device="cpu")
    dist.barrier()
    q.put((rank, ms, bench.job_throughput(1000, 4, world, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [15.0, 15.0]
    assert all(g[2] == pytest.approx(1000 * 4 * 2 / 0.015) for g in got)


def test_single_process_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(10, 3, 1, 30.0) == pytest.approx(1000.0)


def test_a_failing_side_leg_is_reported_in_its_place():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.side_leg("ok", lambda: {"v": 1}) == {"v": 1}

    def boom():
        raise RuntimeError("no such kernel")
    got = bench.side_leg("batched", boom)
    assert got == {"error": "batched: RuntimeError: no such kernel"}
