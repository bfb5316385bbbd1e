"""The multi-rank (replicas) path of bench.py on CPU: two gloo ranks.

Slices are independent, so ranks never exchange data; they only meet to
take the slowest rank's time, and the reported throughput counts every
rank's slices over that time.  The reference arm prints on rank 0 only.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [100.0 + 50.0 * rank, 2.0 - rank]
    got = bench.max_over_ranks(times, torch.device("cpu"), world)
    v = bench.job_throughput(3, 5, world, got[0])
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, v))


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, v in res:
        assert got == [150.0, 2.0]                  # max over ranks, element-wise
        assert v == pytest.approx(3 * 5 * 2 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], torch.device("cpu"), 1) == [1.5, 2.5]
    assert bench.job_throughput(3, 10, 1, 1000.0) == pytest.approx(30.0)


def test_reference_arm_prints_on_rank_zero_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
