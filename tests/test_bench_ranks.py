"""The multi-rank path of bench.py on the CPU: two gloo ranks take the
slowest rank's time and report the units of both (weak scaling, instances
are independent, no data-path collective); the reference arm runs on rank 0
only.  No GPU involved."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    v = bench.job_value(world, 1024, 3, ms)
    dist.barrier()
    q.put((rank, ms, v))
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_time_and_all_units():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, v in out:
        assert ms == 15.0
        assert v == pytest.approx(2 * 1024 * 3 / 0.015)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_value(1, 1024, 10, 500.0) == pytest.approx(20480.0)


def test_reference_arm_only_on_rank_zero(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    class A:  # the fields reference_arm reads
        batch, cpu_sample, warmup, steps, gpus = 1024, 4, 1, 1, 2
    bench.reference_arm(A())
    assert capsys.readouterr().out == ""
