"""The N > 1 host path of bench.py on CPU: two gloo ranks run independent
replicas (no data-path collective), the timing is the maximum over ranks and
only rank 0 reports."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench._dist()
        assert (w, r) == (world, rank)
        # each rank times its own replica; the reported time is the slowest rank's
        ms = 10.0 + 5.0 * rank
        bench._barrier(dist)
        t = bench._max_over_ranks(dist, ms, torch.device("cpu"))
        out[rank] = t
        # whole-job throughput counts every rank's units
        out[world + rank] = 1000.0 * world / t
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_timing():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Array("d", 2 * world)
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert list(out[:world]) == [15.0, 15.0]
    assert out[world] == pytest.approx(1000.0 * 2 / 15.0)


def test_reference_arm_nonzero_rank_exits_quietly(capsys, monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 0, 2

    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
