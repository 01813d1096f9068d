"""Multi-GPU runs of bench.py are replicas (one independent reduced system
per rank, no data-path collective): the whole-job step time is the slowest
rank's, the value counts every rank's right-hand sides, and the reference arm
prints from rank 0 only.  Exercised with two gloo ranks on the CPU."""
import io
import os
import socket
import contextlib

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    v = bench.job_value(ws, 128, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_two_gloo_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]                      # max over ranks
    assert out[0][2] == pytest.approx(2 * 128 / 0.015)              # whole-job RHS/s


def test_single_process_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5, "cpu") == 7.5
    assert bench.job_value(1, 128, 100.0) == pytest.approx(1280.0)


def test_reference_arm_is_silent_off_rank_zero(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args())
    assert buf.getvalue() == ""
