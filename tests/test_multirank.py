"""The replica (N > 1) path of bench.py on CPU: two gloo ranks.

Each GPU rank runs its own mixture; the job's time is the slowest rank's (max over ranks)
and the whole-job value is the units of all ranks over that time.  The reference arm runs
on rank 0 only.  These tests exercise that host logic with world size 2 on the gloo
backend (no GPU)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_env()
    local_ms = 10.0 + 5.0 * rank           # rank 1 is the slow one
    mx = bench.reduce_max(local_ms, "cpu")
    value = bench.job_rate(1000.0, w, mx / 1e3)
    dist.barrier()
    out.put((r, w, local, mx, value))
    dist.destroy_process_group()


def test_two_rank_max_and_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time; value counts both ranks' units
    for r, (rank, world, local, mx, value) in enumerate(got):
        assert (rank, world, local) == (r, 2, r)
        assert mx == 15.0
        assert value == pytest.approx(2 * 1000.0 / 0.015)


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.5, "cpu") == 3.5
    assert bench.job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_only_on_rank_zero(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args()) is None   # returns before any oracle work
    assert capsys.readouterr().out == ""
