"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks (one
process each, 127.0.0.1 rendezvous) agree on the slowest rank's time and
on the whole-job throughput; the reference arm does no work off rank 0."""
import io
import contextlib
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        ms_local = 10.0 + 5.0 * rank
        ms_max = bench.max_over_ranks(ms_local, torch.device("cpu"))
        q.put((rank, ms_max, bench.job_rate(world, 3 * 10**8, ms_max)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms_max, rate in got:
        assert ms_max == 15.0
        assert rate == pytest.approx(2 * 3e8 / 15e-3 / 1e9)   # 40 Gpoints/s over the job


def test_single_process_max_is_identity():
    import torch
    assert bench.max_over_ranks(7.5, torch.device("cpu")) == 7.5
    assert bench.job_rate(1, 3e8, 15.0) == pytest.approx(20.0)


def test_reference_arm_is_silent_off_rank_zero(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    class A:
        gpus, steps, warmup, seed, n = 2, 1, 0, 1, 10**8
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(A())
    assert out.getvalue() == ""
