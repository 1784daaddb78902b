"""The multi-GPU path of bench.py is replicas only: every rank advances its own
run, and the only collective is the MAX of the timed region over ranks.  This
checks that host logic with two gloo ranks on the CPU (no GPU): the job time is
the slowest rank's on every rank, the whole-job value counts every replica, and
the reference arm prints only on rank 0; the oracle step timer of the CPU
baseline reads steps, not timing noise."""
import io
import os
import socket
import sys
import contextlib

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 2.0 * rank                 # rank 1 is the slow one
        ms = bench.job_time_ms(local_ms, world, "cpu")
        value = bench.job_value(world, 1000, 50, ms)
        out.put((rank, ms, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_value_counts_every_replica():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 12.0, (rank, ms)
        assert value == pytest.approx(2 * 1000 * 50 / 0.012)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(7.5, 1, "cpu") == 7.5
    assert bench.job_value(1, 10, 4, 2.0) == pytest.approx(10 * 4 / 0.002)


def test_reference_arm_prints_only_on_rank_zero(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"steps": 1, "warmup": 0, "diag_every": 1, "gpus": 2, "deposit_mode": "atomic"})()
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, W.bump_on_tail())
    assert buf.getvalue() == ""


def test_oracle_step_timer_reads_steps_not_noise():
    """The CPU baseline's per-step time is [t(M+1 steps) - t(1 step)]/M with
    M = max(K, 50) for the P1 fields: even at K = 2 the rate is a plausible
    single-core figure, not the run-to-run spread of the one-time dense LU
    divided by two steps."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    spec = W.bump_on_tail()
    n, secs, used, m = bench.time_oracle(spec, 4, 2, 0, 1, threads=1)
    assert (n, used, m) == (4 * spec.lattice.nv, 1, 50)
    rate = n * 2 / secs
    assert 0.0 < rate < 1e10, rate
