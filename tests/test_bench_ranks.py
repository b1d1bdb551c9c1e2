"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
builds its own system (weak scaling, distinct seeds), the job's time is the
slowest rank's, and the whole-job value counts every rank's beads.  The GPU
work itself needs a GPU and is covered by the gpu tests and the bench."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    s = bench.workload(r)
    slowest = bench.max_over_ranks(1.5 + rank)  # rank 1 is the slow one
    value = bench.whole_job_value(s.n_beads, 4, w, slowest)
    first = s.snapshot(0)[:64].copy()
    dist.destroy_process_group()
    out.put((r, w, local, s.n_beads, slowest, value, first.tobytes()))


def test_two_ranks_take_the_slowest_time_and_count_all_beads():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, 2, port, out)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, n0, t0, v0, b0), (r1, w1, l1, n1, t1, v1, b1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert n0 == n1 == 1 << 20                 # the same workload size on every rank
    assert b0 != b1                            # but each rank its own system (seed)
    assert t0 == t1 == 2.5                     # the slowest rank's time, on every rank
    assert v0 == v1 == pytest.approx(2 * 4 * (1 << 20) / 2.5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0
    assert bench.reference_arm(Args()) is None
    assert capsys.readouterr().out == ""
