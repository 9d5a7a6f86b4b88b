"""The multi-rank path of bench.py on the CPU (gloo, world size 2): every
rank evaluates its own replica, the step time is the slowest rank's and the
job rate counts the atoms of all replicas; the reference arm runs on rank 0
only.  No GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [3.0, 5.0][rank]
        ms = bench.max_over_ranks(local_ms, world, device="cpu")
        out[rank] = (ms, bench.job_rate(world, 1000, ms), bench._dist())
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_step_and_sum_the_atoms():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    for rank in range(2):
        ms, rate, (r, w) = res[rank]
        assert ms == 5.0                       # the slower rank decides
        assert rate == pytest.approx(2 * 1000 / 5e-3)
        assert (r, w) == (rank, 2)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.0, 1) == 4.0
    assert bench.job_rate(1, 1000, 4.0) == pytest.approx(250000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"gpus": 2, "steps": 1, "warmup": 0})()
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
