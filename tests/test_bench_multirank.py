"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
builds its own replica, so the job's value is the units of all ranks over
the slowest rank's time, and only rank 0 runs the CPU reference arm."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed 1000 (r + 1) units in 0.5 + r seconds
        units, sec = bench.reduce_job(1000 * (rank + 1), 0.5 + rank, dist, "cpu")
        out.put((rank, units, sec))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_reduce_job_sums_units_and_takes_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, units, sec in got:
        assert units == 3000.0 and sec == 1.5, (rank, units, sec)


def test_reduce_job_without_a_group_passes_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_job(123, 0.25) == (123.0, 0.25)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = bench.argparse.Namespace(workload="uniform_1e5", steps=1, warmup=0, gpus=2)
    called = []
    monkeypatch.setattr(bench, "make_scene", lambda w: called.append(w))
    bench.run_reference(args, 1, 2)   # rank 1: no work, no output
    assert called == [] and capsys.readouterr().out == ""
