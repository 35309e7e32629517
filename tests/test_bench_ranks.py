"""CPU tests of the benchmark's multi-replica path: world size 2 over gloo (no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each replica times its own steps; the job takes the slowest one
        own_ms = 100.0 + 25.0 * rank
        total = bench.max_over_ranks(own_ms, world, device="cpu")
        value = bench.job_value(world, 5, 1e9, total)
        out.put((rank, total, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_world_2():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, total, value in res:
        assert total == 125.0                      # the slower replica's time on both ranks
        assert abs(value - 2 * 5 * 1e9 / 0.125 / 1e9) < 1e-9  # both replicas' bytes / that time


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.job_value(1, 2, 3e9, 1000.0) == 6.0


def test_reference_arm_runs_on_rank_0_only(capsys):
    """Under torchrun the oracle's arm is timed on rank 0; the other ranks exit without work."""
    import types

    import bench

    args = types.SimpleNamespace(n=30, steps=1, warmup=1, gpus=2)
    assert bench.run_reference(args, 1, 2) is None
    assert capsys.readouterr().out == ""
