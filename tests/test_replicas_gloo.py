"""The multi-GPU path of the benchmark is N independent replicas (one grid per
rank, no data-path collective): the job's time is the slowest rank's, its
throughput N x the units of one rank over that time, and only rank 0 runs the
CPU reference arm. Checked here with world_size 2 over gloo on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [125.0, 80.0][rank]
        ms = bench.max_over_ranks(local_ms, device="cpu")
        rate = bench.replicated_rate(10, ms, world)
        # the reference arm: ranks other than 0 leave without work
        ref = None
        if rank != 0:
            ref = bench.run_reference(None, "coarse-fp64", bench.WORKLOADS["coarse-fp64"])
        out[rank] = (ms, rate, ref)
    finally:
        dist.destroy_process_group()


def test_replicas_time_is_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 125.0
    assert res[0][1] == res[1][1] == pytest.approx(world * 10 / 0.125)
    assert res[1][2] == 0


def test_single_process_is_its_own_max():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, device="cpu") == 3.5
    assert bench.replicated_rate(20, 1000.0, 1) == pytest.approx(20.0)
