"""Host-side logic of bench.py's multi-GPU path (replicas, no data-path collective), run as
two gloo ranks on the CPU: the timings are reduced by their maximum and the whole-job value
counts every rank's elements over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    phase, total = (10.0, 12.0) if rank == 0 else (14.0, 11.0)
    m = bench.max_over_ranks([phase, total], world, torch.device("cpu"))
    out[rank] = (m, bench.job_value(24576, 5, world, m[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_value():
    import torch.multiprocessing as mp
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for r in (0, 1):
        m, v = res[r]
        assert m == [14.0, 12.0]
        assert abs(v - 2 * 24576 * 5 / 0.014) < 1e-6 * v


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, None) == [3.0, 4.0]
    assert bench.job_value(100, 2, 1, 1000.0) == 200.0
