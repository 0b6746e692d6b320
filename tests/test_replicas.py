"""Multi-GPU runs are independent replicas (one process per GPU, no
collective on the solve path).  The only cross-rank step is the benchmark's
timing: the job's step time is the maximum over ranks and the job's value
counts the units of every rank.  Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [120.0, 180.0][rank]                 # rank 1 is the slow one
    step = bench.max_over_ranks(local)
    out[rank] = (step, bench.whole_job_value(1000, world, step))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 180.0
    assert res[0][1] == res[1][1] == pytest.approx(1000 * 2 / 0.180)


def test_single_process_keeps_its_own_time():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.whole_job_value(10, 1, 1000.0) == 10.0
