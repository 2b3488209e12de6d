"""The multi-GPU path of the bench runs independent replicas (no data-path
collective): the only cross-rank steps are the barrier and the max over ranks
of the step time.  Checked here with two gloo ranks on the CPU."""
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
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.0, 15.5][rank]                       # rank 1 is the slow one
    ms_max = bench.max_over_ranks(dist, ms, "cpu")
    dist.barrier()
    out[rank] = (ms_max, bench.replica_value(world, 1000, ms_max))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (15.5, pytest.approx(2 * 1000 / 15.5e-3))


def test_single_rank_needs_no_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.0, "cpu") == 3.0
    assert bench.replica_value(1, 10, 2.0) == pytest.approx(5000.0)
