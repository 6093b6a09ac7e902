"""Multi-GPU path (replicas only): each rank runs its own chains with its own
seed; the whole-job value is the proposals of all ranks over the slowest
rank's time.  Exercised here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]
    local_props = [1e6, 3e6][rank]
    value, ms = bench.aggregate(local_ms, local_props)
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_as_replicas():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        value, ms = res[r]
        assert ms == 250.0
        assert value == pytest.approx(4e6 / 0.25)


def test_single_process_aggregate_is_local():
    import bench
    v, ms = bench.aggregate(200.0, 1e6)
    assert ms == 200.0 and v == pytest.approx(5e6)
