"""The multi-rank path of bench.py on CPU: two gloo ranks, independent replicas, barrier and
max-over-ranks timing, whole-job throughput = units of all ranks / slowest rank's time."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    # rank r "took" 1 + r seconds for 100 * (r + 1) units; its replica's workload differs by rank
    value, t_max, units = bench.aggregate(world, 1.0 + rank, 100.0 * (rank + 1), device="cpu")
    systems = bench.workload(rank)
    out[rank] = (value, t_max, units, float(systems[0].xyz[0, 0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, t_max, units, x0 = out[r]
        assert t_max == 2.0 and units == 300.0 and value == 150.0
    # independent replicas: each rank's cavities are drawn from its own seed
    assert out[0][3] != out[1][3]


def test_single_rank_aggregation_is_identity():
    import bench
    value, t_max, units = bench.aggregate(1, 2.0, 10.0, device="cpu")
    assert (value, t_max, units) == (5.0, 2.0, 10.0)
