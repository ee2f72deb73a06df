"""Multi-rank host logic of bench.py (replicas only): with N ranks each
timing its own lattice, the line reports the slowest rank's time and the sum
of all ranks' link updates.  Runs world_size 2 on CPU with the gloo backend;
no GPU and no data-path collective is involved."""
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
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs = [1.5, 2.25][rank]
    units = [100.0, 300.0][rank]
    t, u = bench.reduce_max_sum(world, secs, units, torch.device("cpu"))
    bench.barrier(world)
    out[rank] = (t, u)
    dist.destroy_process_group()


def test_max_time_and_summed_units_over_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.25, 400.0)


def test_single_rank_is_identity():
    import torch
    import bench
    assert bench.reduce_max_sum(1, 3.0, 7.0, torch.device("cpu")) == (3.0, 7.0)
