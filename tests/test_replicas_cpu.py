"""Multi-GPU path of the benchmark: independent replicas (one beam per rank,
no data exchange), timed by the slowest rank.  Runs two gloo ranks on the CPU:
the reduction and the aggregate throughput are the host logic bench.py uses
under torchrun; each rank's synthetic beam must differ from the others'."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 100.0 + 25.0 * rank           # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms_local, world)
        value = bench.replica_value(3.4e10, 3, ms_max, world)
        x = synth.noise(2, 2, 4096, beam=rank)   # the replica's own beam
        q.put((rank, ms_max, value, float(x[0, :16, 0].sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[1] == 125.0 for r in res)                       # every rank sees the slowest time
    want = world * 3.4e10 * 3 / 0.125 / 1e9                       # all ranks' units over that time
    assert all(np.isclose(r[2], want) for r in res)
    assert res[0][3] != res[1][3]                                 # distinct beams


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert np.isclose(bench.replica_value(1e9, 2, 1000.0, 1), 2.0)
