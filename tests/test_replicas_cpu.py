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


def _shard_rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    import oracle
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _shard_workload(synth)
        nd = oracle.overlap(w.nsub, w.f_centre, w.bw, w.dms, w.nchan, w.nint, w.nbin)   # the whole band's
        lo, hi = bench.subband_slice(w.nsub, world, rank)
        v = bench.slice_view(w, lo, hi)
        x = w.voltages(threads=1, sub=(lo, hi))
        fb = oracle.filterbank(x, v.f_centre, v.bw, v.dms, v.nchan, v.nint, v.nbin, nd, nthreads=1)
        S, nseg, _ = oracle.grid(w.nsamp, w.nbin, w.nchan, nd, w.nint)
        units = len(w.dms) * (hi - lo) * nseg * S
        q.put((rank, lo, hi, fb, bench.sum_over_ranks(units, world), nd))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _shard_workload(synth):
    # 5 subbands (an uneven split over 2 ranks: 3 + 2), one pulse, N = 2^11, 8 channels
    return synth.Workload("split", 5, 1 << 14, 135.0, 0.1953125, (0.0, 4.0, 8.0), 8, 4, 1 << 11, 7,
                          (synth.Pulse(0.03, 6.0, 1e-3, 0.5),))


def test_subband_split_union_is_the_whole_filterbank():
    """One beam's subbands split across two gloo ranks (bench.py --shard subbands):
    each rank generates only its slice of the voltages and computes its rows with
    the whole band's overlap; the slices' rows together are the single-rank
    filterbank exactly (subbands are independent, Sec. 4), and the ranks' units
    add up to the whole beam's."""
    import oracle
    import synth
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = _shard_workload(synth)
    nd = res[0][5]
    full = oracle.filterbank(w.voltages(threads=1), w.f_centre, w.bw, w.dms, w.nchan, w.nint, w.nbin, nd)
    assert [(r[1], r[2]) for r in res] == [(0, 3), (3, 5)]
    union = np.concatenate([r[3] for r in res], axis=1)
    assert union.shape == full.shape and np.array_equal(union, full)
    S, nseg, _ = oracle.grid(w.nsamp, w.nbin, w.nchan, nd, w.nint)
    assert all(r[4] == len(w.dms) * w.nsub * nseg * S for r in res)


def test_subband_slices_cover_the_band():
    import bench
    for nsub, world in [(64, 8), (64, 3), (5, 2), (7, 7), (3, 4)]:
        sl = [bench.subband_slice(nsub, world, r) for r in range(world)]
        assert sl[0][0] == 0 and sl[-1][1] == nsub
        assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
        sizes = [hi - lo for lo, hi in sl]
        assert max(sizes) - min(sizes) <= 1
