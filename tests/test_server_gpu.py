"""Streaming server: blocks of several beams, continuously batched.

A beam streamed block by block must give exactly the filterbank of the
offline plan on its whole input (the same overlap-save segments through the
same kernels, so bit-identical); a beam's results must be the same alone and
in a mix with other beams whose blocks overlap on the GPU; int8 blocks must
match their dequantised float equivalent; admission must refuse a beam that
does not fit the HBM budget; a wait that cannot finish must time out.
"""
import numpy as np
import pytest

import synth
from helpers import rel_errors

pytestmark = pytest.mark.gpu
BW = 0.1953125


@pytest.fixture(scope="module")
def cdmt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_00909_gb300 as m
    return m


# block lengths below, at and above N, so that some blocks complete no segment
BEAMS = [
    dict(nsub=2, block_len=1 << 14, f_centre=135.0, dm_first=0.0, dm_step=2.0, ndm=6, nchan=8, nint=4, seed=51),
    dict(nsub=3, block_len=3 << 13, f_centre=150.0, dm_first=1.0, dm_step=1.5, ndm=5, nchan=16, nint=8, seed=52),
    dict(nsub=1, block_len=1 << 15, f_centre=120.0, dm_first=0.0, dm_step=5.0, ndm=3, nchan=8, nint=2, seed=53),
]
NBLK = 8


def _serve(cdmt, beams, inputs, interleave=True, i8=False, scales=None, precision=None, max_slots=0, keep_parts=False):
    import torch
    precision = cdmt.CDMT_PREC_FP16 if precision is None else precision
    srv = cdmt.Server(max_slots=max_slots)
    ids = [srv.add_beam(b["nsub"], b["block_len"], b["f_centre"], BW, b["dm_first"], b["dm_step"], b["ndm"],
                        b["nchan"], b["nint"], precision=precision,
                        in_dtype=cdmt.CDMT_IN_I8 if i8 else cdmt.CDMT_IN_C64, dm_tile=b["ndm"]) for b in beams]
    blocks = []
    for b, x in zip(beams, inputs):
        L = b["block_len"]
        blocks.append([torch.from_numpy(np.ascontiguousarray(x[:, k * L:(k + 1) * L])).pin_memory()
                       for k in range(NBLK)])
    sc = [torch.from_numpy(s).pin_memory() for s in scales] if scales is not None else None
    order = [(k, bi) for k in range(NBLK) for bi in range(len(beams))] if interleave else \
        [(k, bi) for bi in range(len(beams)) for k in range(NBLK)]
    reqs = [(bi, k, srv.submit(ids[bi], blocks[bi][k].data_ptr(), sc[bi].data_ptr() if sc else 0))
            for k, bi in order]
    parts = [dict() for _ in beams]
    for bi, k, rid in reqs:
        res = srv.wait(rid, 120.0)
        b = beams[bi]
        assert res.beam == ids[bi] and res.index == k
        if res.samples > 0:
            parts[bi][res.first_sample] = srv.block_view(res, b["ndm"], b["nsub"] * b["nchan"]).cpu().numpy()
        srv.release(rid)
    st = srv.stats()
    srv.close()
    if keep_parts:
        return parts, st
    out = []
    for p in parts:
        keys = sorted(p)
        pos = 0
        for k in keys:  # the blocks tile the output with no gap or overlap
            assert k == pos
            pos += p[k].shape[2]
        out.append(np.concatenate([p[k] for k in keys], axis=2))
    return out, st


def _offline(cdmt, b, x, precision):
    import torch
    dms = [b["dm_first"] + i * b["dm_step"] for i in range(b["ndm"])]
    p = cdmt.Plan(b["nsub"], x.shape[1], b["f_centre"], BW, dms, b["nchan"], b["nint"], nbin=4096 * b["nchan"],
                  dm_tile=b["ndm"], precision=precision)
    out = cdmt.run(p, torch.from_numpy(np.ascontiguousarray(x)).cuda()).cpu().numpy()
    p.close()
    return out


def _inputs(beams):
    xs = [synth.noise(b["seed"], b["nsub"], NBLK * b["block_len"]) for b in beams]
    synth.add_pulses(xs[0], [synth.Pulse(0.4, 6.0, 1e-3, 0.5)], beams[0]["f_centre"], BW, beams[0]["seed"])
    return xs


@pytest.mark.parametrize("prec", ["fp16", "fp32"])
def test_stream_equals_offline_and_mix_equals_alone(cdmt, prec):
    precision = cdmt.CDMT_PREC_FP16 if prec == "fp16" else cdmt.CDMT_PREC_FP32
    xs = _inputs(BEAMS)
    # two output slots: blocks wait for a free slot, so dispatch order and slot reuse are exercised
    mixed, st = _serve(cdmt, BEAMS, xs, interleave=True, precision=precision, max_slots=2)
    assert st.blocks_done == NBLK * len(BEAMS) and st.slots == 2
    assert 0 < st.latency_p50_ms <= st.latency_p99_ms <= st.latency_max_ms
    assert st.realtime_factor > 0 and st.units_per_s > 0
    for bi, (b, x) in enumerate(zip(BEAMS, xs)):
        alone, _ = _serve(cdmt, [b], [x], interleave=False, precision=precision)
        assert np.array_equal(alone[0], mixed[bi]), bi
        off = _offline(cdmt, b, x, precision)
        assert off.shape == mixed[bi].shape, (off.shape, mixed[bi].shape)
        assert np.array_equal(off, mixed[bi]), bi


@pytest.mark.parametrize("prec,i8", [("fp32", False), ("fp16", False), ("fp32", True), ("fp16", True)])
def test_served_blocks_match_oracle(cdmt, orc, prec, i8):
    """Each block of each beam, served in a mix of three beams whose blocks overlap
    on the GPU (blocks shorter than, equal to and longer than N; two output slots,
    so blocks wait for slots), equals the FP64 oracle's filterbank of the beam's
    whole stream at the block's output positions (Algorithm 1's block loop, Sec. 3):
    within 1e-5 (FP32) or 2e-3 (FP16) of the mean output, sample by sample.  With
    int8 blocks the oracle runs on the dequantised voltages (scale x byte, FP32)."""
    precision = cdmt.CDMT_PREC_FP16 if prec == "fp16" else cdmt.CDMT_PREC_FP32
    tol = 2e-3 if prec == "fp16" else 1e-5
    xs = _inputs(BEAMS)
    scales = None
    if i8:
        scales = [(np.abs(x).reshape(b["nsub"], -1).max(axis=1) / 127.0).astype(np.float32) for b, x in zip(BEAMS, xs)]
        xs = [np.clip(np.rint(x / s[:, None, None]), -127, 127).astype(np.int8) for x, s in zip(xs, scales)]
    parts, st = _serve(cdmt, BEAMS, xs, interleave=True, i8=i8, scales=scales, precision=precision, max_slots=2,
                       keep_parts=True)
    assert st.blocks_done == NBLK * len(BEAMS)
    for bi, (b, x) in enumerate(zip(BEAMS, xs)):
        v = x.astype(np.float32) * scales[bi][:, None, None] if i8 else x
        dms = [b["dm_first"] + i * b["dm_step"] for i in range(b["ndm"])]
        nbin = 4096 * b["nchan"]
        nd = orc.overlap(b["nsub"], b["f_centre"], BW, dms, b["nchan"], b["nint"], nbin)
        o = orc.filterbank(v, b["f_centre"], BW, dms, b["nchan"], b["nint"], nbin, nd)
        assert sum(p.shape[2] for p in parts[bi].values()) == o.shape[2]
        for first, g in parts[bi].items():
            ob = o[:, :, first:first + g.shape[2]]
            assert ob.shape == g.shape and np.all(np.isfinite(g))
            emax, erms = rel_errors(g, ob)
            assert emax <= tol and erms <= tol, (bi, first, emax, erms)


def test_int8_blocks(cdmt):
    b = BEAMS[0]
    x = _inputs([b])[0]
    scale = (np.abs(x).reshape(b["nsub"], -1).max(axis=1) / 127.0).astype(np.float32)
    q = np.clip(np.rint(x / scale[:, None, None]), -127, 127).astype(np.int8)
    deq = q.astype(np.float32) * scale[:, None, None]
    got, _ = _serve(cdmt, [b], [q], interleave=False, i8=True, scales=[scale])
    assert np.array_equal(got[0], _offline(cdmt, b, deq, cdmt.CDMT_PREC_FP16))


def test_admission_and_errors(cdmt):
    srv = cdmt.Server(hbm_budget=64 << 20)
    with pytest.raises(cdmt.CdmtError) as e:
        srv.add_beam(64, 1 << 16, 135.0, BW, 0.0, 0.5, 128, 16, 8)
    assert e.value.status == cdmt.CDMT_EBUDGET
    with pytest.raises(cdmt.CdmtError) as e:
        srv.submit(0, 1)
    assert e.value.status == cdmt.CDMT_EINVAL
    with pytest.raises(cdmt.CdmtError) as e:
        srv.wait(12345, 0.1)
    assert e.value.status == cdmt.CDMT_EINVAL
    srv.close()


def test_u8_blocks_are_the_redigitised_float_blocks(cdmt, orc):
    """A CDMT_OUT_U8 beam carries, per block, the codes, row statistics and
    spectral-kurtosis flags that the redigitisation (Sec. 3, with the flagging of
    Sec. 6) gives for the float32 filterbank of the same block: checked against
    the oracle's redigitisation of a float32 twin beam fed the same blocks on the
    same server."""
    import torch
    from test_redig_gpu import _check_sk
    b = BEAMS[1]
    x = _inputs([b])[0]
    rows, L = b["nsub"] * b["nchan"], b["block_len"]
    srv = cdmt.Server(max_slots=3)
    ids = [srv.add_beam(b["nsub"], L, b["f_centre"], BW, b["dm_first"], b["dm_step"], b["ndm"], b["nchan"], b["nint"],
                        dm_tile=b["ndm"], out_dtype=od, sk_nsigma=2.5)
           for od in (cdmt.CDMT_OUT_F32, cdmt.CDMT_OUT_U8)]
    blocks = [torch.from_numpy(np.ascontiguousarray(x[:, k * L:(k + 1) * L])).pin_memory() for k in range(NBLK)]
    reqs = [(k, [srv.submit(i, blocks[k].data_ptr()) for i in ids]) for k in range(NBLK)]
    checked = 0
    for k, (rf, ru) in reqs:
        a, u = srv.wait(rf, 120.0), srv.wait(ru, 120.0)
        assert (a.first_sample, a.samples) == (u.first_sample, u.samples)
        assert a.d_u8 is None and a.d_flags is None and u.d_out is None
        if u.samples > 0:
            fb = srv.block_view(a, b["ndm"], rows).cpu().numpy()
            codes, stats, flags = (t.cpu().numpy() for t in srv.block_u8_view(u, b["ndm"], rows))
            assert codes.shape == (b["ndm"], u.samples, rows)
            _check_sk(orc, fb, codes, stats, flags, 2 * b["nint"], 2.5)
            checked += 1
        else:
            with pytest.raises(cdmt.CdmtError):
                srv.block_u8_view(a, b["ndm"], rows)
        srv.release(rf)
        srv.release(ru)
    srv.close()
    assert checked >= 2   # 8 blocks of 24576 samples complete 3 segments of N = 65536


def test_u8_blocks_in_dm_ranges_under_a_small_budget(cdmt, orc):
    """An 8-bit beam whose block filterbank would take more than a sixth of the HBM
    budget runs each block's DM stage in 2 ranges through a half-size scratch:
    its codes, statistics and flags equal the oracle's redigitisation of a float32
    twin beam (on a server with the default budget) fed the same blocks."""
    import torch
    from test_redig_gpu import _check_sk
    b = dict(nsub=2, block_len=1 << 14, f_centre=140.0, dm_first=0.0, dm_step=0.25, ndm=64, nchan=8, nint=4, seed=57)
    rows, L, nbin = b["nsub"] * b["nchan"], b["block_len"], 4096 * b["nchan"]
    dms = [b["dm_first"] + i * b["dm_step"] for i in range(b["ndm"])]
    nd = orc.overlap(b["nsub"], b["f_centre"], BW, dms, b["nchan"], b["nint"], nbin)
    S = nbin - nd * b["nchan"]
    seglen = (nbin // b["nchan"] - nd) // b["nint"]
    max_seg = L // S + 1
    stride = (max_seg * seglen + 3) // 4 * 4
    full = 4 * b["ndm"] * rows * stride              # one block's float32 filterbank
    budget = 5 * full                                # full > budget / 6 >= full / 2: two ranges
    x = _inputs([b])[0]
    blocks = [torch.from_numpy(np.ascontiguousarray(x[:, k * L:(k + 1) * L])).pin_memory() for k in range(NBLK)]
    servers = [cdmt.Server(), cdmt.Server(hbm_budget=budget)]
    ids = [srv.add_beam(b["nsub"], L, b["f_centre"], BW, b["dm_first"], b["dm_step"], b["ndm"], b["nchan"],
                        b["nint"], dm_tile=b["ndm"], out_dtype=od, sk_nsigma=2.5)
           for srv, od in zip(servers, (cdmt.CDMT_OUT_F32, cdmt.CDMT_OUT_U8))]
    checked = 0
    for k in range(NBLK):
        ra, ru = (srv.submit(i, blocks[k].data_ptr()) for srv, i in zip(servers, ids))
        a, u = servers[0].wait(ra, 120.0), servers[1].wait(ru, 120.0)
        assert (a.first_sample, a.samples) == (u.first_sample, u.samples)
        if u.samples > 0:
            fb = servers[0].block_view(a, b["ndm"], rows).cpu().numpy()
            codes, stats, flags = (t.cpu().numpy() for t in servers[1].block_u8_view(u, b["ndm"], rows))
            _check_sk(orc, fb, codes, stats, flags, 2 * b["nint"], 2.5)
            checked += 1
        servers[0].release(ra)
        servers[1].release(ru)
    for srv in servers:
        srv.close()
    assert checked >= 4


def test_checkpoint_resumes_a_stream_exactly(cdmt):
    # blocks 0-3 on one server, a checkpoint of the beam, blocks 4-7 on a new server restored
    # from it: the same filterbank at the same positions, bit for bit, as the stream served
    # whole; block indices continue.  The blocks are shorter than N, so the checkpoint holds a
    # partly filled tail.
    import torch
    b = BEAMS[1]
    L = b["block_len"]
    x = synth.noise(b["seed"] + 100, b["nsub"], NBLK * L)
    blocks = [torch.from_numpy(np.ascontiguousarray(x[:, k * L:(k + 1) * L])).pin_memory() for k in range(NBLK)]

    def beam(srv, block_len=L):
        return srv.add_beam(b["nsub"], block_len, b["f_centre"], BW, b["dm_first"], b["dm_step"], b["ndm"],
                            b["nchan"], b["nint"], precision=cdmt.CDMT_PREC_FP16, dm_tile=b["ndm"])

    def serve(srv, bid, ks):
        got = {}
        for k in ks:
            rid = srv.submit(bid, blocks[k].data_ptr())
            res = srv.wait(rid, 120.0)
            assert res.index == k
            if res.samples > 0:
                got[res.first_sample] = srv.block_view(res, b["ndm"], b["nsub"] * b["nchan"]).cpu().numpy()
            srv.release(rid)
        return got

    srv = cdmt.Server()
    ref = serve(srv, beam(srv), range(NBLK))
    srv.close()
    sa = cdmt.Server()
    a = beam(sa)
    part = serve(sa, a, range(4))
    ck = sa.save_beam(a)
    sa.close()
    assert ck.size > 64
    sb = cdmt.Server()
    nb = beam(sb)
    sb.restore_beam(nb, ck)
    part.update(serve(sb, nb, range(4, NBLK)))
    sb.close()
    assert sorted(part) == sorted(ref)
    for k in ref:
        assert np.array_equal(part[k], ref[k])
    # refused: another shape, a truncated checkpoint
    sc = cdmt.Server()
    other = beam(sc, block_len=2 * L)
    same = beam(sc)
    for bad, data in ((other, ck), (same, ck[:ck.size - 16])):
        with pytest.raises(cdmt.CdmtError) as e:
            sc.restore_beam(bad, data)
        assert e.value.status == cdmt.CDMT_EINVAL
    sc.close()
