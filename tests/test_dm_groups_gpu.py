"""Plans with one overlap per DM group (cdmt_opts.dm_groups) against the oracle.

Sec. 2 sizes the overlap for the largest |DM| of the list; digifil (Sec. 5)
sizes it per DM.  A grouped plan gives each contiguous group of trials the
overlap its own largest DM needs and keeps the ungrouped time axis and length.
The layout (overlaps, input offsets) must equal the oracle's, every output
sample must be written, and the values must match the oracle's grouped
filterbank at the tolerances of the forms (FP32 1e-5, FP16 2e-3).
"""
import numpy as np
import pytest

import synth
from helpers import gpu_filterbank, rel_errors

pytestmark = pytest.mark.gpu
BW = 0.1953125


@pytest.fixture(scope="module")
def cdmt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_00909_gb300 as m
    return m


def _case(chirp, nbin=1 << 14):
    # a low band with the subband-wide chirp (overlaps of 54 % of M = 2048 at the largest DM, 27 % of
    # M = 4096), or the per-channel chirp with an uneven DM list; several segments and a ragged tail
    if chirp:
        return dict(nsub=2, fc=60.0, dms=list(np.linspace(0.0, 6.0, 12)), nchan=8, nint=4, nbin=nbin,
                    nsamp=54983 if nbin == 1 << 14 else 4 * nbin + 1999)
    return dict(nsub=3, fc=70.0, dms=[0.0, 1.5, 2.0, 4.0, 7.5, 9.0, 12.0, 20.0, 21.0], nchan=8, nint=4,
                nbin=1 << 14, nsamp=5 * (1 << 14) + 333)


def _plan(cdmt, c, groups, prec, chirp, **kw):
    return cdmt.Plan(c["nsub"], c["nsamp"], c["fc"], BW, c["dms"], c["nchan"], c["nint"], nbin=c["nbin"],
                     precision=prec, chirp=chirp, dm_groups=groups, **kw)


@pytest.mark.parametrize("chirp", [0, 1])
@pytest.mark.parametrize("groups", [2, 4])
def test_grouped_layout_equals_the_oracle(cdmt, orc, chirp, groups):
    c = _case(chirp)
    plan = _plan(cdmt, c, groups, cdmt.CDMT_PREC_FP32, chirp)
    plain = _plan(cdmt, c, 0, cdmt.CDMT_PREC_FP32, chirp)
    layout, nd_max, nout = orc.grouped_layout(c["nsub"], c["nsamp"], c["fc"], BW, c["dms"], c["nchan"], c["nint"],
                                              c["nbin"], groups, chirp)
    assert plan.info["dm_groups"] == groups and plain.info["dm_groups"] == 1
    assert plan.info["nd"] == nd_max == plain.info["nd"]
    assert plan.info["nout"] == nout == plain.info["nout"]
    assert plan.info["units"] == plain.info["units"]
    assert plan.info["seg_chunk"] > 0 and plan.info["workspace_bytes"] > 0
    got = plan.groups()
    m = c["nbin"] // c["nchan"]
    for g, (first, count, nd_g, off, nbin_g) in zip(got, layout):
        assert (g["dm_first"], g["ndm"], g["nd"], g["offset"], g["nbin"]) == (first, count, nd_g, off, nbin_g)
        assert nbin_g == c["nbin"]
        seglen = (m - nd_g) // c["nint"]
        assert g["nseg"] == -(-nout // seglen)   # the segments that cover nout
    assert got[0]["nd"] < nd_max
    assert plain.groups() == [{"dm_first": 0, "ndm": len(c["dms"]), "nd": nd_max, "offset": 0,
                               "nseg": plain.info["nseg"], "nbin": c["nbin"]}]
    plan.close()
    plain.close()


@pytest.mark.parametrize("chirp,nbin", [(0, 1 << 14), (1, 1 << 14), (1, 1 << 15)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 2e-3), (2, 2e-3)])
def test_grouped_filterbank_matches_the_oracle(cdmt, orc, chirp, nbin, prec, tol):
    # FP32, FP16 and BF16 hi/lo forms; M = 2048 and (subband chirp, N = 2^15) M = 4096
    c = _case(chirp, nbin)
    x = synth.noise(40 + chirp, c["nsub"], c["nsamp"])
    plan = _plan(cdmt, c, 4, prec, chirp)
    g = gpu_filterbank(plan, x)   # NaN-filled first: every sample must be written
    plan.device_status()
    o = orc.filterbank_grouped(x, c["fc"], BW, c["dms"], c["nchan"], c["nint"], c["nbin"], 4, chirp=chirp)
    assert g.shape == o.shape
    assert np.all(np.isfinite(g))
    emax, erms = rel_errors(g, o)
    print(f"prec {prec} chirp {chirp} M {nbin // 8} 4 groups: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert emax <= tol and erms <= tol
    plan.close()


# channel lengths each precision runs (cdmt_plan_group_nbin)
LENGTHS = {0: [512, 1024, 2048, 4096, 8192], 1: [2048, 4096], 2: [2048, 4096]}


@pytest.mark.parametrize("chirp", [0, 1])
@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 2e-3)])
def test_grouped_lengths_match_the_oracle(cdmt, orc, chirp, prec, tol):
    """cdmt_opts.group_nbin: each group also takes its own FFT length (Sec. 5, digifil's
    per-DM FFT size).  The layout, lengths included, equals the oracle's with the
    lengths the precision runs; the filterbank matches the oracle's grouped filterbank
    at the same layout, every sample written."""
    c = _case(chirp)
    plan = _plan(cdmt, c, 4, prec, chirp, group_nbin=1)
    layout, nd_max, nout = orc.grouped_layout(c["nsub"], c["nsamp"], c["fc"], BW, c["dms"], c["nchan"], c["nint"],
                                              c["nbin"], 4, chirp, lengths=LENGTHS[prec])
    assert plan.info["nd"] == nd_max and plan.info["nout"] == nout
    got = plan.groups()
    for g, (first, count, nd_g, off, nbin_g) in zip(got, layout):
        assert (g["dm_first"], g["ndm"], g["nd"], g["offset"], g["nbin"]) == (first, count, nd_g, off, nbin_g)
        seglen = (nbin_g // c["nchan"] - nd_g) // c["nint"]
        assert g["nseg"] == -(-nout // seglen)
    print("lengths", [g["nbin"] // c["nchan"] for g in got], "overlaps", [g["nd"] for g in got])
    if prec == 0:
        assert any(g["nbin"] != c["nbin"] for g in got)
    x = synth.noise(60 + chirp, c["nsub"], c["nsamp"])
    fb = gpu_filterbank(plan, x)
    plan.device_status()
    o = orc.filterbank_grouped(x, c["fc"], BW, c["dms"], c["nchan"], c["nint"], c["nbin"], 4, chirp=chirp,
                               lengths=LENGTHS[prec])
    assert fb.shape == o.shape and np.all(np.isfinite(fb))
    emax, erms = rel_errors(fb, o)
    print(f"prec {prec} chirp {chirp} group lengths: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert emax <= tol and erms <= tol
    plan.close()


def test_grouped_plan_chunked_and_int8(cdmt, orc):
    # small workspace chunks and int8 input (offsets of 4-byte samples) give the same
    # filterbank as the float32 grouped plan on the dequantised voltages, bit for bit
    import torch
    c = _case(1)
    x = synth.noise(47, c["nsub"], c["nsamp"])
    scale = (np.abs(x).reshape(c["nsub"], -1).max(axis=1) / 127.0).astype(np.float32)
    q = np.clip(np.rint(x / scale[:, None, None]), -127, 127).astype(np.int8)
    deq = q.astype(np.float32) * scale[:, None, None]
    pf = _plan(cdmt, c, 3, cdmt.CDMT_PREC_FP32, 1)
    want = gpu_filterbank(pf, deq)
    pc = _plan(cdmt, c, 3, cdmt.CDMT_PREC_FP32, 1, seg_chunk=2)
    assert np.array_equal(gpu_filterbank(pc, deq), want)
    pi = _plan(cdmt, c, 3, cdmt.CDMT_PREC_FP32, 1, in_dtype=cdmt.CDMT_IN_I8)
    got = cdmt.run(pi, torch.from_numpy(q).cuda(), scale=torch.from_numpy(scale).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)
    o = orc.filterbank_grouped(deq, c["fc"], BW, c["dms"], c["nchan"], c["nint"], c["nbin"], 3, chirp=1)
    emax, erms = rel_errors(want, o)
    assert emax <= 1e-5 and erms <= 1e-5
    # int8 from host memory, the scales in host memory too
    hin, hsc = torch.from_numpy(q).pin_memory(), torch.from_numpy(scale)
    hout = torch.full(pi.out_shape(), float("nan"), dtype=torch.float32).pin_memory()
    pi.execute_host(hin.data_ptr(), hout.data_ptr(), hsc.data_ptr(), 0)
    assert np.array_equal(hout.numpy(), want)
    with pytest.raises(cdmt.CdmtError) as e:
        pi.execute_host(hin.data_ptr(), hout.data_ptr(), 0, 0)
    assert e.value.status == cdmt.CDMT_EINVAL
    for p in (pf, pc, pi):
        p.close()


def test_grouped_plan_stage_times_and_host_entry_points(cdmt):
    # stage timing sums the groups' launches; from host memory a grouped plan gives the
    # device execute's filterbank, and 8-bit codes of the whole input as one block, bit for bit
    import torch
    c = _case(1)
    x = synth.noise(48, c["nsub"], c["nsamp"])
    plan = _plan(cdmt, c, 4, cdmt.CDMT_PREC_FP16, 1)
    cdmt.cdmt_set_timing(plan.handle, True)
    cdmt.cdmt_stage_times(plan.handle)
    want = gpu_filterbank(plan, x)
    (fwd_ms, dd_ms), (fwd_n, dd_n) = cdmt.cdmt_stage_times(plan.handle)
    assert dd_n == 4 and fwd_n == 8 and fwd_ms > 0 and dd_ms > 0
    cdmt.cdmt_set_timing(plan.handle, False)
    hin = torch.from_numpy(x).pin_memory()
    hout = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32).pin_memory()
    plan.execute_host(hin.data_ptr(), hout.data_ptr(), 0, 0)
    assert np.array_equal(hout.numpy(), want)
    ndm, rows, nt = plan.out_shape()
    codes = plan.redigitise(torch.from_numpy(want).cuda())
    torch.cuda.synchronize()
    hu8 = torch.empty((ndm, nt, rows), dtype=torch.uint8).pin_memory()
    assert plan.execute_host_u8(hin.data_ptr(), hu8.data_ptr(), 0) == plan.info["nseg"]
    assert np.array_equal(hu8.numpy(), codes.cpu().numpy())
    plan.close()


def test_grouped_filterbank_feeds_redigitisation_and_the_incoherent_stage(cdmt, orc):
    # the grouped plan's filterbank has the ungrouped geometry, so the 8-bit and
    # incoherent stages take it as they take any plan's
    import torch
    c = _case(0)
    x = synth.noise(49, c["nsub"], c["nsamp"])
    plan = _plan(cdmt, c, 3, cdmt.CDMT_PREC_FP32, 0)
    fb = torch.from_numpy(gpu_filterbank(plan, x)).cuda()
    ndm, rows, nt = fb.shape
    u8 = torch.empty((ndm, nt, rows), dtype=torch.uint8, device="cuda")
    plan.redigitise(fb, u8)
    torch.cuda.synchronize()
    want, _ = orc.redigitise(fb.cpu().numpy())
    assert np.abs(u8.cpu().numpy().astype(int) - want.astype(int)).max() <= 1
    inc = plan.incoherent(fb, -0.5, 0.25, 5)
    torch.cuda.synchronize()
    o, _ = orc.incoherent(fb.cpu().numpy(), c["nsub"], c["nchan"], c["fc"], BW, c["nint"], c["dms"], -0.5, 0.25, 5)
    emax, _ = rel_errors(inc.cpu().numpy(), o)
    assert emax <= 1e-5
    plan.close()
