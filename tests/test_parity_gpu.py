"""GPU filterbanks against the FP64 oracle (run through the C ABI).

Tolerance for the plain FP32 path: max |gpu - oracle| / mean(oracle) <= 1e-5
and ||gpu - oracle|| / ||oracle|| <= 1e-5 (relative errors against the mean
output; the FP32 FFTs, the 32-bit fixed-point chirp phase and the FP32 sine /
cosine each contribute ~1e-7 relative to the field).  Integer plan quantities
(n_d, S, nseg, nout) must equal the oracle's exactly.
"""
import numpy as np
import pytest

import synth
from helpers import gpu_filterbank, pulse_snr, rel_errors

pytestmark = pytest.mark.gpu

TOL_MAX = 1e-5
TOL_RMS = 1e-5
BW = 0.1953125


@pytest.fixture(scope="module")
def cdmt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_00909_gb300 as m
    return m


def _plan(cdmt, nsub, nsamp, fc, dms, nchan, nint, **kw):
    return cdmt.Plan(nsub, nsamp, fc, BW, dms, nchan, nint, **kw)


def _compare(orc, plan, x, fc, dms, nchan, nint):
    i = plan.info
    g = gpu_filterbank(plan, x)
    assert np.all(np.isfinite(g)), "output not fully written"
    o = orc.filterbank(x, fc, BW, dms, nchan, nint, i["nbin"], i["nd"])
    assert g.shape == o.shape
    return g, o, rel_errors(g, o)


def test_tiny_workload_full_parity(cdmt, orc):
    w = synth.tiny()
    x = w.voltages()
    plan = _plan(cdmt, w.nsub, w.nsamp, w.f_centre, w.dms, w.nchan, w.nint, nbin=w.nbin)
    i = plan.info
    # plan quantities, bit-exact against the oracle's own rule and grid
    assert i["nd"] == orc.overlap(w.nsub, w.f_centre, w.bw, w.dms, w.nchan, w.nint, w.nbin) == 32
    assert (i["nvalid"], i["nseg"], i["nout"]) == orc.grid(w.nsamp, w.nbin, w.nchan, i["nd"], w.nint)
    g, o, (emax, erms) = _compare(orc, plan, x, w.f_centre, w.dms, w.nchan, w.nint)
    print(f"tiny: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert emax <= TOL_MAX and erms <= TOL_RMS
    # the injected pulse keeps its S/N to 1 %
    p = w.pulses[0]
    sg = pulse_snr(g, w.dms, p, w.f_centre, w.bw, w.nsub, w.nchan, w.nint, i["nd"])
    so = pulse_snr(o, w.dms, p, w.f_centre, w.bw, w.nsub, w.nchan, w.nint, i["nd"])
    assert so > 5
    assert abs(sg / so - 1) <= 0.01


@pytest.mark.parametrize("nchan,mbin,nint", [(2, 512, 1), (4, 1024, 2), (8, 2048, 4), (16, 4096, 8),
                                             (32, 512, 16), (32, 2048, 3), (16, 1024, 5), (8, 8192, 4),
                                             (2, 8192, 3)])
def test_channel_and_fft_shapes(cdmt, orc, nchan, mbin, nint):
    nbin = nchan * mbin
    nsamp = 3 * nbin + 777          # several segments and a ragged tail
    dms = [0.0, 2.5, 5.0, 7.5, 10.0]
    x = synth.noise(3, 2, nsamp)
    plan = _plan(cdmt, 2, nsamp, 150.0, dms, nchan, nint, nbin=nbin)
    g, o, (emax, erms) = _compare(orc, plan, x, 150.0, dms, nchan, nint)
    assert plan.info["nseg"] >= 3
    assert emax <= TOL_MAX and erms <= TOL_RMS, (emax, erms)


def test_uneven_dm_list_uses_fp64_products(cdmt, orc):
    dms = [0.0, 3.7, -5.0, 12.1, 40.0, 39.99]
    x = synth.noise(4, 1, 1 << 15)
    plan = _plan(cdmt, 1, 1 << 15, 120.0, dms, 8, 2, nbin=1 << 13)
    assert plan.info["uniform_dm"] == 0
    g, o, (emax, erms) = _compare(orc, plan, x, 120.0, dms, 8, 2)
    assert emax <= TOL_MAX and erms <= TOL_RMS, (emax, erms)


@pytest.mark.parametrize("mbin", [2048, 4096])
def test_uneven_dm_list_paired_kernel(cdmt, orc, mbin):
    """Uneven DM lists (the FP64 phase per bin and DM) at the sizes the FP32 form runs with both
    polarisations per thread, several segments and a ragged tail."""
    dms = [0.0, 3.7, -5.0, 12.1, 40.0, 39.99, 7.25]
    nbin = 8 * mbin
    nsamp = 3 * nbin + 1234
    x = synth.noise(41, 2, nsamp)
    plan = _plan(cdmt, 2, nsamp, 125.0, dms, 8, 4, nbin=nbin)
    assert plan.info["uniform_dm"] == 0 and plan.info["mbin"] == mbin
    g, o, (emax, erms) = _compare(orc, plan, x, 125.0, dms, 8, 4)
    assert emax <= TOL_MAX and erms <= TOL_RMS, (emax, erms)


def test_dm_zero_only_needs_no_overlap(cdmt, orc):
    x = synth.noise(5, 1, 1 << 14)
    plan = _plan(cdmt, 1, 1 << 14, 135.0, [0.0], 8, 4, nbin=1 << 12)
    assert plan.info["nd"] == 0 and plan.info["nvalid"] == 1 << 12
    g, o, (emax, erms) = _compare(orc, plan, x, 135.0, [0.0], 8, 4)
    assert emax <= TOL_MAX and erms <= TOL_RMS


def test_chunked_workspace_and_ragged_dm_tiles(cdmt, orc):
    dms = [1.0 * i for i in range(7)]
    nsamp = 6 * (1 << 12) + 100
    x = synth.noise(6, 3, nsamp)
    ref = _plan(cdmt, 3, nsamp, 140.0, dms, 4, 2, nbin=1 << 12, dm_tile=3)
    plan = _plan(cdmt, 3, nsamp, 140.0, dms, 4, 2, nbin=1 << 12, seg_chunk=3, dm_tile=3)
    assert plan.info["seg_chunk"] == 3 and plan.info["dm_tile"] == 3 and ref.info["seg_chunk"] == ref.info["nseg"]
    g, o, (emax, erms) = _compare(orc, plan, x, 140.0, dms, 4, 2)
    assert emax <= TOL_MAX and erms <= TOL_RMS
    # chunking the workspace changes the schedule, not the arithmetic (a different
    # DM tiling would: each tile rounds its own fixed-point start phase)
    assert np.array_equal(g, gpu_filterbank(ref, x))


def test_execute_host_matches_execute(cdmt):
    import torch
    w = synth.tiny()
    x = w.voltages()
    plan = _plan(cdmt, w.nsub, w.nsamp, w.f_centre, w.dms, w.nchan, w.nint, nbin=w.nbin)
    dev = gpu_filterbank(plan, x)
    hin = torch.from_numpy(x).pin_memory()
    hout = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32).pin_memory()
    plan.execute_host(hin.data_ptr(), hout.data_ptr(), 0, torch.cuda.current_stream().cuda_stream)
    assert np.array_equal(hout.numpy(), dev)
    # pageable host memory also works
    hout2 = np.full(plan.out_shape(), np.nan, dtype=np.float32)
    plan.execute_host(x.ctypes.data, hout2.ctypes.data, 0, 0)
    assert np.array_equal(hout2, dev)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("uniform,ndm", [(True, 70), (False, 70), (True, 97)])
def test_execute_host_dm_ranges(cdmt, prec, uniform, ndm):
    """float32 host output of a plan with one DM tile runs each block's DM stage in
    DM ranges (70 DMs: 2 of 35; 97 DMs: 33, 33 and 31; 3 blocks of 3 segments):
    bit-identical to the device path, for evenly spaced (phase steps from the
    range's offset) and uneven DM lists."""
    import torch
    nsub, nsamp = 2, 9 * (1 << 14) + 5
    x = synth.noise(91, nsub, nsamp)
    dms = [17.0 * i / ndm for i in range(ndm)]
    if not uniform:
        dms = sorted(np.random.default_rng(5).uniform(0.0, 17.0, ndm).tolist())
    precision = cdmt.CDMT_PREC_FP16 if prec == "fp16" else cdmt.CDMT_PREC_FP32
    plan = _plan(cdmt, nsub, nsamp, 140.0, dms, 8, 4, nbin=1 << 14, dm_tile=ndm, precision=precision, host_block=3)
    assert plan.info["nseg"] == 9
    dev = gpu_filterbank(plan, x)
    hin = torch.from_numpy(x).pin_memory()
    hout = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32).pin_memory()
    plan.execute_host(hin.data_ptr(), hout.data_ptr(), 0, 0)
    assert np.array_equal(hout.numpy(), dev)
    plan.close()


def test_repeatable_and_stream_ordered(cdmt):
    import torch
    w = synth.tiny()
    x = w.voltages()
    plan = _plan(cdmt, w.nsub, w.nsamp, w.f_centre, w.dms, w.nchan, w.nint, nbin=w.nbin)
    s = torch.cuda.Stream()
    a = gpu_filterbank(plan, x, stream=s)
    b = gpu_filterbank(plan, x)
    assert np.array_equal(a, b)


def test_noise_mean_on_gpu(cdmt):
    # unitary transforms: complex white noise, E|x|^2 = 1 per pol -> mean 2 nint
    x = synth.noise(8, 4, 1 << 18)
    plan = _plan(cdmt, 4, 1 << 18, 135.0, [0.0, 10.0, 20.0], 16, 8, nbin=1 << 16)
    g = gpu_filterbank(plan, x)
    v = g.ravel().astype(np.float64)
    assert abs(v.mean() - 16.0) < 3 * v.std() / np.sqrt(v.size)


def test_plan_errors_on_device(cdmt):
    with pytest.raises(cdmt.CdmtError) as e:
        _plan(cdmt, 1, 1 << 14, 135.0, [0.0, 5000.0], 8, 4, nbin=1 << 14)  # overlap does not fit
    assert e.value.status == cdmt.CDMT_EINVAL
    with pytest.raises(cdmt.CdmtError) as e:
        _plan(cdmt, 1, 1 << 14, 135.0, [0.0], 16, 4, nbin=1 << 16)         # nsamp < N
    assert e.value.status == cdmt.CDMT_EINVAL
    with pytest.raises(cdmt.CdmtError) as e:
        _plan(cdmt, 1, 1 << 17, 135.0, [0.0], 8, 4, nbin=1 << 17)          # M = 16384: no kernel
    assert e.value.status == cdmt.CDMT_ENOTSUP
    with pytest.raises(cdmt.CdmtError) as e:                              # M = 8192: FP32 form only
        _plan(cdmt, 1, 1 << 16, 135.0, [0.0], 8, 4, nbin=1 << 16, precision=cdmt.CDMT_PREC_FP16)
    assert e.value.status == cdmt.CDMT_ENOTSUP
    with pytest.raises(cdmt.CdmtError) as e:
        _plan(cdmt, 64, 1 << 20, 135.0, [0.0], 16, 8, nbin=1 << 16, mem_budget=1 << 20)
    assert e.value.status == cdmt.CDMT_EBUDGET


@pytest.mark.slow
def test_lofar64_full_size_sampled_tiles(cdmt, orc):
    """The 64-subband, 2^22-sample, 128-DM workload in the launch configuration
    the benchmark times; 40 random (subband, segment, DM) tiles recomputed by
    the oracle, plus whole-output properties."""
    import torch
    w = synth.lofar64()
    x = w.voltages(threads=16)
    plan = _plan(cdmt, w.nsub, w.nsamp, w.f_centre, w.dms, w.nchan, w.nint, nbin=w.nbin)
    i = plan.info
    assert i["nd"] == orc.overlap(w.nsub, w.f_centre, w.bw, w.dms, w.nchan, w.nint, w.nbin)
    xt = torch.from_numpy(x).cuda()
    del x
    out = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32, device="cuda")
    import paper_1607_00909_gb300 as m
    m.run(plan, xt, out)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all())
    x = xt.cpu().numpy()
    del xt
    g = np.random.default_rng(2024)
    ntile = 40
    sub = g.integers(0, w.nsub, ntile)
    seg = g.integers(0, i["nseg"], ntile)
    seg[:2] = [0, i["nseg"] - 1]
    dmi = g.integers(0, len(w.dms), ntile)
    o = orc.tiles(x, w.f_centre, w.bw, w.dms, w.nchan, w.nint, w.nbin, i["nd"], sub, seg, dmi)
    L = (i["mbin"] - i["nd"]) // w.nint
    gt = np.stack([out[dmi[t], sub[t] * w.nchan:(sub[t] + 1) * w.nchan, seg[t] * L:(seg[t] + 1) * L].cpu().numpy()
                   for t in range(ntile)])
    emax, erms = rel_errors(gt, o)
    print(f"lofar64 tiles: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert emax <= TOL_MAX and erms <= TOL_RMS


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_int8_input_equals_dequantised_float(cdmt, prec):
    """CDMT_IN_I8 plans read 4-byte samples times a per-subband scale (the paper's
    8-bit voltages): bit-identical to a float32 plan on the dequantised voltages,
    on the device and through the host pipeline (float32 and 8-bit output); the scales are
    required."""
    import torch
    nsub, nsamp = 3, 4 * (1 << 14) + 77
    x = synth.noise(71, nsub, nsamp)
    scale = (np.abs(x).reshape(nsub, -1).max(axis=1) / 127.0).astype(np.float32)
    q = np.clip(np.rint(x / scale[:, None, None]), -127, 127).astype(np.int8)
    deq = q.astype(np.float32) * scale[:, None, None]
    precision = cdmt.CDMT_PREC_FP16 if prec == "fp16" else cdmt.CDMT_PREC_FP32
    dms = [0.0, 3.0, 6.0]
    pf = _plan(cdmt, nsub, nsamp, 140.0, dms, 8, 4, nbin=1 << 14, precision=precision)
    want = gpu_filterbank(pf, deq)
    pf_bytes = pf.info["in_bytes"]
    pf.close()
    pi = _plan(cdmt, nsub, nsamp, 140.0, dms, 8, 4, nbin=1 << 14, precision=precision, in_dtype=cdmt.CDMT_IN_I8,
               host_block=2)
    assert pi.info["in_dtype"] == cdmt.CDMT_IN_I8
    assert pi.info["in_bytes"] == nsub * nsamp * 4 and pf_bytes == nsub * nsamp * 16
    qd, sd = torch.from_numpy(q).cuda(), torch.from_numpy(scale).cuda()
    got = cdmt.run(pi, qd, scale=sd)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)
    hin, hsc = torch.from_numpy(q).pin_memory(), torch.from_numpy(scale)
    hout = torch.full(pi.out_shape(), float("nan"), dtype=torch.float32).pin_memory()
    pi.execute_host(hin.data_ptr(), hout.data_ptr(), hsc.data_ptr(), 0)
    assert np.array_equal(hout.numpy(), want)
    with pytest.raises(cdmt.CdmtError) as e:
        pi.execute(qd.data_ptr(), got.data_ptr(), 0, 0)
    assert e.value.status == cdmt.CDMT_EINVAL
    # 8-bit in, 8-bit out (the paper's own I/O): the codes equal those of the float32 plan on the
    # dequantised voltages; without scales the int8 plan is refused
    shape8 = (len(dms), pi.out_shape()[2], pi.out_shape()[1])
    u8, ref8 = torch.empty(shape8, dtype=torch.uint8).pin_memory(), torch.empty(shape8, dtype=torch.uint8).pin_memory()
    assert pi.execute_host_u8(hin.data_ptr(), u8.data_ptr(), 0, hsc.data_ptr()) == 2
    pf = _plan(cdmt, nsub, nsamp, 140.0, dms, 8, 4, nbin=1 << 14, precision=precision, host_block=2)
    pf.execute_host_u8(torch.from_numpy(deq).pin_memory().data_ptr(), ref8.data_ptr())
    pf.close()
    assert np.array_equal(u8.numpy(), ref8.numpy())
    with pytest.raises(cdmt.CdmtError) as e:
        pi.execute_host_u8(hin.data_ptr(), u8.data_ptr())
    assert e.value.status == cdmt.CDMT_EINVAL
    pi.close()
