"""Tensor-core (FP16, BF16 hi/lo) forms of the DM stage against the FP64 oracle.

Tolerance of the tensor-core forms: max |gpu - oracle| / mean(oracle) <= 2e-3
and ||gpu - oracle|| / ||oracle|| <= 2e-3; injected-pulse S/N within 1 % of the
oracle's.  Error budget (FP16): the chirped spectrum, the pass-A result and the
DFT-matrix entries are each rounded once to 11 significant bits (unit roundoff
2^-11 = 4.9e-4); averaged over 64-term sums and the 2 x nint detected samples
of one output, the RMS error of an output is ~3e-4 of the mean and its maximum
over ~10^6 outputs stays below 2e-3.  BF16 splits data and matrix into hi + lo
parts, which brings it below the FP16 error.
"""
import numpy as np
import pytest

import synth
from helpers import gpu_filterbank, pulse_snr, rel_errors

pytestmark = pytest.mark.gpu

TOL = 2e-3
BW = 0.1953125


@pytest.fixture(scope="module")
def cdmt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_00909_gb300 as m
    return m


PRECS = [("fp16", 1), ("bf16", 2)]


@pytest.mark.parametrize("name,prec", PRECS)
def test_tc_pulse_workload(cdmt, orc, name, prec):
    # the tiny workload's voltages (1 subband, 2^17 samples, pulse at DM 10),
    # channelised with M = 4096 (N = 2^15, 8 channels)
    w = synth.tiny()
    x = w.voltages()
    nbin = 1 << 15
    plan = cdmt.Plan(1, w.nsamp, w.f_centre, BW, w.dms, 8, w.nint, nbin=nbin, precision=prec)
    i = plan.info
    assert i["precision"] == prec and i["mbin"] == 4096
    g = gpu_filterbank(plan, x)
    plan.device_status()
    assert np.all(np.isfinite(g))
    o = orc.filterbank(x, w.f_centre, BW, w.dms, 8, w.nint, nbin, i["nd"])
    emax, erms = rel_errors(g, o)
    print(f"{name}: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert emax <= TOL and erms <= TOL
    p = w.pulses[0]
    sg = pulse_snr(g, w.dms, p, w.f_centre, BW, 1, 8, w.nint, i["nd"])
    so = pulse_snr(o, w.dms, p, w.f_centre, BW, 1, 8, w.nint, i["nd"])
    print(f"{name}: S/N gpu {sg:.3f} oracle {so:.3f}")
    assert so > 5 and abs(sg / so - 1) <= 0.01


@pytest.mark.parametrize("name,prec", PRECS)
def test_tc_multi_subband_shapes(cdmt, orc, name, prec):
    # 3 subbands, 16 channels (N = 2^16), ragged tail, 5 DMs (odd: one warpgroup idles on the last)
    nsamp = 3 * (1 << 16) + 999
    dms = [0.0, 7.0, 14.0, 21.0, 28.0]
    x = synth.noise(21, 3, nsamp)
    plan = cdmt.Plan(3, nsamp, 150.0, BW, dms, 16, 8, nbin=1 << 16, precision=prec)
    g = gpu_filterbank(plan, x)
    plan.device_status()
    o = orc.filterbank(x, 150.0, BW, dms, 16, 8, 1 << 16, plan.info["nd"])
    emax, erms = rel_errors(g, o)
    print(f"{name} 3-subband: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert np.all(np.isfinite(g)) and emax <= TOL and erms <= TOL


def test_tc_uneven_dm_list(cdmt, orc):
    dms = [0.0, 3.7, -5.0, 12.1, 40.0, 39.99, 63.3]
    x = synth.noise(22, 1, 1 << 17)
    plan = cdmt.Plan(1, 1 << 17, 120.0, BW, dms, 8, 4, nbin=1 << 15, precision=cdmt.CDMT_PREC_FP16)
    assert plan.info["uniform_dm"] == 0
    g = gpu_filterbank(plan, x)
    plan.device_status()
    o = orc.filterbank(x, 120.0, BW, dms, 8, 4, 1 << 15, plan.info["nd"])
    emax, erms = rel_errors(g, o)
    assert emax <= TOL and erms <= TOL


def test_tc_strong_signal_scaling(cdmt, orc):
    # a bright tone plus noise 40 dB below it: the per-CTA power-of-two scaling
    # must keep the half-precision operands in range
    nsamp = 1 << 16
    x = synth.noise(23, 1, nsamp, sigma2=1e-4)
    nbin, nchan = 1 << 15, 8
    m = nbin // nchan
    off = (2 * m + m // 2 - nbin // 2) * BW / nbin
    x += synth.tone(nsamp, off, BW, 300.0 + 200.0j, -100.0 + 50.0j)
    dms = [0.0, 10.0, 20.0]
    plan = cdmt.Plan(1, nsamp, 135.0, BW, dms, nchan, 4, nbin=nbin, precision=cdmt.CDMT_PREC_FP16)
    g = gpu_filterbank(plan, x)
    plan.device_status()
    o = orc.filterbank(x, 135.0, BW, dms, nchan, 4, nbin, plan.info["nd"])
    assert np.all(np.isfinite(g))
    emax, erms = rel_errors(g, o)
    assert emax <= TOL and erms <= TOL


def test_tc_size_limits(cdmt):
    # channels of 1024 bins, and an integration that does not divide 32, are not supported
    with pytest.raises(cdmt.CdmtError) as e:
        cdmt.Plan(1, 1 << 17, 135.0, BW, [0.0, 5.0], 8, 4, nbin=1 << 13, precision=cdmt.CDMT_PREC_FP16)
    assert e.value.status == cdmt.CDMT_ENOTSUP
    with pytest.raises(cdmt.CdmtError) as e:
        cdmt.Plan(1, 1 << 17, 135.0, BW, [0.0, 5.0], 8, 3, nbin=1 << 15, precision=cdmt.CDMT_PREC_FP16)
    assert e.value.status == cdmt.CDMT_ENOTSUP


@pytest.mark.parametrize("name,prec", PRECS)
def test_tc_tiny_workload_own_shapes(cdmt, orc, name, prec):
    # the tiny workload exactly as the FP32 path runs it: N = 2^14, 8 channels of M = 2048
    w = synth.tiny()
    x = w.voltages()
    plan = cdmt.Plan(1, w.nsamp, w.f_centre, BW, w.dms, w.nchan, w.nint, nbin=w.nbin, precision=prec)
    i = plan.info
    assert i["mbin"] == 2048 and i["nd"] == 32
    g = gpu_filterbank(plan, x)
    plan.device_status()
    assert np.all(np.isfinite(g))
    o = orc.filterbank(x, w.f_centre, BW, w.dms, w.nchan, w.nint, w.nbin, i["nd"])
    emax, erms = rel_errors(g, o)
    print(f"{name} M=2048: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert emax <= TOL and erms <= TOL
    p = w.pulses[0]
    sg = pulse_snr(g, w.dms, p, w.f_centre, BW, 1, w.nchan, w.nint, i["nd"])
    so = pulse_snr(o, w.dms, p, w.f_centre, BW, 1, w.nchan, w.nint, i["nd"])
    print(f"{name} M=2048: S/N gpu {sg:.3f} oracle {so:.3f}")
    assert so > 5 and abs(sg / so - 1) <= 0.01


@pytest.mark.parametrize("nint", [16, 32])
@pytest.mark.parametrize("name,prec", PRECS)
def test_tc_m2048_many_channels(cdmt, orc, name, prec, nint):
    # 32 channels of 2048 bins (N = 2^16), 2 subbands, ragged tail, 7 DMs (six FP16 pipes, one idle on the last)
    nsamp = 2 * (1 << 16) + 5001
    dms = [0.0, 9.0, 18.0, 27.0, 36.0, 45.0, 54.0]
    x = synth.noise(24, 2, nsamp)
    plan = cdmt.Plan(2, nsamp, 140.0, BW, dms, 32, nint, nbin=1 << 16, precision=prec)
    assert plan.info["mbin"] == 2048
    g = gpu_filterbank(plan, x)
    plan.device_status()
    o = orc.filterbank(x, 140.0, BW, dms, 32, nint, 1 << 16, plan.info["nd"])
    emax, erms = rel_errors(g, o)
    print(f"{name} M=2048 nint {nint}: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert np.all(np.isfinite(g)) and emax <= TOL and erms <= TOL


@pytest.mark.slow
def test_tc_lofar64_full_size_sampled_tiles(cdmt, orc):
    import torch

    import paper_1607_00909_gb300 as m
    w = synth.lofar64()
    x = w.voltages(threads=16)
    plan = cdmt.Plan(w.nsub, w.nsamp, w.f_centre, BW, w.dms, w.nchan, w.nint, nbin=w.nbin,
                     precision=cdmt.CDMT_PREC_FP16)
    i = plan.info
    xt = torch.from_numpy(x).cuda()
    out = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32, device="cuda")
    m.run(plan, xt, out)
    torch.cuda.synchronize()
    plan.device_status()
    assert bool(torch.isfinite(out).all())
    del xt
    g = np.random.default_rng(77)
    ntile = 32
    sub = g.integers(0, w.nsub, ntile)
    seg = g.integers(0, i["nseg"], ntile)
    seg[:2] = [0, i["nseg"] - 1]
    dmi = g.integers(0, len(w.dms), ntile)
    o = orc.tiles(x, w.f_centre, BW, w.dms, w.nchan, w.nint, w.nbin, i["nd"], sub, seg, dmi)
    L = (i["mbin"] - i["nd"]) // w.nint
    gt = np.stack([out[dmi[t], sub[t] * w.nchan:(sub[t] + 1) * w.nchan, seg[t] * L:(seg[t] + 1) * L].cpu().numpy()
                   for t in range(ntile)])
    emax, erms = rel_errors(gt, o)
    print(f"tc fp16 lofar64 tiles: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert emax <= TOL and erms <= TOL
