"""Incoherent dedispersion of the coherent filterbanks over fine DM trials
(Sec. 4, semi-coherent search) against the oracle.

The shift table is integer work computed in FP64 on both sides: it must be
identical.  The sums are FP32 over the channel rows on the GPU and FP64 in the
oracle, from the same float filterbank: max |gpu - oracle| / mean(oracle) and
the RMS ratio within 1e-5.
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


def _run(cdmt, orc, plan, fb, nsub, nchan, fc, nint, dms, lo, step, nk, chirp=0):
    import torch
    nt_out, tab = cdmt.cdmt_incoherent_info(plan.handle, lo, step, nk, delays=True)
    out = plan.incoherent(fb, lo, step, nk)
    torch.cuda.synchronize()
    o, otab = orc.incoherent(fb.cpu().numpy(), nsub, nchan, fc, BW, nint, dms, lo, step, nk, chirp=chirp)
    assert np.array_equal(tab, otab)
    assert out.shape == o.shape and nt_out == o.shape[2]
    emax, erms = rel_errors(out.cpu().numpy(), o)
    assert emax <= 1e-5 and erms <= 1e-5, (emax, erms)
    return out.cpu().numpy(), o


def test_incoherent_tiny_workload(cdmt, orc):
    import torch
    w = synth.tiny()
    plan = cdmt.Plan(1, w.nsamp, w.f_centre, BW, w.dms, w.nchan, w.nint, nbin=w.nbin)
    fb = cdmt.run(plan, torch.from_numpy(w.voltages()).cuda())
    # 37 fine trials (two blocks of 16 and a ragged one) around every coherent DM
    _run(cdmt, orc, plan, fb, 1, w.nchan, w.f_centre, w.nint, w.dms, -0.5, 0.03, 37)
    plan.close()


@pytest.mark.parametrize("chirp", [0, 1])
def test_incoherent_multi_subband(cdmt, orc, chirp):
    import torch
    nsub, nsamp, fc, nchan, nint = 4, 3 * (1 << 15) + 321, 130.0, 8, 2
    dms = [0.5, 3.0, 7.5]
    x = synth.noise(26, nsub, nsamp)
    plan = cdmt.Plan(nsub, nsamp, fc, BW, dms, nchan, nint, nbin=1 << 15, chirp=chirp)
    fb = cdmt.run(plan, torch.from_numpy(x).cuda())
    g, _ = _run(cdmt, orc, plan, fb, nsub, nchan, fc, nint, dms, -0.5, 0.002, 500, chirp=chirp)
    # detected noise summed over rows: every trial has mean rows * 2 sigma^2 nint
    rows = nsub * nchan
    assert abs(g.mean() / (rows * 2.0 * nint) - 1.0) < 0.02
    plan.close()


def test_incoherent_coarse_trials(cdmt, orc):
    # steps of 1 pc cm^-3: shifts jump by many samples between trials, most rows change
    import torch
    nsub, nsamp, fc, nchan, nint = 2, 1 << 17, 125.0, 8, 4
    dms = [5.0, 20.0]
    x = synth.noise(27, nsub, nsamp)
    plan = cdmt.Plan(nsub, nsamp, fc, BW, dms, nchan, nint, nbin=1 << 15)
    fb = cdmt.run(plan, torch.from_numpy(x).cuda())
    _run(cdmt, orc, plan, fb, nsub, nchan, fc, nint, dms, -4.0, 1.0, 40)
    plan.close()


def test_incoherent_rejects_empty_grid(cdmt):
    w = synth.tiny()
    plan = cdmt.Plan(1, w.nsamp, w.f_centre, BW, w.dms, w.nchan, w.nint, nbin=w.nbin)
    with pytest.raises(cdmt.CdmtError) as e:
        cdmt.cdmt_incoherent_info(plan.handle, 0.0, 1000.0, 8)   # shifts longer than the filterbank
    assert e.value.status == cdmt.CDMT_EINVAL
    plan.close()
