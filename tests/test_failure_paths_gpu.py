"""Failure paths of the tensor-core kernels, exercised without a GPU fault.

The kernels bound every wait for a GEMM's completion (a time limit on the GPU's
global timer and a cap on polls); a CTA whose wait gives up sets the plan's
status word, later launches return at once, and cdmt_device_status reports
CDMT_ETIMEOUT and clears the word.  Here the bounded wait runs on a barrier that
nothing arrives on (in a one-warp kernel of its own), and the status word is set
from the host; nothing waits without a limit and nothing faults.
"""
import numpy as np
import pytest

import synth
from helpers import gpu_filterbank

pytestmark = pytest.mark.gpu
BW = 0.1953125


@pytest.fixture(scope="module")
def cdmt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_00909_gb300 as m
    return m


def test_bounded_wait_gives_up_and_the_context_stays_usable(cdmt, orc):
    gave_up, waited = cdmt.cdmt_selftest_wait(2.0)
    assert gave_up and 2.0 <= waited < 200.0, waited
    gave_up, waited = cdmt.cdmt_selftest_wait(2.0, arrive=True)   # the phase completes: no timeout
    assert not gave_up and waited < 2.0, waited
    # the device still computes correctly afterwards
    w = synth.tiny()
    x = w.voltages()
    plan = cdmt.Plan(1, w.nsamp, w.f_centre, BW, w.dms, w.nchan, w.nint, nbin=w.nbin,
                     precision=cdmt.CDMT_PREC_FP16)
    g = gpu_filterbank(plan, x)
    plan.device_status()
    o = orc.filterbank(x, w.f_centre, BW, w.dms, w.nchan, w.nint, w.nbin, plan.info["nd"])
    assert np.max(np.abs(g - o)) / np.mean(o) <= 2e-3
    plan.close()


@pytest.mark.parametrize("groups", [0, 2])
def test_status_word_skips_launches_until_reported(cdmt, groups):
    # after the injection the DM stage writes nothing (NaN fill survives); the status is
    # reported once as CDMT_ETIMEOUT, then cleared, and the next execute is correct again
    w = synth.tiny()
    x = w.voltages()
    plan = cdmt.Plan(1, w.nsamp, w.f_centre, BW, w.dms, w.nchan, w.nint, nbin=w.nbin,
                     precision=cdmt.CDMT_PREC_FP16, dm_groups=groups)
    want = gpu_filterbank(plan, x)
    plan.device_status()
    cdmt.cdmt_inject_timeout(plan.handle)
    skipped = gpu_filterbank(plan, x)
    assert np.all(np.isnan(skipped))
    with pytest.raises(cdmt.CdmtError) as e:
        plan.device_status()
    assert e.value.status == cdmt.CDMT_ETIMEOUT
    plan.device_status()   # cleared
    assert np.array_equal(gpu_filterbank(plan, x), want)
    plan.device_status()
    plan.close()
