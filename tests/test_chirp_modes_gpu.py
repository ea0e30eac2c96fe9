"""One transfer function per subband (the alternative to per-channel chirps that
Sec. 2 weighs) against the oracle, in the FP32 and tensor-core forms.

The kernels are the same for both modes; only the chirp-phase table and the
overlap differ, so the tolerances are those of the forms (FP32 1e-5, FP16 2e-3).
That the subband-wide chirp lines the channels up is pinned on the oracle.
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


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 2e-3)])
def test_subband_chirp_tiny_workload(cdmt, orc, prec, tol):
    w = synth.tiny()
    x = w.voltages()
    plan = cdmt.Plan(1, w.nsamp, w.f_centre, BW, w.dms, w.nchan, w.nint, nbin=w.nbin, precision=prec,
                     chirp=cdmt.CDMT_CHIRP_SUBBAND)
    nd = plan.info["nd"]
    assert nd == orc.overlap(1, w.f_centre, BW, w.dms, w.nchan, w.nint, w.nbin, chirp=1)
    assert nd > orc.overlap(1, w.f_centre, BW, w.dms, w.nchan, w.nint, w.nbin)
    g = gpu_filterbank(plan, x)
    plan.device_status()
    o = orc.filterbank(x, w.f_centre, BW, w.dms, w.nchan, w.nint, w.nbin, nd, chirp=1)
    emax, erms = rel_errors(g, o)
    print(f"prec {prec} subband chirp: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert np.all(np.isfinite(g)) and emax <= tol and erms <= tol
    plan.close()


def test_subband_chirp_multi_subband_uneven_dms(cdmt, orc):
    nsamp = 3 * (1 << 15) + 777
    dms = [0.0, 2.5, -1.0, 6.0]
    x = synth.noise(25, 3, nsamp)
    plan = cdmt.Plan(3, nsamp, 130.0, BW, dms, 8, 2, nbin=1 << 15, chirp=cdmt.CDMT_CHIRP_SUBBAND)
    assert plan.info["uniform_dm"] == 0
    g = gpu_filterbank(plan, x)
    o = orc.filterbank(x, 130.0, BW, dms, 8, 2, 1 << 15, plan.info["nd"], chirp=1)
    emax, erms = rel_errors(g, o)
    assert emax <= 1e-5 and erms <= 1e-5
    plan.close()


def test_chirp_mode_rejected(cdmt):
    with pytest.raises(cdmt.CdmtError) as e:
        cdmt.Plan(1, 1 << 17, 135.0, BW, [0.0], 8, 4, nbin=1 << 14, chirp=2)
    assert e.value.status == cdmt.CDMT_EINVAL
