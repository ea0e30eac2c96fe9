"""cdmt_execute_static, the entry point for callers that cannot allocate device
memory (their memory belongs to another framework's pool, or a real-time loop
cannot afford cudaMalloc's synchronisation), against the plan-based entry point.

Called through the C ABI twice in a row, with two different inputs, so that a
result leaking from the first call into the second would show.  Tolerance: the
same as the FP32 parity tests (max |a - b| / mean(b) <= 1e-5); the two paths run
the same kernels and are normally bit-identical.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from helpers import rel_errors

pytestmark = pytest.mark.gpu

BW = 0.1953125
TOL = 1e-5


@pytest.fixture(scope="module")
def cdmt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_00909_gb300 as m
    return m


def _static_call(cdmt, x, out, stream, nsub, nsamp, fc, dm_first, dm_step, ndm, nchan, nint, nbin, nd):
    rc = cdmt.lib().cdmt_execute_static(nsub, nsamp, fc, BW, dm_first, dm_step, ndm, nchan, nint, nbin, nd,
                                        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(stream))
    return rc


def test_static_entry_matches_plan_on_two_calls(cdmt):
    import torch
    nsub, nsamp, fc, nchan, nint, nbin = 2, 1 << 17, 135.0, 8, 4, 1 << 14
    dm_first, dm_step, ndm = 0.0, 5.0, 4
    dms = [dm_first + i * dm_step for i in range(ndm)]
    plan = cdmt.Plan(nsub, nsamp, fc, BW, dms, nchan, nint, nbin=nbin)
    nd = plan.info["nd"]
    stream = torch.cuda.current_stream().cuda_stream
    inputs = [synth.noise(31, nsub, nsamp), synth.noise(32, nsub, nsamp)]
    synth.add_pulses(inputs[1], [synth.Pulse(0.3, 10.0, 1e-3, 0.5)], fc, BW, 32)
    outs = []
    for x in inputs:
        xt = torch.from_numpy(x).cuda()
        out = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32, device="cuda")
        rc = _static_call(cdmt, xt, out, stream, nsub, nsamp, fc, dm_first, dm_step, ndm, nchan, nint, nbin, nd)
        assert rc == cdmt.CDMT_OK, cdmt.cdmt_last_error(None)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    for x, got in zip(inputs, outs):
        ref = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32, device="cuda")
        cdmt.run(plan, torch.from_numpy(x).cuda(), ref)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        emax, erms = rel_errors(got, ref)
        assert emax <= TOL and erms <= TOL, (emax, erms)
    assert not np.array_equal(outs[0], outs[1])
    plan.close()


def test_static_entry_overlap_rule_and_limit(cdmt):
    import torch
    # nd < 0: the overlap rule; the result equals a plan that chose the same nd
    nsub, nsamp, fc, nchan, nint, nbin = 1, 1 << 16, 140.0, 16, 8, 1 << 16
    plan = cdmt.Plan(nsub, nsamp, fc, BW, [0.0, 10.0, 20.0], nchan, nint, nbin=nbin)
    x = torch.from_numpy(synth.noise(33, nsub, nsamp)).cuda()
    out = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32, device="cuda")
    rc = _static_call(cdmt, x, out, torch.cuda.current_stream().cuda_stream, nsub, nsamp, fc, 0.0, 10.0, 3,
                      nchan, nint, nbin, -1)
    assert rc == cdmt.CDMT_OK, cdmt.cdmt_last_error(None)
    ref = cdmt.run(plan, x)
    torch.cuda.synchronize()
    emax, erms = rel_errors(out.cpu().numpy(), ref.cpu().numpy())
    assert emax <= TOL and erms <= TOL
    # beyond the fixed scratch: a clear refusal, nothing launched
    rc = _static_call(cdmt, x, out, 0, 64, 1 << 22, 135.0, 0.0, 0.5, 128, 16, 8, 1 << 16, -1)
    assert rc == cdmt.CDMT_EBUDGET
    assert "static scratch" in cdmt.cdmt_last_error(None)
    plan.close()


def test_static_entry_chunked_segments(cdmt):
    """16 subbands of N = 2^16: the fixed scratch holds the forward spectra of 3
    segments at a time, so the 16 segments run in 6 chunks (forward stage and DM
    stage per chunk, the spectrum region reused); the result equals the plan's."""
    import torch
    nsub, nsamp, fc, nchan, nint, nbin = 16, 1 << 20, 135.0, 16, 8, 1 << 16
    dm_first, dm_step, ndm = 1.0, 2.5, 6
    dms = [dm_first + i * dm_step for i in range(ndm)]
    plan = cdmt.Plan(nsub, nsamp, fc, BW, dms, nchan, nint, nbin=nbin)
    i = plan.info
    per_seg = 16 * nsub * nbin
    assert i["nseg"] >= 3 * (cdmt.CDMT_STATIC_SCRATCH_BYTES // per_seg)   # several chunks
    x = torch.from_numpy(synth.noise(34, nsub, nsamp)).cuda()
    out = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32, device="cuda")
    rc = _static_call(cdmt, x, out, torch.cuda.current_stream().cuda_stream, nsub, nsamp, fc, dm_first, dm_step,
                      ndm, nchan, nint, nbin, i["nd"])
    assert rc == cdmt.CDMT_OK, cdmt.cdmt_last_error(None)
    ref = cdmt.run(plan, x)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    emax, erms = rel_errors(got, ref.cpu().numpy())
    assert emax <= TOL and erms <= TOL, (emax, erms)
    plan.close()
