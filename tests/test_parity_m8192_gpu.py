"""Channels of M = 8192 bins in the FP32 form, against the FP64 oracle: the
paper's own application setup (Sec. 4: N_bin = 65536, n_c = 8, M_bin = 8192,
n_d = 2048, no averaging, 195.31-kHz subbands at the bottom of the 114.93 -
116.88 MHz band, DM trials from 0.5 up to 79.5 pc cm^-3).

Tolerance as in the other FP32 parity tests: max |gpu - oracle| / mean(oracle)
<= 1e-5 and ||gpu - oracle|| / ||oracle|| <= 1e-5; an injected pulse keeps its
S/N to 1 %.  At M = 8192 the DM stage runs 512 threads per channel, the last
radix-32 pass shared by lane pairs, so every path through it is checked at this
size too: uneven DM lists (FP64 phase), int8 input, the host pipeline's DM
ranges and the allocation-free entry point."""
import ctypes

import numpy as np
import pytest

import synth
from helpers import gpu_filterbank, pulse_snr, rel_errors

pytestmark = pytest.mark.gpu

TOL = 1e-5
BW = 0.1953125
NBIN = 1 << 16
NCHAN = 8
# the two lowest subbands of the paper's band (edges 114.93 MHz and 115.32 MHz)
FC = 114.93 + BW
# evenly spaced trials over the paper's DM range
DMS = [0.5 + 15.8 * i for i in range(6)]


@pytest.fixture(scope="module")
def cdmt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_00909_gb300 as m
    return m


def _plan(cdmt, nsub, nsamp, fc, dms, nint, **kw):
    return cdmt.Plan(nsub, nsamp, fc, BW, dms, NCHAN, nint, nbin=NBIN, **kw)


@pytest.mark.parametrize("nd", [2048, None])
def test_paper_setup_parity_and_pulse(cdmt, orc, nd):
    """2 subbands, 4 segments and a ragged tail (S = 65536 - 8 n_d), nint 1, a
    pulse at DM 47.9; n_d = 2048 as in the paper, or the overlap rule's own."""
    nsub, nint = 2, 1
    nsamp = NBIN + 3 * (NBIN - 2048 * NCHAN) + 1000
    x = synth.noise(81, nsub, nsamp)
    pulse = synth.Pulse(0.45, DMS[3], 2e-3, 1.0)
    synth.add_pulses(x, [pulse], FC, BW, 81)
    kw = {} if nd is None else {"nd": nd}
    plan = _plan(cdmt, nsub, nsamp, FC, DMS, nint, **kw)
    i = plan.info
    assert i["mbin"] == 8192
    if nd is None:
        assert i["nd"] == orc.overlap(nsub, FC, BW, DMS, NCHAN, nint, NBIN)
    else:
        assert i["nd"] == 2048
    assert (i["nvalid"], i["nseg"], i["nout"]) == orc.grid(nsamp, NBIN, NCHAN, i["nd"], nint)
    g = gpu_filterbank(plan, x)
    assert np.all(np.isfinite(g)), "output not fully written"
    o = orc.filterbank(x, FC, BW, DMS, NCHAN, nint, NBIN, i["nd"])
    emax, erms = rel_errors(g, o)
    print(f"M = 8192, nd {i['nd']}: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert emax <= TOL and erms <= TOL, (emax, erms)
    sg = pulse_snr(g, DMS, pulse, FC, BW, nsub, NCHAN, nint, i["nd"])
    so = pulse_snr(o, DMS, pulse, FC, BW, nsub, NCHAN, nint, i["nd"])
    assert so > 5
    assert abs(sg / so - 1) <= 0.01, (sg, so)
    plan.close()


def test_uneven_dm_list_m8192(cdmt, orc):
    dms = [0.0, 3.7, -5.0, 12.1, 40.0, 39.99]
    nsamp = 2 * NBIN + 4321
    x = synth.noise(82, 1, nsamp)
    plan = _plan(cdmt, 1, nsamp, 120.0, dms, 2)
    assert plan.info["uniform_dm"] == 0 and plan.info["mbin"] == 8192
    g = gpu_filterbank(plan, x)
    o = orc.filterbank(x, 120.0, BW, dms, NCHAN, 2, NBIN, plan.info["nd"])
    emax, erms = rel_errors(g, o)
    assert emax <= TOL and erms <= TOL, (emax, erms)
    plan.close()


def test_int8_input_m8192_equals_dequantised_float(cdmt):
    import torch
    nsub, nsamp = 2, 2 * NBIN + 99
    x = synth.noise(83, nsub, nsamp)
    scale = (np.abs(x).reshape(nsub, -1).max(axis=1) / 127.0).astype(np.float32)
    q = np.clip(np.rint(x / scale[:, None, None]), -127, 127).astype(np.int8)
    deq = q.astype(np.float32) * scale[:, None, None]
    dms = [0.0, 10.0, 20.0]
    pf = _plan(cdmt, nsub, nsamp, 130.0, dms, 4)
    want = gpu_filterbank(pf, deq)
    pf.close()
    pi = _plan(cdmt, nsub, nsamp, 130.0, dms, 4, in_dtype=cdmt.CDMT_IN_I8)
    got = cdmt.run(pi, torch.from_numpy(q).cuda(), scale=torch.from_numpy(scale).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)
    pi.close()


@pytest.mark.parametrize("uniform", [True, False])
def test_host_pipeline_dm_ranges_m8192(cdmt, uniform):
    """float32 host output of a one-tile plan runs each block's DM stage in DM
    ranges (70 DMs: two of 35): bit-identical to the device path."""
    import torch
    nsub, ndm = 2, 70
    nsamp = NBIN + 5 * (NBIN - 512 * NCHAN) + 7
    x = synth.noise(84, nsub, nsamp)
    dms = [30.0 * i / ndm for i in range(ndm)]
    if not uniform:
        dms = sorted(np.random.default_rng(6).uniform(0.0, 30.0, ndm).tolist())
    plan = _plan(cdmt, nsub, nsamp, 140.0, dms, 4, nd=512, dm_tile=ndm, host_block=3)
    assert plan.info["nseg"] == 6
    dev = gpu_filterbank(plan, x)
    hin = torch.from_numpy(x).pin_memory()
    hout = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32).pin_memory()
    plan.execute_host(hin.data_ptr(), hout.data_ptr(), 0, 0)
    assert np.array_equal(hout.numpy(), dev)
    plan.close()


def test_static_entry_m8192(cdmt):
    import torch
    nsub, nsamp, nint = 2, 3 * NBIN + 11, 2
    dm_first, dm_step, ndm = 0.5, 15.8, 6
    dms = [dm_first + i * dm_step for i in range(ndm)]
    plan = _plan(cdmt, nsub, nsamp, FC, dms, nint, nd=2048)
    x = torch.from_numpy(synth.noise(85, nsub, nsamp)).cuda()
    out = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32, device="cuda")
    rc = cdmt.lib().cdmt_execute_static(nsub, nsamp, FC, BW, dm_first, dm_step, ndm, NCHAN, nint, NBIN, 2048,
                                        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == cdmt.CDMT_OK, cdmt.cdmt_last_error(None)
    ref = cdmt.run(plan, x)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    emax, erms = rel_errors(got, ref.cpu().numpy())
    assert emax <= TOL and erms <= TOL, (emax, erms)
    plan.close()
