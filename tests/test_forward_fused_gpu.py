"""The forward stage in one persistent launch (M = 4096, n_c <= 16): the decimated
M-point transforms and the n_c-point column DFTs (Sec. 3: "forward FFT", "swap
halves per subband") taken from one ordered work queue, a column item waiting for
its chunk's transforms.  Checked against the FP64 oracle for every column size,
with fewer chunks than the queue's lag and with many, on a partial last chunk,
with int8 input, and bit for bit against the same arithmetic in two launches
(the allocation-free entry point, which keeps them)."""
import ctypes

import numpy as np
import pytest

import synth
from helpers import gpu_filterbank, rel_errors

pytestmark = pytest.mark.gpu

TOL = 1e-5
BW = 0.1953125
MBIN = 4096


@pytest.fixture(scope="module")
def cdmt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_00909_gb300 as m
    return m


@pytest.mark.parametrize("nchan,nsub,nseg", [(2, 3, 5), (4, 3, 5), (8, 1, 3), (16, 3, 5), (16, 4, 9)])
def test_fused_forward_matches_the_oracle(cdmt, orc, nchan, nsub, nseg):
    """nsub * nseg segments in chunks of two: 15 (8 chunks, a partial last one, no more
    than the queue's lag), 3 (2 chunks) and 36 (18 chunks, the steady state)."""
    nbin = nchan * MBIN
    dms = [0.0, 4.0, 8.0, 12.0]
    nint = 4
    nd = orc.overlap(nsub, 140.0, BW, dms, nchan, nint, nbin)
    nsamp = nbin + (nseg - 1) * (nbin - nd * nchan) + 333   # nseg segments and a ragged tail
    x = synth.noise(200 + nchan, nsub, nsamp)
    plan = cdmt.Plan(nsub, nsamp, 140.0, BW, dms, nchan, nint, nbin=nbin)
    assert plan.info["mbin"] == MBIN and plan.info["nd"] == nd
    assert plan.info["nseg"] in (nseg, nseg + 1), plan.info["nseg"]
    g = gpu_filterbank(plan, x)
    assert np.all(np.isfinite(g)), "output not fully written"
    o = orc.filterbank(x, 140.0, BW, dms, nchan, nint, nbin, plan.info["nd"])
    emax, erms = rel_errors(g, o)
    print(f"nchan {nchan}, {nsub} x {nseg} segments: rel_max {emax:.3e} rel_rms {erms:.3e}")
    assert emax <= TOL and erms <= TOL, (emax, erms)
    plan.close()


def test_fused_forward_int8_equals_dequantised_float(cdmt):
    import torch
    nsub, nchan = 5, 16
    nsamp = 7 * (1 << 16) + 99
    x = synth.noise(211, nsub, nsamp)
    scale = (np.abs(x).reshape(nsub, -1).max(axis=1) / 127.0).astype(np.float32)
    q = np.clip(np.rint(x / scale[:, None, None]), -127, 127).astype(np.int8)
    deq = q.astype(np.float32) * scale[:, None, None]
    dms = [0.0, 10.0, 20.0]
    pf = cdmt.Plan(nsub, nsamp, 130.0, BW, dms, nchan, 8, nbin=1 << 16)
    want = gpu_filterbank(pf, deq)
    pf.close()
    pi = cdmt.Plan(nsub, nsamp, 130.0, BW, dms, nchan, 8, nbin=1 << 16, in_dtype=cdmt.CDMT_IN_I8)
    assert pi.info["nseg"] >= 7
    got = cdmt.run(pi, torch.from_numpy(q).cuda(), scale=torch.from_numpy(scale).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)
    pi.close()


def test_fused_forward_equals_two_launches(cdmt):
    """The plan's forward stage (one launch) and the allocation-free entry point's
    (the decimated transforms, then the column DFTs) give the same filterbank bit for
    bit: same FP32 form, DM list, tables and DM-stage kernel."""
    import torch
    nsub, nchan, nint = 6, 16, 8
    nbin = 1 << 16
    dm_first, dm_step, ndm = 1.0, 3.0, 5
    dms = [dm_first + i * dm_step for i in range(ndm)]
    nsamp = 6 * nbin + 4321
    plan = cdmt.Plan(nsub, nsamp, 140.0, BW, dms, nchan, nint, nbin=nbin, dm_tile=ndm)
    nd = plan.info["nd"]
    x = torch.from_numpy(synth.noise(212, nsub, nsamp)).cuda()
    ref = cdmt.run(plan, x)
    out = torch.full(plan.out_shape(), float("nan"), dtype=torch.float32, device="cuda")
    rc = cdmt.lib().cdmt_execute_static(nsub, nsamp, 140.0, BW, dm_first, dm_step, ndm, nchan, nint, nbin, nd,
                                        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == cdmt.CDMT_OK, cdmt.cdmt_last_error(None)
    torch.cuda.synchronize()
    got, want = out.cpu().numpy(), ref.cpu().numpy()
    assert np.all(np.isfinite(want))
    assert np.array_equal(got, want), float(np.max(np.abs(got - want)))
    plan.close()
