"""Every output writer stays inside its buffer (canary guards, checked on the host).

compute-sanitizer is not available, so each output is written into the middle of
a larger buffer whose guard regions hold a sentinel; after the call the guards
must be unchanged and the output fully written.  Covered: the device execute
(FP32 and FP16, plain and with DM groups, whose last segments are clipped at
the filterbank's end), the host pipelines (float32 with DM ranges per block, and
8-bit), redigitisation with statistics and flags, and the incoherent stage.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
BW = 0.1953125
GUARD = 8192   # elements on each side


@pytest.fixture(scope="module")
def cdmt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_00909_gb300 as m
    return m


def _guarded(n, dtype, sentinel, device=None, pinned=False):
    import torch
    buf = torch.full((n + 2 * GUARD,), sentinel, dtype=dtype, device=device)
    if pinned:
        buf = buf.pin_memory()
    return buf, buf[GUARD:GUARD + n]


def _guards_intact(buf, n, sentinel):
    b = buf.cpu().numpy()
    return bool(np.all(b[:GUARD] == sentinel) and np.all(b[GUARD + n:] == sentinel))


CASE = dict(nsub=2, fc=60.0, dms=list(np.linspace(0.0, 6.0, 12)), nchan=8, nint=4, nbin=1 << 14, nsamp=54983)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("groups", [0, 3])
def test_device_execute_stays_in_bounds(cdmt, prec, groups):
    import torch
    c = CASE
    plan = cdmt.Plan(c["nsub"], c["nsamp"], c["fc"], BW, c["dms"], c["nchan"], c["nint"], nbin=c["nbin"],
                     precision=prec, chirp=cdmt.CDMT_CHIRP_SUBBAND, dm_groups=groups)
    x = torch.from_numpy(synth.noise(60, c["nsub"], c["nsamp"])).cuda()
    n = int(np.prod(plan.out_shape()))
    buf, out = _guarded(n, torch.float32, -7.25, device="cuda")
    out.fill_(float("nan"))
    plan.execute(x.data_ptr(), out.data_ptr(), 0, 0)
    torch.cuda.synchronize()
    plan.device_status()
    assert _guards_intact(buf, n, -7.25)
    assert torch.isfinite(out).all().item()
    plan.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_host_pipelines_stay_in_bounds(cdmt, prec):
    # float32 blocks whose DM stage runs in DM ranges, and 8-bit blocks, into guarded pinned buffers
    import torch
    nsub, nsamp = 3, 9 * (1 << 14) + 1234
    dms = list(np.linspace(0.0, 12.0, 128))   # one DM tile of 128: float32 blocks in 4 DM ranges
    plan = cdmt.Plan(nsub, nsamp, 135.0, BW, dms, 8, 4, nbin=1 << 14, precision=prec, host_block=3, dm_tile=128)
    assert plan.info["dm_tile"] == 128
    hin = torch.from_numpy(synth.noise(61, nsub, nsamp)).pin_memory()
    n = int(np.prod(plan.out_shape()))
    buf, out = _guarded(n, torch.float32, -7.25, pinned=True)
    out.fill_(float("nan"))
    plan.execute_host(hin.data_ptr(), out.data_ptr(), 0, 0)
    assert _guards_intact(buf, n, -7.25)
    assert torch.isfinite(out).all().item()
    b8, o8 = _guarded(n, torch.uint8, 0xA5, pinned=True)
    plan.execute_host_u8(hin.data_ptr(), o8.data_ptr(), 0)
    assert _guards_intact(b8, n, 0xA5)
    plan.close()


def test_redigitisation_and_incoherent_stage_stay_in_bounds(cdmt):
    import torch
    c = CASE
    plan = cdmt.Plan(c["nsub"], c["nsamp"], c["fc"], BW, c["dms"], c["nchan"], c["nint"], nbin=c["nbin"],
                     precision=cdmt.CDMT_PREC_FP16)
    x = torch.from_numpy(synth.noise(62, c["nsub"], c["nsamp"])).cuda()
    fb = cdmt.run(plan, x)
    ndm, rows, nt = fb.shape
    bc, codes = _guarded(ndm * nt * rows, torch.uint8, 0xA5, device="cuda")
    bs, stats = _guarded(ndm * rows * 2, torch.float32, -7.25, device="cuda")
    bf, flags = _guarded(ndm * rows, torch.uint8, 0xA5, device="cuda")
    plan.redigitise(fb, codes.view(ndm, nt, rows), stats.view(ndm, rows, 2), sk_nsigma=3.0,
                    flags=flags.view(ndm, rows))
    torch.cuda.synchronize()
    assert _guards_intact(bc, codes.numel(), 0xA5) and _guards_intact(bs, stats.numel(), -7.25)
    assert _guards_intact(bf, flags.numel(), 0xA5)
    nt_out, _ = cdmt.cdmt_incoherent_info(plan.handle, -0.5, 0.01, 37)
    bi, inc = _guarded(ndm * 37 * nt_out, torch.float32, -7.25, device="cuda")
    inc.fill_(float("nan"))
    plan.incoherent(fb, -0.5, 0.01, 37, out=inc.view(ndm, 37, nt_out))
    torch.cuda.synchronize()
    assert _guards_intact(bi, inc.numel(), -7.25)
    assert torch.isfinite(inc).all().item()
    plan.close()
