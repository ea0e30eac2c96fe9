"""8-bit redigitisation of the filterbank (Sec. 3) against the oracle.

Both sides decide each code in FP32 from the row's mean and standard deviation
rounded to FP32 and the gain 16 / sigma divided in FP32, so a row's codes are
unique given its (mu, sigma): wherever the GPU reports the statistics it used
(cdmt_redigitise, 8-bit served beams) its codes must equal, byte for byte, the
oracle's code step (oracle.codes) applied with them, and the statistics must
agree with the oracle's FP64 ones within 1e-5.  The statistics differ only in
their arithmetic (FP64 sums in order in the oracle; on the GPU FP32 partial sums
per thread with an FP64 combination for long rows, FP32 two-pass mean and
deviation for short ones), so against the oracle's own codes a code may differ
by one where the unrounded value sits within 1e-3 of a rounding boundary; the
host pipeline, which does not report its per-block statistics, is held to that
(at most 1e-4 of the codes).
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


def _boundary_codes(orc, fb, codes):
    """Codes that differ from the oracle's own redigitisation: each by one, on a
    rounding boundary of the oracle's unrounded value.  Returns their number."""
    fb = np.ascontiguousarray(fb, dtype=np.float32)
    rows = fb.shape[1]
    oc, ost = orc.redigitise(fb)
    scale = np.maximum(ost[..., 1], 1e-30)
    diff = codes.astype(np.int32) - oc.astype(np.int32)
    assert np.all(np.abs(diff) <= 1)
    d, t, p = np.nonzero(diff)
    r = rows - 1 - p
    x = 128.0 + (fb[d, r, t].astype(np.float64) - ost[d, r, 0]) * 16.0 / scale[d, r]
    assert np.all(np.abs(x - np.floor(x) - 0.5) < 1e-3), "a code differs away from a rounding boundary"
    return len(d)


def _check(orc, fb, codes, stats, flags=None):
    """Reported statistics within 1e-5 of the oracle's; codes byte for byte the
    oracle's code step with the reported statistics (and flags)."""
    fb = np.ascontiguousarray(fb, dtype=np.float32)
    _, ost = orc.redigitise(fb)
    keep = np.ones(ost.shape[:2], dtype=bool) if flags is None else flags == 0
    mu_g, sg_g = stats[..., 0].astype(np.float64), stats[..., 1].astype(np.float64)
    scale = np.maximum(ost[..., 1], 1e-30)
    assert np.max((np.abs(mu_g - ost[..., 0]) / (np.abs(ost[..., 0]) + scale))[keep], initial=0.0) <= 1e-5
    assert np.max((np.abs(sg_g - ost[..., 1]) / (np.abs(ost[..., 0]) + scale))[keep], initial=0.0) <= 1e-5
    exact = orc.codes(fb, stats, flags)
    assert np.array_equal(codes, exact), f"{int(np.count_nonzero(codes != exact))} codes differ"
    return _boundary_codes(orc, fb, codes) if flags is None else 0


def test_redigitise_tiny_workload(cdmt, orc):
    import torch
    w = synth.tiny()
    x = w.voltages()
    plan = cdmt.Plan(1, w.nsamp, w.f_centre, BW, w.dms, w.nchan, w.nint, nbin=w.nbin)
    fb = cdmt.run(plan, torch.from_numpy(x).cuda())
    stats = torch.empty((len(w.dms), w.nchan, 2), dtype=torch.float32, device="cuda")
    codes = plan.redigitise(fb, stats=stats)
    torch.cuda.synchronize()
    _check(orc, fb.cpu().numpy(), codes.cpu().numpy(), stats.cpu().numpy())
    plan.close()


def test_redigitise_ragged_tiles_and_degenerate_rows(cdmt, orc):
    import torch
    # 3 subbands x 16 channels = 48 rows (< one 64-row tile), nout not a multiple of 64
    nsamp = 3 * (1 << 16) + 999
    plan = cdmt.Plan(3, nsamp, 150.0, BW, [0.0, 7.0, 14.0], 16, 8, nbin=1 << 16)
    ndm, rows, nout = plan.out_shape()
    assert rows % 64 and nout % 64
    g = np.random.default_rng(3)
    fb = g.gamma(8.0, 2.0, (ndm, rows, nout)).astype(np.float32)
    fb[0, 5, :] = 3.5                     # constant row: every code 128
    fb[1, 7, 123] = 1e4                   # an outlier clips at 255
    fb[2, 9, :] = np.where(np.arange(nout) % 2 == 0, 10.0, 14.0)   # two levels: 112 / 144
    fbt = torch.from_numpy(fb).cuda()
    stats = torch.empty((ndm, rows, 2), dtype=torch.float32, device="cuda")
    codes = plan.redigitise(fbt, stats=stats).cpu().numpy()
    torch.cuda.synchronize()
    _check(orc, fb, codes, stats.cpu().numpy())
    assert np.all(codes[0, :, rows - 1 - 5] == 128)
    assert codes[1, 123, rows - 1 - 7] == 255
    assert set(codes[2, 0::2, rows - 1 - 9]) == {112} and set(codes[2, 1::2, rows - 1 - 9]) == {144}
    plan.close()


def test_redigitise_full_tiles_tensor_core_plan(cdmt, orc):
    import torch
    # 8 subbands x 16 channels = 128 rows (two full tiles), FP16 tensor-core filterbank
    nsub, nsamp = 8, 4 * (1 << 16)
    x = synth.noise(41, nsub, nsamp)
    dms = [0.0, 10.0, 20.0, 30.0]
    plan = cdmt.Plan(nsub, nsamp, 135.0, BW, dms, 16, 8, nbin=1 << 16, precision=cdmt.CDMT_PREC_FP16)
    fb = cdmt.run(plan, torch.from_numpy(x).cuda())
    stats = torch.empty((len(dms), nsub * 16, 2), dtype=torch.float32, device="cuda")
    codes = plan.redigitise(fb, stats=stats)
    torch.cuda.synchronize()
    c = codes.cpu().numpy()
    _check(orc, fb.cpu().numpy(), c, stats.cpu().numpy())
    # detected noise: codes centred on 128 with 16 steps per sigma
    assert abs(c.mean() - 128.0) < 0.5 and abs(c.astype(np.float64).std() - 16.0) < 0.5
    plan.close()


@pytest.mark.parametrize("host_block,sk_nsigma", [(2, 0.0), (4, 0.0), (4, 2.0)])
def test_host_pipeline_8bit_blocks(cdmt, orc, host_block, sk_nsigma):
    # Algorithm 1 up to "redigitize" and "copy to host": every block of host_block segments
    # (the last one shorter) has its own statistics; codes must match the oracle applied
    # block by block to the float filterbank of the same plan
    import torch
    nsub, nsamp = 2, 9 * (1 << 14) + 123
    x = synth.noise(42, nsub, nsamp)
    plan = cdmt.Plan(nsub, nsamp, 135.0, BW, [0.0, 6.0, 12.0], 8, 4, nbin=1 << 14, host_block=host_block,
                     sk_nsigma=sk_nsigma)
    ndm, rows, nout = plan.out_shape()
    fb = cdmt.run(plan, torch.from_numpy(x).cuda()).cpu().numpy()
    xh = torch.from_numpy(x).pin_memory()
    u8 = torch.empty((ndm, nout, rows), dtype=torch.uint8).pin_memory()
    kb = plan.execute_host_u8(xh.data_ptr(), u8.data_ptr())
    seglen = nout // plan.info["nseg"]
    assert kb == host_block and plan.info["nseg"] % kb   # several blocks, the last one shorter
    codes = u8.numpy()
    nbad = nflag = 0
    for s0 in range(0, plan.info["nseg"], kb):
        t0, t1 = s0 * seglen, min(plan.info["nseg"], s0 + kb) * seglen
        block = np.ascontiguousarray(fb[:, :, t0:t1])
        oc, ost = orc.redigitise(block)
        diff = codes[:, t0:t1, :].astype(np.int32) - oc.astype(np.int32)
        if sk_nsigma > 0:   # flagged rows (k = 2 nint = 8) are all 128; rows at the threshold are not compared
            oc, _, of = orc.redigitise_sk(block, 8, sk_nsigma)
            sk, _ = orc.spectral_kurtosis(block, 8, sk_nsigma)
            thr = sk_nsigma * orc.sk_sigma(t1 - t0, 8)
            near = np.abs(np.abs(sk - 1.0) - thr) < 1e-4 * thr
            diff = codes[:, t0:t1, :].astype(np.int32) - oc.astype(np.int32)
            diff[:, :, ::-1][np.broadcast_to(near[:, None, :], diff.shape)] = 0
            nflag += int(of.sum())
        d, t, p = np.nonzero(diff)
        r = rows - 1 - p
        xv = 128.0 + (block[d, r, t].astype(np.float64) - ost[d, r, 0]) * 16.0 / ost[d, r, 1]
        assert np.all(np.abs(xv - np.floor(xv) - 0.5) < 1e-3)
        nbad += len(d)
    assert nbad <= max(1, 1e-4 * codes.size), f"{nbad} codes differ on rounding boundaries"
    if sk_nsigma > 0:
        assert nflag >= 1   # a 2-sigma rule flags a few noise rows out of 3 blocks x 3 DMs x 16 rows
    plan.close()


@pytest.mark.parametrize("nsamp_segments", [3, 18])
def test_redigitise_short_and_long_rows(cdmt, orc, nsamp_segments):
    """Rows below 8192 samples take the warp-per-row statistics, longer rows the
    CTA-per-row form: both against the oracle (3066 samples per row: scalar
    loads; 18396: float4 loads)."""
    import torch
    nsamp = nsamp_segments * (1 << 16) + 777
    plan = cdmt.Plan(1, nsamp, 140.0, BW, [0.0, 9.0], 16, 4, nbin=1 << 16)
    ndm, rows, nout = plan.out_shape()
    assert (nout < 8192) == (nsamp_segments == 3)
    g = np.random.default_rng(nsamp_segments)
    fb = g.gamma(4.0, 3.0, (ndm, rows, nout)).astype(np.float32)
    stats = torch.empty((ndm, rows, 2), dtype=torch.float32, device="cuda")
    codes = plan.redigitise(torch.from_numpy(fb).cuda(), stats=stats).cpu().numpy()
    torch.cuda.synchronize()
    _check(orc, fb, codes, stats.cpu().numpy())
    plan.close()


def test_host_pipeline_block_choice_and_staging_growth(cdmt, orc):
    """With host_block left to the plan, 8-bit output takes shorter blocks than
    float32 output; the staging grows when a call needs longer blocks, and every
    call still gives the same result: float32 equal to the device path, codes
    equal between calls and to the oracle's redigitisation block by block."""
    import torch
    nsub, nsamp = 16, 17 * (1 << 14) + 99
    x = synth.noise(77, nsub, nsamp)
    dms = [0.0, 1.5, 3.0, 4.5, 6.0, 7.5, 9.0, 10.5, 12.0, 13.5]
    plan = cdmt.Plan(nsub, nsamp, 140.0, BW, dms, 8, 4, nbin=1 << 14, dm_tile=1)
    ndm, rows, nout = plan.out_shape()
    nseg = plan.info["nseg"]
    seglen = nout // nseg
    fb = cdmt.run(plan, torch.from_numpy(x).cuda()).cpu().numpy()
    xh = torch.from_numpy(x).pin_memory()
    u8a = torch.empty((ndm, nout, rows), dtype=torch.uint8).pin_memory()
    kb = plan.execute_host_u8(xh.data_ptr(), u8a.data_ptr())
    # 10 tiles x 16 subbands x 8 channels = 1280 items per segment: two segments fill 152 SMs x 16
    assert kb == max(2, -(-nseg // 16))
    hout = torch.full((ndm, rows, nout), float("nan"), dtype=torch.float32).pin_memory()
    plan.execute_host(xh.data_ptr(), hout.data_ptr(), 0, 0)   # float32: longer blocks, staging grows
    assert np.array_equal(hout.numpy(), fb)
    u8b = torch.empty_like(u8a)
    assert plan.execute_host_u8(xh.data_ptr(), u8b.data_ptr()) == kb
    assert np.array_equal(u8a.numpy(), u8b.numpy())
    codes = u8a.numpy()
    nbad = 0
    for s0 in range(0, nseg, kb):
        t0, t1 = s0 * seglen, min(nseg, s0 + kb) * seglen
        oc, _ = orc.redigitise(np.ascontiguousarray(fb[:, :, t0:t1]))
        diff = np.abs(codes[:, t0:t1, :].astype(np.int32) - oc.astype(np.int32))
        assert diff.max() <= 1
        nbad += int(np.count_nonzero(diff))
    assert nbad <= max(1, 1e-4 * codes.size), f"{nbad} codes differ on rounding boundaries"
    plan.close()


def _check_sk(orc, fb, codes, stats, flags, k, nsigma):
    """Flags equal to the oracle's except where |SK - 1| lies within 1e-4 of the
    threshold (the two sides take SK from statistics rounded differently); codes
    byte for byte the oracle's code step with the reported statistics and flags
    (flagged rows all 128); statistics of unflagged rows as _check."""
    fb = np.ascontiguousarray(fb, dtype=np.float32)
    nt = fb.shape[2]
    sk, of = orc.spectral_kurtosis(fb, k, nsigma)
    thr = nsigma * orc.sk_sigma(nt, k)
    near = np.abs(np.abs(sk - 1.0) - thr) < 1e-4 * thr
    assert np.all((flags == of) | near)
    _check(orc, fb, codes, stats, flags)
    return int(of.sum())


@pytest.mark.parametrize("nsamp_segments", [3, 18])
def test_redigitise_sk_flags(cdmt, orc, nsamp_segments):
    """Spectral-kurtosis flagging on the warp-per-row (3066 samples) and
    CTA-per-row (18396 samples) statistics: Gamma(2 nint) rows plus impulsive,
    steady and dead rows, against the oracle."""
    import torch
    nsamp = nsamp_segments * (1 << 16) + 777
    nint = 4
    plan = cdmt.Plan(1, nsamp, 140.0, BW, [0.0, 9.0, 18.0], 16, nint, nbin=1 << 16)
    ndm, rows, nout = plan.out_shape()
    k = 2 * nint
    g = np.random.default_rng(60 + nsamp_segments)
    fb = g.gamma(float(k), 1.5, (ndm, rows, nout)).astype(np.float32)
    fb[0, 3, ::25] *= 40.0                     # impulsive RFI
    fb[1, 7] = 12.0 + 0.001 * g.standard_normal(nout).astype(np.float32)   # steady carrier
    fb[2, 11] = 0.0                            # dead channel
    stats = torch.empty((ndm, rows, 2), dtype=torch.float32, device="cuda")
    flags = torch.full((ndm, rows), 7, dtype=torch.uint8, device="cuda")
    codes = plan.redigitise(torch.from_numpy(fb).cuda(), stats=stats, sk_nsigma=3.0, flags=flags)
    torch.cuda.synchronize()
    f = flags.cpu().numpy()
    assert set(np.unique(f)) <= {0, 1}
    assert f[0, 3] == 1 and f[1, 7] == 1 and f[2, 11] == 1
    nflag = _check_sk(orc, fb, codes.cpu().numpy(), stats.cpu().numpy(), f, k, 3.0)
    assert nflag <= 3 + max(2, 0.02 * ndm * rows)
    # sk_nsigma = 0 flags nothing and gives the plain redigitisation
    c0 = plan.redigitise(torch.from_numpy(fb).cuda(), sk_nsigma=0.0, flags=flags)
    torch.cuda.synchronize()
    assert not flags.cpu().numpy().any()
    assert np.array_equal(c0.cpu().numpy(), plan.redigitise(torch.from_numpy(fb).cuda()).cpu().numpy())
    plan.close()
