"""Batches of uneven beams in one graph-captured persistent launch per round.

Every round's output of every beam must equal the same segments of a
standalone plan with the beam's chosen parameters (the same kernels run the
same arithmetic, so the match is exact), and one beam is checked against the
FP64 oracle (tolerance of the tensor-core form, 2e-3).
"""
import os

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


def _beams():
    # uneven: subbands, samples, channels, integration and DM lists all differ
    return [
        dict(nsub=3, nsamp=3 * (1 << 16) + 555, f_centre=135.0, dm_first=0.0, dm_step=1.0, ndm=16, nchan=16, nint=8,
             seed=41),
        dict(nsub=2, nsamp=(1 << 17) + 77, f_centre=150.0, dm_first=2.0, dm_step=0.5, ndm=14, nchan=8, nint=4,
             seed=42),
        dict(nsub=1, nsamp=1 << 18, f_centre=120.0, dm_first=0.0, dm_step=3.0, ndm=5, nchan=32, nint=16, seed=43),
    ]


def _device_inputs(beams):
    import torch
    xs, ts = [], []
    for b in beams:
        x = synth.noise(b["seed"], b["nsub"], b["nsamp"])
        xs.append(x)
        ts.append(torch.from_numpy(x).cuda())
    return xs, ts




def test_batch_rounds_match_standalone_plans(cdmt, orc):
    import torch
    beams = _beams()
    xs, ts = _device_inputs(beams)
    for b, t in zip(beams, ts):
        b["d_in"] = t.data_ptr()
        b["bw_sub"] = BW
    batch = cdmt.Batch(beams, out_budget=4 << 20)
    assert batch.nround >= 2
    refs = []
    for b, x, t, inf in zip(beams, xs, ts, batch.infos):
        dms = [b["dm_first"] + i * b["dm_step"] for i in range(b["ndm"])]
        p = cdmt.Plan(b["nsub"], b["nsamp"], b["f_centre"], BW, dms, b["nchan"], b["nint"], nbin=inf.tune.nbin,
                      nd=inf.plan.nd, dm_tile=inf.tune.dm_tile, precision=inf.tune.precision)
        refs.append(cdmt.run(p, t).cpu().numpy())
        p.close()
    stream = torch.cuda.current_stream().cuda_stream
    for r in range(batch.nround):
        batch.run_round(r, stream)
        torch.cuda.synchronize()
        batch.status()
        for i, (b, inf, ref) in enumerate(zip(beams, batch.infos, refs)):
            kc = inf.seg_per_round
            seglen = (inf.plan.mbin - inf.plan.nd) // b["nint"]
            k0 = r * kc
            nk = max(0, min(kc, inf.plan.nseg - k0))
            if nk == 0:
                continue
            got = batch.round_output(i).cpu().numpy()[:, :, :nk * seglen]
            want = ref[:, :, k0 * seglen:(k0 + nk) * seglen]
            assert np.array_equal(got, want), (r, i, float(np.max(np.abs(got - want))))
    # the whole input in one call (rounds in stream order), and beam 0 against the oracle
    batch.run(stream)
    torch.cuda.synchronize()
    batch.status()
    b, inf = beams[0], batch.infos[0]
    dms = [b["dm_first"] + i * b["dm_step"] for i in range(b["ndm"])]
    o = orc.filterbank(xs[0], b["f_centre"], BW, dms, b["nchan"], b["nint"], inf.plan.nbin, inf.plan.nd)
    emax, erms = rel_errors(refs[0], o)
    assert emax <= 2e-3 and erms <= 2e-3
    batch.close()


def test_batch_autotuner_and_cache(cdmt, tmp_path):
    import torch
    beams = _beams()[:2]
    xs, ts = _device_inputs(beams)
    for b, t in zip(beams, ts):
        b["d_in"] = t.data_ptr()
        b["bw_sub"] = BW
    cache = str(tmp_path / "tune.txt")
    stream = torch.cuda.current_stream().cuda_stream
    b1 = cdmt.Batch(beams, autotune=True, tune_cache=cache, stream=stream)
    for inf in b1.infos:
        assert inf.tune.units_per_s > 0 and inf.tune.from_cache == 0
        assert inf.tune.precision in (cdmt.CDMT_PREC_FP32, cdmt.CDMT_PREC_FP16)
    assert os.path.exists(cache) and len(open(cache).read().splitlines()) == 2
    b1.run(stream)
    torch.cuda.synchronize()
    b1.status()
    b2 = cdmt.Batch(beams, autotune=True, tune_cache=cache, stream=stream)
    for i1, i2 in zip(b1.infos, b2.infos):
        assert i2.tune.from_cache == 1
        assert (i2.tune.precision, i2.tune.nbin, i2.tune.dm_tile) == (i1.tune.precision, i1.tune.nbin, i1.tune.dm_tile)
    b1.close()
    b2.close()


def test_batch_rejects_bad_beams(cdmt):
    with pytest.raises(cdmt.CdmtError) as e:
        cdmt.Batch([dict(nsub=1, nsamp=1 << 16, f_centre=135.0, bw_sub=BW, dm_first=0.0, dm_step=1.0, ndm=4,
                         nchan=8, nint=4, d_in=0)])
    assert e.value.status == cdmt.CDMT_EINVAL
