"""S/N of the five pulses injected into the 64-subband LOFAR-shaped workload,
from the GPU filterbank of each precision form against the FP64 oracle's.

The workload is the benchmark's (64 x 195.3125 kHz subbands 128.75-141.25 MHz,
2^22 samples, N = 2^16, 128 DMs 0..63.5, 16 channels, nint 8) with its five
pulses at DM ~ U(5, 60) and widths 0.2-5 ms.  For each pulse the harness takes
the DM trial nearest the pulse's DM, shifts every channel back by the
closed-form inter-channel delay of Eq. 2, sums the 1024 channels, applies a
boxcar of the pulse width and measures the peak against the median and MAD of
the rest of a window of 2 x 1000 output samples around the pulse (1.3 s).
The oracle computes only the (subband, segment) tiles at that DM that the
window reaches in each channel (Algorithm 1 per segment; segments are
independent).  Each form's S/N must be within 1 % of the oracle's.
"""
import numpy as np
import pytest

import synth
from helpers import pulse_geometry, windowed_snr

pytestmark = pytest.mark.gpu

HALF = 1000
FORMS = [("fp32", 0), ("fp16", 1), ("bf16", 2)]


@pytest.fixture(scope="module")
def cdmt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_00909_gb300 as m
    return m


def test_lofar64_pulse_snr_every_form(cdmt, orc):
    import torch
    w = synth.lofar64()
    x = w.voltages(threads=16)
    xt = torch.from_numpy(x).cuda()
    gpu = {}
    geo = None
    nd = None
    for name, prec in FORMS:
        plan = cdmt.Plan(w.nsub, w.nsamp, w.f_centre, w.bw, w.dms, w.nchan, w.nint, nbin=w.nbin, precision=prec)
        i = plan.info
        if nd is None:
            nd = i["nd"]
            assert nd == orc.overlap(w.nsub, w.f_centre, w.bw, w.dms, w.nchan, w.nint, w.nbin)
            geo = [pulse_geometry(p, w.dms, w.f_centre, w.bw, w.nsub, w.nchan, w.nint, nd) for p in w.pulses]
        assert i["nd"] == nd
        out = torch.empty(plan.out_shape(), dtype=torch.float32, device="cuda")
        cdmt.run(plan, xt, out)
        torch.cuda.synchronize()
        plan.device_status()
        for k, (idm, shifts, wbox, t_exp) in enumerate(geo):
            rows = out[idm].cpu().numpy().astype(np.float64)
            gpu[(name, k)] = windowed_snr(lambda r, a, b: rows[r, a:b], shifts, wbox, t_exp, HALF)
        del out
        plan.close()
        torch.cuda.empty_cache()
    del xt
    L = (w.nbin // w.nchan - nd) // w.nint
    for k, (idm, shifts, wbox, t_exp) in enumerate(geo):
        # the (subband, segment) tiles at this DM trial that the window reaches in each channel
        sh = shifts.reshape(w.nsub, w.nchan)
        need = []
        for s in range(w.nsub):
            a = (t_exp - HALF + int(sh[s].min())) // L
            b = (t_exp + HALF + int(sh[s].max()) - 1) // L
            need += [(s, q) for q in range(a, b + 1)]
        sub = np.array([s for s, _ in need])
        seg = np.array([q for _, q in need])
        tiles = orc.tiles(x, w.f_centre, w.bw, w.dms, w.nchan, w.nint, w.nbin, nd, sub, seg,
                          np.full(len(need), idm))
        # per subband, its segments a_s .. b_s laid end to end: rows from output sample a_s L on
        first = {}
        blocks = {}
        t = 0
        for s in range(w.nsub):
            n = sum(1 for s2, _ in need if s2 == s)
            first[s] = seg[t]
            blocks[s] = np.concatenate([tiles[t + j] for j in range(n)], axis=1)
            t += n

        def rows_at(r, a, b):
            s, c = divmod(r, w.nchan)
            return blocks[s][c, a - first[s] * L:b - first[s] * L]

        so = windowed_snr(rows_at, shifts, wbox, t_exp, HALF)
        assert so > 10, (k, so)
        for name, _ in FORMS:
            sg = gpu[(name, k)]
            print(f"pulse {k} (DM {w.pulses[k].dm:.2f}, trial {w.dms[idm]}): {name} S/N {sg:.3f}, oracle {so:.3f}")
            assert abs(sg / so - 1) <= 0.01, (name, k, sg, so)
