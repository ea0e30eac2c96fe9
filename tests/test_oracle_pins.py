"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (golden files under tests/golden/), closed forms derived from
Eq. 1 and the unitary transforms, an independent library FFT, a brute-force
dense-matrix evaluation on tiny inputs, and the physics of a pulse dispersed
with the subband-wide transfer function.  No GPU is needed.
"""
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BW = 0.1953125
D = 4.148808e3


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------- FFT


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64, 128, 256])
@pytest.mark.parametrize("sign", [-1, +1])
def test_fft_matches_naive_dft(orc, n, sign):
    g = np.random.default_rng(n)
    x = g.standard_normal(n) + 1j * g.standard_normal(n)
    a, b = orc.fft(x, sign), orc.dft(x, sign)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.sqrt(n) * np.max(np.abs(b))


@pytest.mark.parametrize("n", [2 ** 10, 2 ** 14, 2 ** 16])
def test_fft_matches_numpy(orc, n):
    g = np.random.default_rng(n)
    x = g.standard_normal(n) + 1j * g.standard_normal(n)
    assert np.allclose(orc.fft(x, -1), np.fft.fft(x), rtol=0, atol=1e-10 * np.sqrt(n))
    assert np.allclose(orc.fft(x, +1), np.fft.ifft(x) * n, rtol=0, atol=1e-10 * np.sqrt(n))


def test_naive_dft_on_unit_vectors(orc):
    # the DFT of e_p is the p-th column of the DFT matrix: exp(-2 pi i p k / n)
    n = 12
    for p in range(n):
        e = np.zeros(n, complex)
        e[p] = 1.0
        k = np.arange(n)
        assert np.allclose(orc.dft(e, -1), np.cos(2 * np.pi * p * k / n) - 1j * np.sin(2 * np.pi * p * k / n),
                           atol=1e-13)


# ------------------------------------------------------- printed numbers


def test_eq2_worked_values(orc):
    for nu, dnu, dm, td_ms, dec in _read_table("eq2_worked_values.txt"):
        nu, dnu, dm, td_ms = float(nu), float(dnu), float(dm), float(td_ms)
        got = orc.sweep(nu - dnu / 2, nu + dnu / 2, dm) * 1e3
        assert round(got, int(dec)) == td_ms, (dm, got)


def test_lofar_channelisation_and_volume(orc):
    t = {r[0]: r[1] for r in _read_table("lofar_setup.txt")[1:]}
    bw, nch = float(t["subband_mhz"]), int(t["nchan"])
    nu_s = 135.0
    c0, c1 = orc.channel_centre(nu_s, bw, nch, 0), orc.channel_centre(nu_s, bw, nch, 1)
    assert round((c1 - c0) * 1e3, 2) == float(t["chan_khz_printed"])
    assert round(nch / (bw * 1e6) * 1e6, 2) == float(t["tsamp_us_printed"])
    assert int(t["nbin"]) // nch == int(t["mbin"])
    nsamp = int(float(t["seconds_perf"]) * bw * 1e6)
    _, _, nout = orc.grid(nsamp, int(t["nbin"]), nch, int(t["nd"]), 1)
    gib = nout * nch * int(t["nsub_perf"]) / 2 ** 30
    assert round(gib, 1) == float(t["out_gib_per_dm"]), gib


def test_paper_overlap_covers_rule(orc):
    # Sec. 5: N_bin 65536, n_d 2048, n_c 8 for subbands 114.93-116.88 MHz up to DM 80.
    # The rule's n_d (lowest channel, Eq. 2) must not exceed the n_d the paper used.
    nd = orc.overlap(10, (114.93 + 116.88) / 2, BW, [80.0], 8, 1, 65536)
    assert 0 < nd <= 2048


# ------------------------------------------------ closed forms from Eq. 1


def _fb(orc, x, dms, nchan, nint, nbin, nd, fc=135.0):
    return orc.filterbank(x, fc, BW, dms, nchan, nint, nbin, nd)


@pytest.mark.parametrize("c", [0, 3, 5, 7])
def test_tone_at_channel_centre_is_dm_invariant(orc, c):
    # A tone at exactly nu_c sits on bin j = M/2 of channel c, where Eq. 1 is 1 at
    # every DM; unitary transforms give |y|^2 = n_c |A|^2 per polarisation.
    nchan, nint, nbin, nd = 8, 4, 1024, 16
    m = nbin // nchan
    off = (c * m + m // 2 - nbin // 2) * BW / nbin
    ax, ay = 0.7 - 0.2j, 0.3 + 0.4j
    x = synth.tone(3 * nbin, off, BW, ax, ay)
    fb = _fb(orc, x, [0.0, 7.3, 50.0], nchan, nint, nbin, nd)
    want = nint * nchan * (abs(ax) ** 2 + abs(ay) ** 2)
    # the voltages are float32, so the tone carries ~1e-8 relative rounding noise
    assert np.allclose(fb[:, c, :], want, rtol=1e-6, atol=0)
    others = np.delete(fb, c, axis=1)
    assert np.max(np.abs(others)) < 1e-6 * want


def test_impulse_lands_in_one_sample_per_channel(orc):
    # An impulse A at input n0 = k S + n_c m0 (inside segment k's kept region) at
    # DM 0 gives |y|^2 = |A|^2 / n_c in every channel at output m0 - nd/2 of that
    # segment, and zero elsewhere.
    nchan, nint, nbin, nd = 8, 1, 512, 8
    m = nbin // nchan
    s_valid = nbin - nd * nchan
    x = np.zeros((1, 3 * nbin, 4), np.float32)
    k, m0 = 1, 20
    n0 = k * s_valid + nchan * m0
    x[0, n0, 0], x[0, n0, 1] = 1.5, -0.5
    fb = _fb(orc, x, [0.0], nchan, nint, nbin, nd)[0]
    t = k * (m - nd) + m0 - nd // 2
    want = (1.5 ** 2 + 0.5 ** 2) / nchan
    assert np.allclose(fb[:, t], want, rtol=1e-12)
    fb[:, t] = 0
    assert np.max(np.abs(fb)) < 1e-12
    # moving the impulse by n_c input samples moves the output by exactly one sample
    x2 = np.zeros_like(x)
    x2[0, n0 + nchan, 0] = 1.0
    fb2 = _fb(orc, x2, [0.0], nchan, nint, nbin, nd)[0]
    assert np.all(np.argmax(fb2, axis=1) == t + 1)


def test_parseval_per_segment(orc):
    # |H| = 1 and both transforms are unitary, so energy is conserved before the
    # overlap is discarded, at any DM.
    g = np.random.default_rng(5)
    n, nchan = 4096, 16
    xx = g.standard_normal(n) + 1j * g.standard_normal(n)
    for dm in (0.0, 30.0):
        y = orc.segment_channels(xx, nchan, 120.0, BW, dm)
        assert np.isclose(np.sum(np.abs(y) ** 2), np.sum(np.abs(xx) ** 2), rtol=1e-12)


def test_channel_chirp_inverts_in_segment_dispersion(orc):
    # Disperse one segment's impulse by the inverse of the dedispersion chirp of
    # each channel (the oracle-internal closed form) and dedisperse at DM_true:
    # the result equals the undispersed impulse; other trials do not.
    nchan, n = 8, 2048
    m = n // nchan
    nu_s, dm_true = 120.0, 40.0
    x = np.zeros(n, complex)
    x[nchan * 100] = 1.0
    ref = orc.segment_channels(x, nchan, nu_s, BW, 0.0)
    X = np.fft.fftshift(np.fft.fft(x))
    nu = (np.arange(m) - m / 2) * BW / n
    for c in range(nchan):
        nuc = nu_s - BW / 2 + (c + 0.5) * BW / nchan
        X[c * m:(c + 1) * m] *= np.exp(2j * np.pi * 1e6 * D * dm_true * nu ** 2 / (nuc ** 2 * (nuc + nu)))
    xd = np.fft.ifft(np.fft.ifftshift(X))
    y = orc.segment_channels(xd, nchan, nu_s, BW, dm_true)
    assert np.max(np.abs(y - ref)) < 1e-10
    y2 = orc.segment_channels(xd, nchan, nu_s, BW, dm_true - 10.0)
    assert np.max(np.abs(np.abs(y2) - np.abs(ref))) > 0.1


def _physical_impulse(nsamp, fc, dm, t0_samp):
    # a one-sample impulse at time t0 (subband centre), dispersed with the
    # subband-wide transfer function: the independent physical forward model
    x = np.zeros(nsamp, complex)
    x[t0_samp] = 1.0
    f = np.fft.fftfreq(nsamp, d=1.0 / (BW * 1e6)) / 1e6
    h = np.exp(2j * np.pi * 1e6 * D * dm * f ** 2 / (fc ** 2 * (fc + f)))
    xd = np.fft.ifft(np.fft.fft(x) * h)
    out = np.zeros((1, nsamp, 4), np.float32)
    out[0, :, 0], out[0, :, 1] = xd.real, xd.imag
    return out


def test_physical_impulse_recovered_at_true_dm(orc):
    # At the true DM, channel c holds the pulse at the closed-form inter-channel
    # delay D DM (nu_c^-2 - nu_s^-2) (Eq. 1 per channel minus Eq. 1 per subband is
    # a pure delay), concentrated in the two nearest samples; at the DM = 0 trial
    # the pulse is smeared and arrives earlier in higher channels.
    fc, dm_true, nchan, nbin, nd = 135.0, 10.0, 8, 1 << 14, 32
    nsamp = 1 << 15
    r = BW * 1e6
    t0 = 20000
    x = _physical_impulse(nsamp, fc, dm_true, t0)
    dms = [0.0, 5.0, 10.0, 15.0]
    fb = _fb(orc, x, dms, nchan, 1, nbin, nd, fc)
    m = nbin // nchan
    sv = nbin - nd * nchan
    for c in range(nchan):
        nuc = fc - BW / 2 + (c + 0.5) * BW / nchan
        delay = D * dm_true * (1 / nuc ** 2 - 1 / fc ** 2) * r / nchan   # output samples
        t_exp = t0 / nchan + delay - nd / 2     # global output index (segments tile seamlessly)
        row = fb[2, c]
        e = np.sum(row)
        i0 = int(np.floor(t_exp))
        frac = (row[i0] + row[i0 + 1]) / e
        assert abs(np.argmax(row) - t_exp) <= 1.0, (c, np.argmax(row), t_exp)
        assert frac >= 0.8, (c, frac)
        for idm in (0, 1, 3):
            other = fb[idm, c]
            j = int(np.argmax(other))
            assert (other[j] + max(other[j - 1], other[j + 1])) / np.sum(other) < 0.6
    # sign pin: at DM 0 the dispersed pulse's centroid is earlier in higher channels
    cen = [np.sum(np.arange(fb.shape[2]) * fb[0, c]) / np.sum(fb[0, c]) for c in range(nchan)]
    assert np.all(np.diff(cen) < 0)
    assert sv * 2 <= nsamp  # the pulse sits inside the segment grid


def test_brute_force_dense_matrices(orc):
    # Tiny sizes: the whole filterbank written with dense DFT matrices and
    # explicit loops (no FFT), nsamp 256, N 64, n_c 4, nd 4, 2 DMs.
    g = np.random.default_rng(11)
    nsamp, nbin, nchan, nd, nint = 256, 64, 4, 4, 2
    fc = 60.0
    dms = [3.0, 17.0]
    x = (g.standard_normal((1, nsamp, 4)) * 0.7).astype(np.float32)
    fb = _fb(orc, x, dms, nchan, nint, nbin, nd, fc)
    m = nbin // nchan
    sv = nbin - nd * nchan
    nseg = (nsamp - nbin) // sv + 1
    n = np.arange(nbin)
    FN = np.exp(-2j * np.pi * np.outer(n, n) / nbin) / np.sqrt(nbin)
    jj = np.arange(m)
    FMi = np.exp(2j * np.pi * np.outer(jj, jj) / m) / np.sqrt(m)
    L = (m - nd) // nint
    want = np.zeros((len(dms), nchan, nseg * L))
    for k in range(nseg):
        pw = np.zeros((len(dms), nchan, m))
        for p in range(2):
            seg = x[0, k * sv:k * sv + nbin, 2 * p] + 1j * x[0, k * sv:k * sv + nbin, 2 * p + 1]
            spec = FN @ seg.astype(complex)
            spec = np.concatenate([spec[nbin // 2:], spec[:nbin // 2]])
            for a, dm in enumerate(dms):
                for c in range(nchan):
                    nuc = fc - BW / 2 + (c + 0.5) * BW / nchan
                    nu = (jj - m / 2) * BW / nbin
                    ch = spec[c * m:(c + 1) * m] * np.exp(-2j * np.pi * 1e6 * D * dm * nu ** 2 / (nuc ** 2 * (nuc + nu)))
                    ch = np.concatenate([ch[m // 2:], ch[:m // 2]])
                    pw[a, c] += np.abs(FMi @ ch) ** 2
        kept = pw[:, :, nd // 2:m - nd // 2]
        want[:, :, k * L:(k + 1) * L] = kept.reshape(len(dms), nchan, L, nint).sum(-1)
    assert np.allclose(fb, want, rtol=1e-11, atol=1e-12)


def test_noise_mean_and_variance(orc):
    # Complex white noise with E|x|^2 = sigma2 per pol stays white under unitary
    # maps, so each output is Gamma(2 nint, sigma2): mean 2 sigma2 nint, variance
    # 2 nint sigma2^2.
    sigma2, nint, nchan, nbin = 1.0, 4, 8, 4096
    x = synth.noise(7, 1, 1 << 16, sigma2)
    fb = _fb(orc, x, [0.0, 20.0], nchan, nint, nbin, 16)
    v = fb.ravel()
    mu, se = v.mean(), v.std() / np.sqrt(v.size)
    assert abs(mu - 2 * sigma2 * nint) < 3 * se + 0.0
    var_want = 2 * nint * sigma2 ** 2
    # standard error of a sample variance for a Gamma(k) variable: var * sqrt((2 + 6/k)/n)
    se_var = var_want * np.sqrt((2 + 6 / (2 * nint)) / v.size)
    assert abs(v.var() - var_want) < 4 * se_var


def test_tiles_reproduce_filterbank(orc):
    w = synth.tiny()
    x = w.voltages()[:, :1 << 16]
    nd = 32
    fb = orc.filterbank(x, w.f_centre, w.bw, w.dms, w.nchan, w.nint, w.nbin, nd)
    sub, seg, dmi = [0, 0, 0], [0, 2, 3], [1, 3, 0]
    t = orc.tiles(x, w.f_centre, w.bw, w.dms, w.nchan, w.nint, w.nbin, nd, sub, seg, dmi)
    L = (w.nbin // w.nchan - nd) // w.nint
    for i in range(3):
        assert np.array_equal(t[i], fb[dmi[i], :, seg[i] * L:(seg[i] + 1) * L])


def test_overlap_rule_values(orc):
    # tiny workload: lowest channel 134.9023-134.9268 MHz, DM 15 -> r t_d / n_c = 30.2 -> 32
    assert orc.overlap(1, 135.0, BW, [0, 5, 10, 15], 8, 4, 1 << 14) == 32
    # 64 subbands 128.75-141.25 MHz, DM 63.5, n_c 16 -> 36.8 -> 38, (4096-38) % 8 != 0 -> 40
    assert orc.overlap(64, 135.0, BW, [0.5 * i for i in range(128)], 16, 8, 1 << 16) == 40
    # no dispersion at all needs no overlap
    assert orc.overlap(1, 135.0, BW, [0.0], 8, 4, 1 << 14) == 0


def test_grid_rejects_bad_shapes(orc):
    with pytest.raises(ValueError):
        orc.grid(100, 1024, 8, 8, 4)        # nsamp < N
    with pytest.raises(ValueError):
        orc.grid(4096, 1024, 8, 128, 4)     # S <= 0
    assert orc.grid(4096, 1024, 8, 8, 4) == (960, 4, 4 * 120 // 4)


def test_overlap_covers_every_channel_and_is_minimal(orc):
    # Sec. 2: the overlap must hold the chirp of the channel with the largest sweep
    # (the lowest one).  Invariant: nd >= r t_d(c) / n_c for every channel of every
    # subband (t_d from Eq. 2, pinned above), and nd - 2 fails that or the
    # divisibility of (M - nd) by nint.  A low, wide band makes channels differ.
    nsub, fc, nchan, nint, nbin = 4, 60.0, 4, 2, 1 << 16
    dms = [0.0, 37.0, 100.0]
    nd = orc.overlap(nsub, fc, BW, dms, nchan, nint, nbin)
    r = BW * 1e6
    need = 0.0
    for s in range(nsub):
        nus = orc.subband_centre(nsub, fc, BW, s)
        for c in range(nchan):
            nuc = orc.channel_centre(nus, BW, nchan, c)
            lo, hi = nuc - BW / nchan / 2, nuc + BW / nchan / 2
            need = max(need, r * orc.sweep(lo, hi, max(dms)) / nchan)
    m = nbin // nchan
    assert nd >= need and nd % 2 == 0 and (m - nd) % nint == 0
    assert nd - 2 < need or (m - nd + 2) % nint != 0


# ---------------------------------------------------------------- one transfer function per subband
# The alternative Sec. 2 sets the per-channel chirp against: Eq. 1 about the subband
# centre for every bin.  It removes the dispersion across the whole subband, so all
# channels of a subband line up, at the cost of an overlap that holds the subband's sweep.


def test_subband_chirp_aligns_channels(orc):
    fc, dm_true, nchan, nbin = 135.0, 10.0, 8, 1 << 14
    dms = [0.0, 5.0, 10.0, 15.0]
    nd = orc.overlap(1, fc, BW, dms, nchan, 1, nbin, chirp=1)
    assert nd > orc.overlap(1, fc, BW, dms, nchan, 1, nbin)
    nsamp, t0 = 1 << 15, 20000
    x = _physical_impulse(nsamp, fc, dm_true, t0)
    fb = orc.filterbank(x, fc, BW, dms, nchan, 1, nbin, nd, chirp=1)
    t_exp = t0 / nchan - nd / 2    # the same output sample in every channel: no inter-channel delay
    for c in range(nchan):
        row = fb[2, c]
        i0 = int(np.floor(t_exp))
        assert abs(np.argmax(row) - t_exp) <= 1.0, (c, np.argmax(row), t_exp)
        assert (row[i0] + row[i0 + 1]) / np.sum(row) >= 0.8
        for idm in (0, 1, 3):
            other = fb[idm, c]
            j = int(np.argmax(other))
            assert (other[j] + max(other[j - 1], other[j + 1])) / np.sum(other) < 0.6


def test_subband_chirp_is_the_channel_chirp_for_one_channel(orc):
    g = np.random.default_rng(21)
    x = (g.standard_normal((2, 1 << 15, 4)) * 0.5).astype(np.float32)
    dms = [0.0, 4.0, 9.0]
    nd0 = orc.overlap(2, 135.0, BW, dms, 1, 2, 1 << 13)
    assert 0 < nd0 and orc.overlap(2, 135.0, BW, dms, 1, 2, 1 << 13, chirp=1) == nd0
    a = orc.filterbank(x, 135.0, BW, dms, 1, 2, 1 << 13, nd0)
    b = orc.filterbank(x, 135.0, BW, dms, 1, 2, 1 << 13, nd0, chirp=1)
    assert np.array_equal(a, b)


def test_subband_overlap_covers_subband_sweep_and_is_minimal(orc):
    nsub, fc, nchan, nint, nbin = 4, 60.0, 4, 2, 1 << 16
    dms = [0.0, 37.0, 11.0]
    nd = orc.overlap(nsub, fc, BW, dms, nchan, nint, nbin, chirp=1)
    r = BW * 1e6
    need = max(r * orc.sweep(orc.subband_centre(nsub, fc, BW, s) - BW / 2,
                             orc.subband_centre(nsub, fc, BW, s) + BW / 2, max(dms)) / nchan for s in range(nsub))
    m = nbin // nchan
    assert nd >= need and nd % 2 == 0 and (m - nd) % nint == 0
    assert nd - 2 < need or (m - nd + 2) % nint != 0


def test_subband_chirp_is_unitary(orc):
    g = np.random.default_rng(22)
    x = g.standard_normal(4096) + 1j * g.standard_normal(4096)
    y = orc.segment_channels(x, 8, 135.0, BW, 33.0, chirp=1)
    assert np.isclose(np.sum(np.abs(y) ** 2), np.sum(np.abs(x) ** 2), rtol=1e-12)


# ---------------------------------------------------------------- redigitisation (Sec. 3)
# Offsets and scales come from each channel's mean and standard deviation over the
# block; 128 is the mean and 16 code steps span one standard deviation.


def test_redigitise_two_level_channel(orc):
    # half the samples at a, half at b: mean (a+b)/2, sigma (b-a)/2, so a -> 128 - 16, b -> 128 + 16
    fb = np.tile(np.array([10.0, 14.0], dtype=np.float32), 50)[None, None, :]
    codes, st = orc.redigitise(fb)
    assert st[0, 0, 0] == 12.0 and st[0, 0, 1] == 2.0
    assert set(codes[0, 0::2, 0]) == {112} and set(codes[0, 1::2, 0]) == {144}


def test_redigitise_constant_channel_is_the_mean_code(orc):
    fb = np.full((2, 3, 40), 7.25, dtype=np.float32)
    codes, st = orc.redigitise(fb)
    assert np.all(codes == 128) and np.all(st[..., 1] == 0.0)


def test_redigitise_clips_an_outlier(orc):
    # N-1 zeros and one X: the outlier sits 16 sqrt(N-1) = 160 steps above the mean -> 255;
    # the zeros sit 16 / sqrt(N-1) = 1.6 steps below -> 126
    n = 101
    fb = np.zeros((1, 1, n), dtype=np.float32)
    fb[0, 0, 37] = 100.0
    codes, _ = orc.redigitise(fb)
    assert codes[0, 37, 0] == 255
    assert set(np.delete(codes[0, :, 0], 37)) == {126}


def test_redigitise_gaussian_row_statistics(orc):
    g = np.random.default_rng(11)
    fb = (40.0 + 3.0 * g.standard_normal((1, 1, 200000))).astype(np.float32)
    codes, st = orc.redigitise(fb)
    c = codes[0, :, 0].astype(np.float64)
    assert abs(st[0, 0, 0] - 40.0) < 0.05 and abs(st[0, 0, 1] - 3.0) < 0.05
    assert abs(c.mean() - 128.0) < 0.1 and abs(c.std() - 16.0) < 0.1


def test_redigitise_order_and_independence(orc):
    # each (DM, channel) is quantised on its own statistics, and channel r of the
    # increasing-frequency rows lands at position rows - 1 - r (decreasing frequency)
    g = np.random.default_rng(12)
    fb = (g.random((3, 5, 64)) * (1.0 + np.arange(5))[None, :, None]).astype(np.float32)
    codes, _ = orc.redigitise(fb)
    assert codes.shape == (3, 64, 5)
    for d in range(3):
        for r in range(5):
            one, _ = orc.redigitise(fb[d:d + 1, r:r + 1, :])
            assert np.array_equal(codes[d, :, 5 - 1 - r], one[0, :, 0])


def test_redigitise_scale_invariance(orc):
    # scaling a channel by a power of two scales mean and sigma exactly: codes unchanged
    g = np.random.default_rng(13)
    fb = g.gamma(4.0, 2.0, (2, 4, 500)).astype(np.float32)
    a, _ = orc.redigitise(fb)
    b, _ = orc.redigitise(fb * np.float32(8.0))
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- incoherent stage (Sec. 4)
# Each coherent filterbank is incoherently dedispersed over fine DM trials around its
# coherent DM by shifting every channel by its dispersive delay and summing.

INC = dict(nsub=3, nchan=4, f_centre=135.0, bw=BW, nint=2)


def _row_freqs(nsub, nchan, f_centre, bw, chirp=0):
    out = []
    for s in range(nsub):
        nus = f_centre + (s - (nsub - 1) / 2) * bw
        for c in range(nchan):
            out.append(nus if chirp else nus - bw / 2 + (c + 0.5) * bw / nchan)
    return np.array(out)


def test_incoherent_zero_dm_is_the_channel_sum(orc):
    g = np.random.default_rng(31)
    rows = INC["nsub"] * INC["nchan"]
    fb = g.random((1, rows, 300)).astype(np.float32)
    out, d = orc.incoherent(fb, INC["nsub"], INC["nchan"], INC["f_centre"], BW, INC["nint"], [0.5], -0.5, 0.002, 1)
    assert np.all(d == 0) and out.shape == (1, 1, 300)
    assert np.allclose(out[0, 0], fb[0].astype(np.float64).sum(axis=0), rtol=1e-12, atol=0)


@pytest.mark.parametrize("chirp", [0, 1])
def test_incoherent_dispersed_impulse_lines_up_at_its_dm(orc, chirp):
    # rows get a unit impulse at their arrival time for DM 2.4 (Eq. 2 delays relative to the
    # top reference frequency, at the output sample time nint * nchan / bw); the trial at
    # DM 2.4 collects all of them in one sample, every other trial fewer
    nsub, nchan, fc, nint = INC["nsub"], INC["nchan"], INC["f_centre"], INC["nint"]
    nu = _row_freqs(nsub, nchan, fc, BW, chirp)
    tsamp = nint * nchan / (BW * 1e6)
    dm_true, t0 = 2.4, 50
    arr = np.rint(D * dm_true * (nu ** -2 - nu.max() ** -2) / tsamp).astype(int)
    fb = np.zeros((1, len(nu), 400), np.float32)
    fb[0, np.arange(len(nu)), t0 + arr] = 1.0
    out, d = orc.incoherent(fb, nsub, nchan, fc, BW, nint, [2.0], -0.5, 0.05, 21, chirp=chirp)
    k_true = 18   # 2.0 - 0.5 + 18 * 0.05 = 2.4
    assert np.isclose(out[0, k_true].max(), len(nu))
    best = out[0].max(axis=1)
    assert np.argmax(best) == k_true and np.all(np.delete(best, k_true) < len(nu))


def test_incoherent_delay_table(orc):
    nsub, nchan, fc, nint = INC["nsub"], INC["nchan"], INC["f_centre"], INC["nint"]
    fb = np.zeros((2, nsub * nchan, 4000), np.float32)
    _, d = orc.incoherent(fb, nsub, nchan, fc, BW, nint, [3.0, 40.0], -0.5, 0.002, 500)
    top = np.argmax(_row_freqs(nsub, nchan, fc, BW))
    assert d.min() == 0
    assert np.all(np.diff(d.astype(int), axis=1) >= 0)                 # more DM, more delay
    assert np.all(d[..., top] == d[..., top][0, 0])                     # the top channel never moves
    assert np.all(np.diff(d[:, :, ::-1].astype(int), axis=2) >= 0)      # lower channels arrive later


def test_incoherent_is_linear_and_shift_covariant(orc):
    g = np.random.default_rng(32)
    nsub, nchan, fc, nint = INC["nsub"], INC["nchan"], INC["f_centre"], INC["nint"]
    a = g.random((2, nsub * nchan, 600)).astype(np.float32)
    b = g.random((2, nsub * nchan, 600)).astype(np.float32)
    args = (nsub, nchan, fc, BW, nint, [1.0, 6.0], -0.5, 0.1, 11)
    oa, _ = orc.incoherent(a, *args)
    ob, _ = orc.incoherent(b, *args)
    oab, _ = orc.incoherent(a + np.float32(2.0) * b, *args)
    assert np.allclose(oab, oa + 2.0 * ob, rtol=1e-6)
    sh, _ = orc.incoherent(np.roll(a, 5, axis=2), *args)
    assert np.allclose(sh[..., 5:], oa[..., :-5], rtol=1e-12)


# ---- spectral kurtosis (Sec. 6, future work: generalised SK estimator)

@pytest.mark.parametrize("k", [1, 16])
def test_sk_gamma_noise_mean_and_spread(orc, k):
    # rows of Gamma(k) samples (each a sum of k exponential powers): SK averages 1 and spreads
    # by sqrt(2 (k + 1) / (k n)); k = 1 is the classic estimator, whose variance is 4 / n
    g = np.random.default_rng(21 + k)
    n, nrow = 800, 3000
    fb = g.gamma(float(k), 2.5, (1, nrow, n)).astype(np.float32)
    sk, fl = orc.spectral_kurtosis(fb, k, 3.0)
    s = orc.sk_sigma(n, k)
    assert abs(s - np.sqrt(2.0 * (k + 1) / (k * n))) < 1e-15
    if k == 1:
        assert abs(s * s - 4.0 / n) < 1e-15
    assert abs(sk.mean() - 1.0) < 4.0 * s / np.sqrt(nrow)
    assert abs(sk.std() / s - 1.0) < 0.08
    assert fl.mean() < 0.01          # a 3-sigma test flags a few rows in a thousand


def test_sk_equals_brute_force_moments(orc):
    # SK from the definition with numpy sums in FP64, on a ragged row length
    g = np.random.default_rng(31)
    fb = g.gamma(8.0, 1.0, (2, 3, 37)).astype(np.float32)
    sk, _ = orc.spectral_kurtosis(fb, 8, 3.0)
    x = fb.astype(np.float64)
    n = x.shape[2]
    s1, s2 = x.sum(axis=2), (x * x).sum(axis=2)
    want = (n * 8 + 1.0) / (n - 1.0) * (n * s2 / (s1 * s1) - 1.0)
    assert np.allclose(sk, want, rtol=1e-12, atol=0)


def test_sk_flags_impulsive_and_steady_rows(orc):
    g = np.random.default_rng(41)
    k, n = 16, 2000
    fb = g.gamma(float(k), 1.0, (1, 4, n)).astype(np.float32)
    fb[0, 1, ::20] *= 30.0                       # impulsive RFI in 5 % of the samples: SK >> 1
    fb[0, 2] = 100.0 + 0.01 * g.standard_normal(n).astype(np.float32)   # a steady carrier: SK << 1
    fb[0, 3] = 0.0                               # a dead channel: SK = 0
    sk, fl = orc.spectral_kurtosis(fb, k, 3.0)
    assert fl[0, 0] == 0 and abs(sk[0, 0] - 1.0) < 3.0 * orc.sk_sigma(n, k)
    assert fl[0, 1] == 1 and sk[0, 1] > 5.0
    assert fl[0, 2] == 1 and sk[0, 2] < 0.01
    assert fl[0, 3] == 1 and sk[0, 3] == 0.0
    # single-sample rows are never flagged
    _, f1 = orc.spectral_kurtosis(fb[:, :, :1], k, 3.0)
    assert not f1.any()


def test_redigitise_sk_zaps_flagged_rows_only(orc):
    g = np.random.default_rng(51)
    k, n, rows = 16, 1000, 6
    fb = g.gamma(float(k), 1.0, (2, rows, n)).astype(np.float32)
    fb[1, 4, ::10] *= 50.0
    codes, st, fl = orc.redigitise_sk(fb, k, 3.0)
    c0, st0 = orc.redigitise(fb)
    assert np.array_equal(st, st0)
    _, f2 = orc.spectral_kurtosis(fb, k, 3.0)
    assert np.array_equal(fl, f2) and fl[1, 4] == 1
    for d in range(2):
        for r in range(rows):
            col = rows - 1 - r
            if fl[d, r]:
                assert np.all(codes[d, :, col] == 128)
            else:
                assert np.array_equal(codes[d, :, col], c0[d, :, col])


# ---------------------------------------------------------------- overlap per DM group
# Sec. 5: digifil picks the overlap per DM, where cdmt sizes one overlap for the
# largest DM of the list.  Grouped plans give each contiguous group of trials the
# overlap its own largest DM needs, and keep the ungrouped time axis and length.


def _grouped_need(orc, nsub, fc, nchan, dm_abs, chirp):
    # r t_d / n_c for the widest sweep of any channel (chirp 0) or subband (chirp 1), Eq. 2
    r, need = BW * 1e6, 0.0
    for s in range(nsub):
        nus = orc.subband_centre(nsub, fc, BW, s)
        spans = [(nus - BW / 2, nus + BW / 2)] if chirp else [
            (orc.channel_centre(nus, BW, nchan, c) - BW / nchan / 2, orc.channel_centre(nus, BW, nchan, c) + BW / nchan / 2)
            for c in range(nchan)]
        for lo, hi in spans:
            need = max(need, r * orc.sweep(lo, hi, dm_abs) / nchan)
    return need


@pytest.mark.parametrize("chirp,groups", [(0, 2), (1, 4), (1, 3)])
def test_grouped_overlaps_cover_their_group_and_are_minimal(orc, chirp, groups):
    # Invariants of each group's overlap: even, (M - nd_g) divisible by nint, at least
    # r t_d / n_c for the group's largest |DM| (Eq. 2 over every channel or subband), its
    # segments (starting off_g = (nd_max - nd_g) n_c / 2 samples in) cover the ungrouped
    # length, and the next smaller candidate fails one of these.  The group holding the
    # largest |DM| has nd_max and no offset.
    nsub, fc, nchan, nint, nbin = 2, 60.0, 8, 2, 1 << 13
    nsamp = 6 * nbin + 1000
    dms = np.linspace(0.0, 4.2, 8) if chirp else np.linspace(0.0, 30.0, 7)
    layout, nd_max, nout = orc.grouped_layout(nsub, nsamp, fc, BW, dms, nchan, nint, nbin, groups, chirp)
    m = nbin // nchan
    assert [g[0] for g in layout] == [g * len(dms) // groups for g in range(groups)]
    assert sum(g[1] for g in layout) == len(dms)
    assert nd_max >= _grouped_need(orc, nsub, fc, nchan, dms.max(), chirp)
    assert nout == (((nsamp - nbin) // (nbin - nd_max * nchan)) + 1) * ((m - nd_max) // nint)

    def covers(nd_g):
        off = (nd_max - nd_g) * nchan // 2
        sv = nbin - nd_g * nchan
        return nsamp - off >= nbin and ((nsamp - off - nbin) // sv + 1) * ((m - nd_g) // nint) >= nout

    for first, count, nd_g, off, nbin_g in layout:
        assert nbin_g == nbin
        need = _grouped_need(orc, nsub, fc, nchan, np.abs(dms[first:first + count]).max(), chirp)
        assert nd_g % 2 == 0 and (m - nd_g) % nint == 0 and nd_g <= nd_max
        assert nd_g >= need and covers(nd_g)
        assert off == (nd_max - nd_g) * nchan // 2
        cand = nd_g - 2
        while cand >= 0 and (cand % 2 or (m - cand) % nint):
            cand -= 2
        assert cand < 0 or cand < need or not covers(cand)
    assert layout[-1][2] == nd_max and layout[-1][3] == 0
    assert layout[0][2] < nd_max   # the grouping does save overlap here


def test_grouped_filterbank_keeps_the_ungrouped_time_axis(orc):
    # Noise in: one group is the ungrouped filterbank exactly; with four groups the
    # group of the largest DM is the ungrouped rows exactly, and the other rows differ
    # from them only by the wrap-around leakage of the shorter overlaps (about 1 %
    # rms), while one output sample of misalignment would differ by about 60 %.
    nsub, fc, nchan, nint, nbin = 2, 60.0, 8, 2, 1 << 13
    nsamp = 6 * nbin + 1000
    dms = np.linspace(0.0, 4.2, 8)
    x = np.random.default_rng(5).standard_normal((nsub, nsamp, 4)).astype(np.float32)
    nd = orc.overlap(nsub, fc, BW, dms, nchan, nint, nbin, 1)
    plain = orc.filterbank(x, fc, BW, dms, nchan, nint, nbin, nd, chirp=1)
    assert np.array_equal(orc.filterbank_grouped(x, fc, BW, dms, nchan, nint, nbin, 1, chirp=1), plain)
    g = orc.filterbank_grouped(x, fc, BW, dms, nchan, nint, nbin, 4, chirp=1)
    assert g.shape == plain.shape
    assert np.array_equal(g[6:], plain[6:])
    for i in range(6):
        rel = np.sqrt(np.mean((g[i] - plain[i]) ** 2) / np.mean(plain[i] ** 2))
        assert rel < 0.03, (i, rel)
        shifted = np.sqrt(np.mean((g[i][:, 1:] - plain[i][:, :-1]) ** 2) / np.mean(plain[i] ** 2))
        assert shifted > 0.3, (i, shifted)


@pytest.mark.parametrize("dm_true", [5.0, 10.0])
def test_grouped_impulse_at_the_closed_form_time(orc, dm_true):
    # A physical impulse dispersed at dm_true (a DM in a group with a shorter overlap
    # and an input offset): at its DM row, channel c peaks at the closed-form time of
    # the ungrouped axis, t0 / n_c + D DM (nu_c^-2 - nu_s^-2) r / n_c - nd_max / 2, with
    # >= 0.8 of the row's energy in the two nearest samples.
    fc, nchan, nbin = 135.0, 8, 1 << 14
    nsamp, t0, r = 1 << 15, 20000, BW * 1e6
    x = _physical_impulse(nsamp, fc, dm_true, t0)
    dms = [0.0, 5.0, 10.0, 15.0, 40.0, 45.0]
    layout, nd_max, _ = orc.grouped_layout(1, nsamp, fc, BW, dms, nchan, 1, nbin, 3)
    gi = [g for g, (first, count, _, _, _) in enumerate(layout) if first <= dms.index(dm_true) < first + count][0]
    assert layout[gi][3] > 0   # the DM's group starts its segments later
    fb = orc.filterbank_grouped(x, fc, BW, dms, nchan, 1, nbin, 3)
    for c in range(nchan):
        nuc = fc - BW / 2 + (c + 0.5) * BW / nchan
        t_exp = t0 / nchan + D * dm_true * (1 / nuc ** 2 - 1 / fc ** 2) * r / nchan - nd_max / 2
        row = fb[dms.index(dm_true), c]
        i0 = int(np.floor(t_exp))
        assert abs(np.argmax(row) - t_exp) <= 1.0, (c, np.argmax(row), t_exp)
        assert (row[i0] + row[i0 + 1]) / np.sum(row) >= 0.8


LENGTHS = [512, 1024, 2048, 4096, 8192]


@pytest.mark.parametrize("chirp", [0, 1])
def test_grouped_lengths_cover_and_save_work(orc, chirp):
    # With FFT lengths per group (Sec. 5: digifil picks the FFT size per DM): every group's
    # length is one offered, its overlap satisfies the rule's conditions at that length,
    # holds the group's Eq. 2 sweep, stays within the whole list's and lets its segments
    # cover the ungrouped length from the same offset (which does not depend on the
    # length); the group of the largest |DM| keeps nd_max and no offset; some group does
    # take another length; and the total nominal FFT work, sum over DMs of
    # M log2(M) / (M - nd) (10 N log2 M / S per unit, over 10 n_c), is no more than that of
    # the same grouping at the plan's length.
    nsub, fc, nchan, nint, nbin = 2, 60.0, 8, 2, 1 << 14
    nsamp = 6 * nbin + 1000
    dms = np.linspace(0.0, 4.2, 8) if chirp else np.linspace(0.0, 30.0, 8)
    layout, nd_max, nout = orc.grouped_layout(nsub, nsamp, fc, BW, dms, nchan, nint, nbin, 4, chirp, lengths=LENGTHS)
    fixed, _, _ = orc.grouped_layout(nsub, nsamp, fc, BW, dms, nchan, nint, nbin, 4, chirp)
    m_plan = nbin // nchan
    work = work_fixed = 0.0
    for (first, count, nd_g, off, nbin_g), fx in zip(layout, fixed):
        m = nbin_g // nchan
        assert m in LENGTHS and nbin_g == m * nchan
        need = _grouped_need(orc, nsub, fc, nchan, np.abs(dms[first:first + count]).max(), chirp)
        assert nd_g % 2 == 0 and (m - nd_g) % nint == 0 and need <= nd_g <= nd_max
        assert off == (nd_max - nd_g) * nchan // 2
        sv = nbin_g - nd_g * nchan
        assert nsamp - off >= nbin_g and ((nsamp - off - nbin_g) // sv + 1) * ((m - nd_g) // nint) >= nout
        work += count * m * np.log2(m) / (m - nd_g)
        work_fixed += count * m_plan * np.log2(m_plan) / (m_plan - fx[2])
    assert layout[-1][2] == nd_max and layout[-1][3] == 0
    assert any(g[4] != nbin for g in layout)
    assert work <= work_fixed * (1 + 1e-12)


def test_grouped_lengths_keep_the_time_axis(orc):
    # Noise in, groups of the subband-wide chirp with their own FFT lengths: every row stays
    # within the wrap-around leakage of the ungrouped rows (about 1 % rms; rows of a group at
    # the plan's length and overlap, exactly), while one output sample of misalignment would
    # differ by about 60 %.
    nsub, fc, nchan, nint, nbin = 2, 60.0, 8, 2, 1 << 13
    nsamp = 6 * nbin + 1000
    dms = np.linspace(0.0, 4.2, 8)
    x = np.random.default_rng(5).standard_normal((nsub, nsamp, 4)).astype(np.float32)
    nd = orc.overlap(nsub, fc, BW, dms, nchan, nint, nbin, 1)
    plain = orc.filterbank(x, fc, BW, dms, nchan, nint, nbin, nd, chirp=1)
    layout, _, _ = orc.grouped_layout(nsub, nsamp, fc, BW, dms, nchan, nint, nbin, 4, 1, lengths=LENGTHS)
    assert any(g[4] != nbin for g in layout)
    g = orc.filterbank_grouped(x, fc, BW, dms, nchan, nint, nbin, 4, chirp=1, lengths=LENGTHS)
    assert g.shape == plain.shape
    for first, count, nd_g, off, nbin_g in layout:
        for i in range(first, first + count):
            if nd_g == nd and nbin_g == nbin:
                assert np.array_equal(g[i], plain[i])
                continue
            rel = np.sqrt(np.mean((g[i] - plain[i]) ** 2) / np.mean(plain[i] ** 2))
            assert rel < 0.03, (i, rel)
            shifted = np.sqrt(np.mean((g[i][:, 1:] - plain[i][:, :-1]) ** 2) / np.mean(plain[i] ** 2))
            assert shifted > 0.3, (i, shifted)


@pytest.mark.parametrize("dm_true", [5.0, 10.0])
def test_grouped_lengths_impulse_at_the_closed_form_time(orc, dm_true):
    # A physical impulse dispersed at dm_true, in a group whose FFT length (and overlap and
    # offset) differ from the plan's: at its DM row, channel c peaks at the closed-form time of
    # the ungrouped axis, t0 / n_c + D DM (nu_c^-2 - nu_s^-2) r / n_c - nd_max / 2, with
    # >= 0.8 of the row's energy in the two nearest samples.
    fc, nchan, nbin = 135.0, 8, 1 << 14
    nsamp, t0, r = 1 << 15, 20000, BW * 1e6
    x = _physical_impulse(nsamp, fc, dm_true, t0)
    dms = [0.0, 5.0, 10.0, 15.0, 40.0, 45.0]
    layout, nd_max, _ = orc.grouped_layout(1, nsamp, fc, BW, dms, nchan, 1, nbin, 3, lengths=LENGTHS)
    gi = [g for g, (first, count, _, _, _) in enumerate(layout) if first <= dms.index(dm_true) < first + count][0]
    assert layout[gi][4] != nbin and layout[gi][3] > 0
    fb = orc.filterbank_grouped(x, fc, BW, dms, nchan, 1, nbin, 3, lengths=LENGTHS)
    for c in range(nchan):
        nuc = fc - BW / 2 + (c + 0.5) * BW / nchan
        t_exp = t0 / nchan + D * dm_true * (1 / nuc ** 2 - 1 / fc ** 2) * r / nchan - nd_max / 2
        row = fb[dms.index(dm_true), c]
        i0 = int(np.floor(t_exp))
        assert abs(np.argmax(row) - t_exp) <= 1.0, (c, np.argmax(row), t_exp)
        assert (row[i0] + row[i0 + 1]) / np.sum(row) >= 0.8


def test_code_step_given_statistics(orc):
    # the code step alone (oracle.codes), with statistics given by hand: gain 16 / sigma
    # in FP32, rint rounding half to even, clipping to 0..255, flagged rows at 128, rows
    # written in decreasing frequency
    fb = np.array([[[14.0, 10.125, 10.375, 6.0, 100.0, -100.0],
                    [5.0, 5.0, 5.0, 5.0, 5.0, 5.0]]], dtype=np.float32)
    stats = np.array([[[10.0, 4.0], [5.0, 0.0]]], dtype=np.float32)
    c = orc.codes(fb, stats)
    # row 0: (I - 10) * 4 + 128 = 144, 128.5 -> 128, 129.5 -> 130, 112, 488 -> 255, -312 -> 0
    assert list(c[0, :, 1]) == [144, 128, 130, 112, 255, 0]
    assert list(c[0, :, 0]) == [128] * 6          # sigma 0: gain 0
    flagged = orc.codes(fb, stats, np.array([[1, 0]], dtype=np.uint8))
    assert list(flagged[0, :, 1]) == [128] * 6
    # the redigitisation is the code step applied with its own statistics rounded to FP32
    g = np.random.default_rng(14)
    fb = g.gamma(6.0, 2.0, (2, 5, 300)).astype(np.float32)
    codes, st = orc.redigitise(fb)
    assert np.array_equal(codes, orc.codes(fb, st.astype(np.float32)))
