"""FP64 CPU oracle for the coherent-dedispersion filterbank (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  The GPU library never uses it.  The arithmetic lives in
``cdmt_oracle.c`` (plain C, double precision, its own radix-2 FFT); this module
compiles it with gcc on first use and marshals numpy arrays through ctypes.

Every function states the passage of Bassa, Pleunis & Hessels (2016) that it
follows; the C file's header lists the steps and the readings taken where the
paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdmt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

D_CONST = 4.148808e3  # MHz^2 pc^-1 cm^3 s (dispersion constant reading)


def build(force: bool = False) -> str:
    """Compile the oracle to ``liboracle.so`` (gcc -O2, no fast-math, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            i64 = ctypes.c_int64
            lib.orc_sweep.restype = ctypes.c_double
            lib.orc_sweep.argtypes = [ctypes.c_double] * 3
            lib.orc_subband_centre.restype = ctypes.c_double
            lib.orc_subband_centre.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
            lib.orc_channel_centre.restype = ctypes.c_double
            lib.orc_channel_centre.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
            lib.orc_overlap.restype = i64
            lib.orc_overlap.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, i64]
            lib.orc_overlap_m.restype = i64
            lib.orc_overlap_m.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, i64, ctypes.c_int]
            lib.orc_fft.restype = None
            lib.orc_fft.argtypes = [dp, i64, ctypes.c_int]
            lib.orc_dft.restype = None
            lib.orc_dft.argtypes = [dp, dp, i64, ctypes.c_int]
            lib.orc_segment_channels.restype = None
            lib.orc_segment_channels.argtypes = [dp, i64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double, dp]
            lib.orc_segment_channels_m.restype = None
            lib.orc_segment_channels_m.argtypes = [dp, i64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                   ctypes.c_double, dp, ctypes.c_int]
            lib.orc_grid.restype = ctypes.c_int
            lib.orc_grid.argtypes = [i64, i64, ctypes.c_int, i64, ctypes.c_int,
                                     ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
            lib.orc_filterbank.restype = ctypes.c_int
            lib.orc_filterbank.argtypes = [fp, ctypes.c_int, i64, ctypes.c_double, ctypes.c_double, dp,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, i64, dp, ctypes.c_int]
            lib.orc_filterbank_m.restype = ctypes.c_int
            lib.orc_filterbank_m.argtypes = lib.orc_filterbank.argtypes + [ctypes.c_int]
            lib.orc_tiles.restype = ctypes.c_int
            lib.orc_tiles.argtypes = [fp, ctypes.c_int, i64, ctypes.c_double, ctypes.c_double, dp,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, i64, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64),
                                      ctypes.POINTER(ctypes.c_int), dp, ctypes.c_int]
            lib.orc_tiles_m.restype = ctypes.c_int
            lib.orc_tiles_m.argtypes = lib.orc_tiles.argtypes + [ctypes.c_int]
            lib.orc_max_threads.restype = ctypes.c_int
            lib.orc_incoherent.restype = i64
            lib.orc_incoherent.argtypes = [fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_redigitise.argtypes = [fp, ctypes.c_int, ctypes.c_int, i64, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_redigitise.restype = None
            lib.orc_codes.argtypes = [fp, ctypes.c_int, ctypes.c_int, i64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]
            lib.orc_codes.restype = None
            lib.orc_sk_sigma.argtypes = [i64, ctypes.c_int]
            lib.orc_sk_sigma.restype = ctypes.c_double
            lib.orc_spectral_kurtosis.argtypes = [fp, ctypes.c_int, ctypes.c_int, i64, ctypes.c_int, ctypes.c_double,
                                                  ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_spectral_kurtosis.restype = None
            lib.orc_redigitise_sk.argtypes = [fp, ctypes.c_int, ctypes.c_int, i64, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_redigitise_sk.restype = None
            lib.orc_max_threads.argtypes = []
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def sweep(nu_min: float, nu_max: float, dm: float) -> float:
    """Dispersion sweep t_d (s) across [nu_min, nu_max] MHz (Eq. 2)."""
    return _load().orc_sweep(nu_min, nu_max, dm)


def subband_centre(nsub: int, f_centre: float, bw: float, s: int) -> float:
    """Centre (MHz) of subband s of a contiguous band centred on f_centre (Sec. 3 input model)."""
    return _load().orc_subband_centre(nsub, f_centre, bw, s)


def channel_centre(nu_s: float, bw: float, nchan: int, c: int) -> float:
    """Centre (MHz) of channel c of a subband centred on nu_s (Sec. 2, nu_0 of a channel)."""
    return _load().orc_channel_centre(nu_s, bw, nchan, c)


def overlap(nsub, f_centre, bw, dm_list, nchan, nint, nbin, chirp: int = 0) -> int:
    """Overlap nd of Sec. 2 (nd = r t_d / n_c, t_d of Eq. 2 for the lowest channel;
    chirp = 1: for the lowest subband, whose single transfer function spans it)."""
    dm = np.ascontiguousarray(dm_list, dtype=np.float64)
    return int(_load().orc_overlap_m(nsub, f_centre, bw, _dp(dm), len(dm), nchan, nint, nbin, chirp))


def grid(nsamp, nbin, nchan, nd, nint):
    """(S, nseg, nout) of the overlap-save grid (Sec. 2, Fig. 2; Sec. 3 block loop)."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = _load().orc_grid(nsamp, nbin, nchan, nd, nint, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if rc:
        raise ValueError("invalid overlap-save grid")
    return a.value, b.value, c.value


def fft(x, sign: int) -> np.ndarray:
    """Unnormalised radix-2 FFT with kernel exp(sign 2 pi i nk/n) (the oracle's own)."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    _load().orc_fft(_dp(a.view(np.float64)), len(a), sign)
    return a


def dft(x, sign: int) -> np.ndarray:
    """Naive O(n^2) DFT with kernel exp(sign 2 pi i nk/n)."""
    a = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.empty_like(a)
    _load().orc_dft(_dp(a.view(np.float64)), _dp(y.view(np.float64)), len(a), sign)
    return y


def segment_channels(x, nchan: int, nu_s: float, bw: float, dm: float, chirp: int = 0) -> np.ndarray:
    """Channelised, dedispersed complex series [nchan][M] of one polarisation of
    one segment, before the overlap is discarded (Sec. 2 steps 3-5 of Fig. 2)."""
    a = np.ascontiguousarray(x, dtype=np.complex128)
    n = len(a)
    y = np.empty((nchan, n // nchan), dtype=np.complex128)
    _load().orc_segment_channels_m(_dp(a.view(np.float64)), n, nchan, nu_s, bw, dm, _dp(y.view(np.float64)), chirp)
    return y


def filterbank(x, f_centre, bw, dm_list, nchan, nint, nbin, nd, nthreads: int = 0, chirp: int = 0) -> np.ndarray:
    """Whole DM x channel x time filterbank (Algorithm 1 up to detection, plus
    integration over nint).  x: float32 [nsub][nsamp][4]; returns float64
    [ndm][nsub*nchan][nout].  chirp: 0 per-channel transfer functions, 1 one per subband."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    nsub, nsamp = x.shape[0], x.shape[1]
    dm = np.ascontiguousarray(dm_list, dtype=np.float64)
    _, _, nout = grid(nsamp, nbin, nchan, nd, nint)
    out = np.zeros((len(dm), nsub * nchan, nout), dtype=np.float64)
    rc = _load().orc_filterbank_m(_fp(x), nsub, nsamp, f_centre, bw, _dp(dm), len(dm), nchan, nint,
                                  nbin, nd, _dp(out), nthreads, chirp)
    if rc:
        raise ValueError("oracle rejected the arguments")
    return out


def dm_groups(ndm: int, groups: int) -> list[tuple[int, int]]:
    """Contiguous DM-index ranges (first, count) of `groups` near-equal parts of
    the list: part g holds indices [g ndm / groups, (g + 1) ndm / groups)."""
    if not 1 <= groups <= ndm:
        raise ValueError("need 1 <= groups <= ndm")
    return [(g * ndm // groups, (g + 1) * ndm // groups - g * ndm // groups) for g in range(groups)]


def grouped_layout(nsub, nsamp, f_centre, bw, dm_list, nchan, nint, nbin, groups, chirp: int = 0, nd: int = -1,
                   lengths=None):
    """Overlap per DM group (digifil's per-DM overlap, Sec. 5, taken per group of
    trials).  nd_max is Sec. 2's overlap for the whole list (or `nd`), and the
    grouped filterbank keeps its time axis and length nout: a group whose
    overlap is nd_g starts its overlap-save segments off_g = (nd_max - nd_g) n_c / 2
    input samples later, so that its first kept sample (nd_g / 2 channel samples
    into segment 0) is channel sample nd_max / 2 of the input, as with nd_max.
    nd_g is the smallest overlap that is at least Sec. 2's overlap for the
    group's own largest |DM|, satisfies the rule's parity and nint conditions and
    whose segments still cover nout (nd_max always does).

    lengths: channel lengths M the groups may take besides nbin / nchan (Sec. 5:
    digifil also picks the FFT size for the DM at hand).  A group then takes the M
    whose overlap, found as above with N = n_c M, stays within nd_max and lets one
    segment fit the input from off_g, and whose nominal FFT work per unit
    10 N log2(M) / S_g = 10 M log2(M) / (M - nd_g) is least; nbin / nchan on a tie.
    The channel sample rate, hence the time axis and off_g, do not depend on M.
    Returns ([(first, count, nd_g, off_g, nbin_g)], nd_max, nout)."""
    dm = np.ascontiguousarray(dm_list, dtype=np.float64)
    nd_max = nd if nd >= 0 else overlap(nsub, f_centre, bw, dm, nchan, nint, nbin, chirp)
    if nd_max < 0:
        raise ValueError("no overlap < M")
    nout = grid(nsamp, nbin, nchan, nd_max, nint)[2]
    m_plan = nbin // nchan

    def segments_cover(n, nd_g):
        off = (nd_max - nd_g) * nchan // 2
        return nsamp - off >= n and grid(nsamp - off, n, nchan, nd_g, nint)[2] >= nout

    def group_overlap(dms, m):
        # the group's overlap at channel length m, or None where it would exceed nd_max
        n = m * nchan
        nd_g = overlap(nsub, f_centre, bw, dms, nchan, nint, n, chirp)
        if nd_g < 0 or nd_g > nd_max:
            if m != m_plan:
                return None
            nd_g = nd_max
        while not segments_cover(n, nd_g):
            nd_g += 2
            while (m - nd_g) % nint:
                nd_g += 2
            if nd_g > nd_max:
                return None
        return nd_g

    out = []
    for first, count in dm_groups(len(dm), groups):
        dms = dm[first:first + count]
        m_g, nd_g = m_plan, group_overlap(dms, m_plan)
        work = m_g * np.log2(m_g) / (m_g - nd_g)
        for m in (lengths or ()):
            if m == m_plan:
                continue
            v = group_overlap(dms, m)
            if v is None:
                continue
            w = m * np.log2(m) / (m - v)
            if w < work * (1 - 1e-12):
                m_g, nd_g, work = m, v, w
        out.append((first, count, nd_g, (nd_max - nd_g) * nchan // 2, m_g * nchan))
    return out, nd_max, nout


def filterbank_grouped(x, f_centre, bw, dm_list, nchan, nint, nbin, groups, nthreads: int = 0, chirp: int = 0,
                       nd: int = -1, lengths=None) -> np.ndarray:
    """The filterbank of :func:`filterbank` with each DM group's own overlap (and,
    with `lengths`, its own FFT length) (:func:`grouped_layout`): group g's rows are
    the filterbank of the input from sample off_g on, with overlap nd_g and N_g,
    cut to the ungrouped length nout.  float64 [ndm][nsub*nchan][nout], on the
    ungrouped time axis."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    nsub, nsamp = x.shape[0], x.shape[1]
    dm = np.ascontiguousarray(dm_list, dtype=np.float64)
    layout, _, nout = grouped_layout(nsub, nsamp, f_centre, bw, dm, nchan, nint, nbin, groups, chirp, nd, lengths)
    out = np.empty((len(dm), nsub * nchan, nout), dtype=np.float64)
    for first, count, nd_g, off, nbin_g in layout:
        fb = filterbank(x[:, off:], f_centre, bw, dm[first:first + count], nchan, nint, nbin_g, nd_g, nthreads, chirp)
        out[first:first + count] = fb[:, :, :nout]
    return out


def tiles(x, f_centre, bw, dm_list, nchan, nint, nbin, nd, sub, seg, dmi, nthreads: int = 0,
          chirp: int = 0) -> np.ndarray:
    """Filterbank samples of the listed (subband, segment, DM index) tiles:
    float64 [ntile][nchan][(M - nd)/nint].  Equal to the matching slice of
    :func:`filterbank` (each segment is independent given its own input)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    nsub, nsamp = x.shape[0], x.shape[1]
    dm = np.ascontiguousarray(dm_list, dtype=np.float64)
    sub = np.ascontiguousarray(sub, dtype=np.int32)
    seg = np.ascontiguousarray(seg, dtype=np.int64)
    dmi = np.ascontiguousarray(dmi, dtype=np.int32)
    m = nbin // nchan
    out = np.zeros((len(sub), nchan, (m - nd) // nint), dtype=np.float64)
    rc = _load().orc_tiles_m(_fp(x), nsub, nsamp, f_centre, bw, _dp(dm), len(dm), nchan, nint, nbin, nd,
                             len(sub), sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                             seg.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             dmi.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(out), nthreads, chirp)
    if rc:
        raise ValueError("oracle rejected the tile list")
    return out


def redigitise(fb) -> tuple[np.ndarray, np.ndarray]:
    """8-bit redigitisation of a float filterbank [ndm][rows][nt] (Sec. 3):
    returns (codes uint8 [ndm][nt][rows] in decreasing frequency, stats float64
    [ndm][rows][2] = (mean, standard deviation))."""
    fb = np.ascontiguousarray(fb, dtype=np.float32)
    ndm, rows, nt = fb.shape
    out = np.empty((ndm, nt, rows), dtype=np.uint8)
    st = np.empty((ndm, rows, 2), dtype=np.float64)
    _load().orc_redigitise(_fp(fb), ndm, rows, nt, out.ctypes.data, st.ctypes.data)
    return out, st


def codes(fb, stats, flags=None) -> np.ndarray:
    """The code step of the redigitisation (Sec. 3) given each row's statistics:
    stats [ndm][rows][2] = (mean, standard deviation) taken as FP32, flags
    [ndm][rows] (optional) marks rows coded 128.  Returns uint8 [ndm][nt][rows]
    in decreasing frequency, as :func:`redigitise`."""
    fb = np.ascontiguousarray(fb, dtype=np.float32)
    ndm, rows, nt = fb.shape
    st = np.ascontiguousarray(stats, dtype=np.float32).reshape(ndm, rows, 2)
    fl = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8).reshape(ndm, rows)
    out = np.empty((ndm, nt, rows), dtype=np.uint8)
    _load().orc_codes(_fp(fb), ndm, rows, nt, st.ctypes.data, None if fl is None else fl.ctypes.data, out.ctypes.data)
    return out


LEVELS = 16.0


def sk_sigma(n: int, k: int) -> float:
    """Large-n standard deviation of the spectral-kurtosis estimator for n samples
    that are each a sum of k squared magnitudes."""
    return _load().orc_sk_sigma(n, k)


def spectral_kurtosis(fb, k: int, nsigma: float = 3.0) -> tuple[np.ndarray, np.ndarray]:
    """Generalised spectral kurtosis of every row of fb [ndm][rows][nt] whose
    samples each sum k squared magnitudes (k = 2 nint), and the RFI flags
    |SK - 1| > nsigma * sk_sigma(nt, k) (Sec. 6): (sk float64 [ndm][rows],
    flags uint8 [ndm][rows])."""
    fb = np.ascontiguousarray(fb, dtype=np.float32)
    ndm, rows, nt = fb.shape
    sk = np.empty((ndm, rows), dtype=np.float64)
    fl = np.empty((ndm, rows), dtype=np.uint8)
    _load().orc_spectral_kurtosis(_fp(fb), ndm, rows, nt, k, nsigma, sk.ctypes.data, fl.ctypes.data)
    return sk, fl


def redigitise_sk(fb, k: int, nsigma: float) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """redigitise() with spectral-kurtosis flagging: flagged rows are coded 128.
    Returns (codes, stats, flags)."""
    fb = np.ascontiguousarray(fb, dtype=np.float32)
    ndm, rows, nt = fb.shape
    out = np.empty((ndm, nt, rows), dtype=np.uint8)
    st = np.empty((ndm, rows, 2), dtype=np.float64)
    fl = np.empty((ndm, rows), dtype=np.uint8)
    _load().orc_redigitise_sk(_fp(fb), ndm, rows, nt, k, nsigma, out.ctypes.data, st.ctypes.data, fl.ctypes.data)
    return out, st, fl


def incoherent(fb, nsub, nchan, f_centre, bw, nint, dm_c, ddm_lo, ddm_step, nk, chirp: int = 0):
    """Incoherent dedispersion of coherent filterbanks fb [ndm][nsub*nchan][nt]
    over nk fine trials dm_c[i] + ddm_lo + k ddm_step (Sec. 4).  Returns
    (out float64 [ndm][nk][nt_out], delays int32 [ndm][nk][rows] relative to the
    smallest)."""
    fb = np.ascontiguousarray(fb, dtype=np.float32)
    ndm, rows, nt = fb.shape
    dm = np.ascontiguousarray(dm_c, dtype=np.float64)
    delays = np.empty((ndm, nk, rows), dtype=np.int32)
    lib = _load()
    nt_out = lib.orc_incoherent(_fp(fb), ndm, nsub, nchan, nt, f_centre, bw, nint, chirp, _dp(dm), ddm_lo,
                                ddm_step, nk, None, delays.ctypes.data)
    if nt_out < 1:
        raise ValueError("no output sample survives the shifts")
    out = np.empty((ndm, nk, nt_out), dtype=np.float64)
    lib.orc_incoherent(_fp(fb), ndm, nsub, nchan, nt, f_centre, bw, nint, chirp, _dp(dm), ddm_lo, ddm_step, nk,
                       out.ctypes.data, None)
    return out, delays   # code steps per standard deviation (128 = the mean)


def max_threads() -> int:
    """OpenMP threads the oracle uses by default."""
    return int(_load().orc_max_threads())
