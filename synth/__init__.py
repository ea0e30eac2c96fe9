"""Seeded synthetic voltages shaped like LOFAR beam-formed subbands.

This module generates INPUTS only.  It serves the tests, the benchmark and the
FP64 oracle alike, and holds none of the dedispersion method: it draws complex
Gaussian noise from a counter-based generator (numpy's Philox keyed by
``(seed, beam, subband, pol)``), and it simulates the interstellar medium on
injected pulses by multiplying a pulse window's spectrum by the ISM transfer
function of Eq. 1 evaluated across the WHOLE subband (nu_0 = subband centre),
which is the physical forward model, not the per-channel inverse filter that
the method applies.

Layout of every array it returns: float32 ``[nsub][nsamp][4]`` with the four
floats of a time sample being (X re, X im, Y re, Y im): complex, Nyquist
sampled, dual polarisation subbands (Sec. 3 input model; Sec. 4 data).

Noise is "unit variance" in the complex sense: E|x|^2 = sigma2 per
polarisation, real and imaginary parts each N(0, sigma2/2).
"""
from __future__ import annotations

import dataclasses
from concurrent.futures import ThreadPoolExecutor

import numpy as np

D_MHZ = 4.148808e3  # MHz^2 pc^-1 cm^3 s, dispersion constant used for the simulation


@dataclasses.dataclass(frozen=True)
class Pulse:
    """A broadband boxcar of complex Gaussian noise (std ``amp`` * sigma per
    polarisation) lasting ``width_s`` seconds, arriving at ``t0_s`` at the
    reference frequency (top of the band), dispersed at ``dm``."""
    t0_s: float
    dm: float
    width_s: float
    amp: float = 0.5


def subband_centres(nsub: int, f_centre: float, bw: float) -> np.ndarray:
    """Centres (MHz) of nsub contiguous subbands of width bw around f_centre."""
    return f_centre + (np.arange(nsub) - 0.5 * (nsub - 1)) * bw


def _rng(seed: int, beam: int, sub: int, pol: int, stream: int = 0) -> np.random.Generator:
    key = np.array([(seed << 24) | (beam << 8) | stream, (sub << 2) | pol], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def noise(seed: int, nsub: int, nsamp: int, sigma2: float = 1.0, beam: int = 0,
          threads: int = 8, sub0: int = 0) -> np.ndarray:
    """Complex Gaussian noise, float32 [nsub][nsamp][4]: subbands sub0 .. sub0 + nsub - 1
    of a band (each subband's stream is keyed by its own index, so a slice of the band
    equals the same rows of the whole band)."""
    out = np.empty((nsub, nsamp, 4), dtype=np.float32)
    sc = np.float32(np.sqrt(sigma2 / 2.0))

    def one(s):
        for p in range(2):
            g = _rng(seed, beam, s + sub0, p)
            v = g.standard_normal(2 * nsamp, dtype=np.float32)
            v *= sc
            out[s, :, 2 * p] = v[0::2]
            out[s, :, 2 * p + 1] = v[1::2]

    if threads > 1 and nsub > 1:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(one, range(nsub)))
    else:
        for s in range(nsub):
            one(s)
    return out


def ism_sweep(nu_lo: float, nu_hi: float, dm: float) -> float:
    """Delay (s) of nu_lo relative to nu_hi for a cold plasma."""
    return D_MHZ * dm * (1.0 / nu_lo ** 2 - 1.0 / nu_hi ** 2)


def add_pulses(x: np.ndarray, pulses, f_centre: float, bw: float, seed: int,
               sigma2: float = 1.0, beam: int = 0, sub0: int = 0, nsub_band: int = 0) -> None:
    """Add dispersed pulses in place to float32 [nsub][nsamp][4] voltages.

    For each subband the pulse is drawn in a window long enough to hold its
    width plus the subband's own dispersion sweep, the window's spectrum is
    multiplied by the subband-wide transfer function (Eq. 1 with nu_0 the
    subband centre, i.e. exp(+2 pi i 1e6 D DM nu^2 / (nu_0^2 (nu_0 + nu))) for the
    numpy forward-FFT convention), and the result is added at the subband's
    arrival time t0 + D DM (nu_0^-2 - nu_ref^-2), nu_ref the top of the band.
    x may hold subbands sub0 .. sub0 + len(x) - 1 of a band of nsub_band subbands
    centred on f_centre (0: x is the whole band).
    """
    nsub, nsamp = x.shape[0], x.shape[1]
    band = nsub_band if nsub_band > 0 else nsub
    r = bw * 1e6
    nus = subband_centres(band, f_centre, bw)[sub0:sub0 + nsub]
    nu_ref = f_centre + 0.5 * band * bw
    for ip, pu in enumerate(pulses):
        for s in range(nsub):
            nu0 = nus[s]
            td = ism_sweep(nu0 - 0.5 * bw, nu0 + 0.5 * bw, pu.dm)
            wn = max(1, int(round(pu.width_s * r)))
            need = wn + int(np.ceil(td * r)) + 256
            L = 1 << int(np.ceil(np.log2(max(2 * need, 1024))))
            t_arr = pu.t0_s + ism_sweep(nu0, nu_ref, pu.dm)
            centre = int(round(t_arr * r))
            start = centre - L // 2
            f = np.fft.fftfreq(L, d=1.0 / r) / 1e6  # MHz offsets from nu0
            h = np.exp(2j * np.pi * 1e6 * D_MHZ * pu.dm * f ** 2 / (nu0 ** 2 * (nu0 + f)))
            for p in range(2):
                g = _rng(seed, beam, s + sub0, p, stream=16 + ip)
                w = np.zeros(L, dtype=np.complex128)
                b0 = L // 2 - wn // 2
                amp = pu.amp * np.sqrt(sigma2 / 2.0)
                w[b0:b0 + wn] = amp * (g.standard_normal(wn) + 1j * g.standard_normal(wn))
                d = np.fft.ifft(np.fft.fft(w) * h)
                lo, hi = max(start, 0), min(start + L, nsamp)
                if lo >= hi:
                    continue
                seg = d[lo - start:hi - start]
                x[s, lo:hi, 2 * p] += seg.real.astype(np.float32)
                x[s, lo:hi, 2 * p + 1] += seg.imag.astype(np.float32)


def tone(nsamp: int, offset_mhz: float, bw: float, amp_x: complex, amp_y: complex) -> np.ndarray:
    """One subband holding a pure complex tone at ``offset_mhz`` from the subband
    centre, float32 [1][nsamp][4]."""
    n = np.arange(nsamp)
    ph = np.exp(2j * np.pi * offset_mhz * n / bw)
    out = np.zeros((1, nsamp, 4), dtype=np.float32)
    out[0, :, 0], out[0, :, 1] = (amp_x * ph).real, (amp_x * ph).imag
    out[0, :, 2], out[0, :, 3] = (amp_y * ph).real, (amp_y * ph).imag
    return out


# ---------------------------------------------------------------------------
# Named workloads.  Shapes follow the LOFAR survey of Sec. 4 (195.3125 kHz
# subbands near 135 MHz, 8-16 channels, DMs up to ~80); the data themselves
# are synthetic.


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    nsub: int
    nsamp: int
    f_centre: float
    bw: float
    dms: tuple
    nchan: int
    nint: int
    nbin: int
    seed: int
    pulses: tuple = ()
    nd: int = -1        # overlap n_d fixed by the setup (-1: the planner's rule)

    def voltages(self, threads: int = 8, beam: int = 0, sub=None) -> np.ndarray:
        """The workload's voltages, or subbands sub = (lo, hi) of them (equal to those rows
        of the whole band)."""
        lo, hi = (0, self.nsub) if sub is None else sub
        x = noise(self.seed, hi - lo, self.nsamp, beam=beam, threads=threads, sub0=lo)
        if self.pulses:
            add_pulses(x, self.pulses, self.f_centre, self.bw, self.seed, beam=beam, sub0=lo, nsub_band=self.nsub)
        return x


def tiny() -> Workload:
    """1 subband at 135 MHz, 2^17 samples, one 1 ms pulse at DM 10, N = 2^14,
    DMs {0, 5, 10, 15}, 8 channels, integrate 4."""
    return Workload("tiny-1sub-2^17", 1, 1 << 17, 135.0, 0.1953125, (0.0, 5.0, 10.0, 15.0), 8, 4,
                    1 << 14, 1, (Pulse(0.30, 10.0, 1e-3, 0.5),))


def paper(nsamp: int = 1 << 22) -> Workload:
    """The paper's own application setup (Sec. 4): 10 contiguous subbands
    114.93-116.88 MHz, N = 2^16 with n_c = 8 channels (M = 8192 bins) and an
    overlap of n_d = 2048, 80 DMs 0.5..79.5 step 1, no averaging (nint 1); 2^22
    samples (21.5 s) instead of the paper's 20 minutes, 3 pulses at DM ~ U(5, 75),
    widths U(0.2, 2) ms."""
    g = np.random.default_rng(103)
    T = nsamp / 195312.5
    pulses = tuple(Pulse(float(g.uniform(1.0, max(1.5, T - 3.0))), float(g.uniform(5, 75)),
                         float(g.uniform(0.2e-3, 2e-3)), 0.5) for _ in range(3))
    return Workload(f"paper-10sub-2^{int(np.log2(nsamp))}-M8192", 10, nsamp, 114.93 + 5 * 0.1953125, 0.1953125,
                    tuple(0.5 + i for i in range(80)), 8, 1, 1 << 16, 3, pulses, 2048)


def lofar64(nsamp: int = 1 << 22, nsub: int = 64, nchan: int = 16) -> Workload:
    """64 contiguous subbands 128.75-141.25 MHz, 2^22 samples, 5 pulses at
    DM ~ U(5, 60), widths U(0.2, 5) ms; N = 2^16, 128 DMs 0..63.5 step 0.5,
    16 channels, integrate 8.  ``nsub`` < 64 keeps the same per-subband work on
    fewer subbands centred on 135 MHz (a small case for profiling); ``nchan``
    = 32 gives channels of 2048 bins at the same N."""
    g = np.random.default_rng(102)
    T = nsamp / 195312.5
    pulses = tuple(Pulse(float(g.uniform(1.0, max(1.5, T - 3.0))), float(g.uniform(5, 60)),
                         float(g.uniform(0.2e-3, 5e-3)), 0.5) for _ in range(5))
    name = f"lofar-{nsub}sub-2^{int(np.log2(nsamp))}" + ("" if nchan == 16 else f"-{nchan}ch")
    return Workload(name, nsub, nsamp, 135.0, 0.1953125, tuple(0.5 * i for i in range(128)), nchan, 8, 1 << 16, 2,
                    pulses)
