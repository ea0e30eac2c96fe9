"""Shared helpers of the GPU parity tests: running a plan on CUDA tensors, the
error metrics against the oracle, and the pulse S/N harness applied alike to
GPU and oracle filterbanks."""
import numpy as np

D = 4.148808e3


def rel_errors(g, o):
    """(max |g - o| / mean(o), ||g - o||_2 / ||o||_2): errors relative to the
    mean output, since per-element ratios of chi^2 outputs near 0 are ill-posed."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    d = g - o
    return float(np.max(np.abs(d)) / np.mean(o)), float(np.linalg.norm(d) / np.linalg.norm(o))


def gpu_filterbank(plan, x_np, stream=None, fill=np.nan):
    import torch
    import paper_1607_00909_gb300 as cdmt
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    out = torch.full(plan.out_shape(), float(fill), dtype=torch.float32, device="cuda")
    cdmt.run(plan, x, out, stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def pulse_snr(fb, dms, pulse, f_centre, bw, nsub, nchan, nint, nd):
    """S/N of one injected pulse in a filterbank [ndm][nsub*nchan][nout]: take
    the DM trial nearest the pulse's DM, shift every channel back by the
    closed-form inter-channel delay D DM (nu_c^-2 - nu_top^-2) (rounded to output
    samples), sum the channels, convolve with a boxcar of the pulse width, and
    return (peak - median) / (1.4826 MAD)."""
    r = bw * 1e6
    tsamp = nchan * nint / r
    idm = int(np.argmin(np.abs(np.asarray(dms) - pulse.dm)))
    dm = dms[idm]
    nu_top = f_centre + 0.5 * nsub * bw
    nus = f_centre + (np.arange(nsub) - 0.5 * (nsub - 1)) * bw
    rows = fb[idm]
    nout = rows.shape[1]
    series = np.zeros(nout)
    for s in range(nsub):
        for c in range(nchan):
            nuc = nus[s] - bw / 2 + (c + 0.5) * bw / nchan
            sh = int(round(D * dm * (1 / nuc ** 2 - 1 / nu_top ** 2) / tsamp))
            series += np.roll(rows[s * nchan + c], -sh)
    wbox = max(1, int(round(pulse.width_s / tsamp)))
    sm = np.convolve(series, np.ones(wbox), mode="same")
    t_exp = int(round((pulse.t0_s * r / nchan - nd / 2) / nint))
    lo, hi = max(0, t_exp - 4 * wbox - 8), min(nout, t_exp + 4 * wbox + 8)
    off = np.concatenate([sm[:max(0, lo - 4 * wbox)], sm[hi + 4 * wbox:]])
    med = np.median(off)
    mad = np.median(np.abs(off - med)) * 1.4826
    return float((sm[lo:hi].max() - med) / mad)


def pulse_geometry(pulse, dms, f_centre, bw, nsub, nchan, nint, nd):
    """The quantities of the S/N harness of :func:`pulse_snr` for one pulse:
    (index of the DM trial nearest the pulse's DM, per-row shift in output
    samples D DM (nu_c^-2 - nu_top^-2) at that trial, boxcar width in output
    samples, expected output sample of the pulse at the top of the band)."""
    r = bw * 1e6
    tsamp = nchan * nint / r
    idm = int(np.argmin(np.abs(np.asarray(dms) - pulse.dm)))
    dm = dms[idm]
    nu_top = f_centre + 0.5 * nsub * bw
    nus = f_centre + (np.arange(nsub) - 0.5 * (nsub - 1)) * bw
    nuc = (nus[:, None] - bw / 2 + (np.arange(nchan)[None, :] + 0.5) * bw / nchan).ravel()
    shifts = np.rint(D * dm * (1 / nuc ** 2 - 1 / nu_top ** 2) / tsamp).astype(np.int64)
    wbox = max(1, int(round(pulse.width_s / tsamp)))
    t_exp = int(round((pulse.t0_s * r / nchan - nd / 2) / nint))
    return idm, shifts, wbox, t_exp


def windowed_snr(rows_at, shifts, wbox, t_exp, half):
    """The S/N of :func:`pulse_snr` computed on the window [t_exp - half,
    t_exp + half) of the dedispersed series only: rows_at(r, a, b) returns
    samples a..b-1 of filterbank row r at the pulse's DM trial.  The series is
    the sum over rows of each row shifted back by its delay, convolved with a
    boxcar of the pulse width; S/N = (peak within 4 widths + 8 samples of t_exp
    - median of the rest of the window) / (1.4826 MAD of the rest)."""
    lo = t_exp - half
    series = np.zeros(2 * half)
    for r, sh in enumerate(shifts):
        series += rows_at(r, lo + sh, lo + sh + 2 * half)
    sm = np.convolve(series, np.ones(wbox), mode="same")
    c = half
    a, b = c - 4 * wbox - 8, c + 4 * wbox + 8
    off = np.concatenate([sm[2 * wbox:max(2 * wbox, a - 4 * wbox)], sm[b + 4 * wbox:2 * half - 2 * wbox]])
    med = np.median(off)
    mad = np.median(np.abs(off - med)) * 1.4826
    return float((sm[a:b].max() - med) / mad)
