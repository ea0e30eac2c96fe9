#!/usr/bin/env python3
"""Throughput of the coherent-dedispersion hot path on GB300.

One step = the whole filterbank of the 64-subband LOFAR-shaped workload
(64 x 195.3125 kHz subbands 128.75-141.25 MHz, 2^22 complex dual-pol samples
each with 5 dispersed pulses, N_bin 2^16, 128 DM trials 0..63.5, 16 channels,
nint 8): forward FFTs of every overlap-save segment, then chirp, backward FFTs,
detection and integration for every DM.  The metric is DM-trial x input samples
per second (units = ndm * nsub * nseg * S).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cdmt|reference]

Multi-GPU (torchrun, one rank per GPU): --shard replicas (default) runs one
independent beam per rank (weak scaling); --shard subbands splits one beam's
subbands across the ranks, each planning its slice with the whole band's
overlap, no data exchanged (strong scaling).

Timing: W untimed steps, then K steps between barrier + synchronize, CUDA
events on the launching stream, max over ranks.  The inputs (4.3 GB) are larger
than L2, so no flush is needed between steps.  --impl reference times the FP64
CPU oracle on a bounded sample of the same workload on the host cores.
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DM-trial·Gsamples/s on 1 GB300, FP32 vs tensor-core form at stated error"
UNIT = "DM-trial·Gsamples/s"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload(name, nsamp=0):
    """The named workload; nsamp > 0 shortens (or lengthens) its input, for profiling small cases."""
    import dataclasses
    w = _workload(name)
    return dataclasses.replace(w, nsamp=nsamp, name=f"{w.name}[nsamp {nsamp}]") if nsamp > 0 else w


def _workload(name):
    import synth
    if name == "lofar64":
        return synth.lofar64()
    if name == "lofar8":
        return synth.lofar64(nsub=8)
    if name == "lofar64c32":
        return synth.lofar64(nchan=32)
    if name == "tiny":
        return synth.tiny()
    if name == "paper":
        return synth.paper()
    raise SystemExit(f"unknown workload {name}")


def describe(w, info=None):
    d = {"workload": w.name, "nsub": w.nsub, "nsamp": w.nsamp, "f_centre_mhz": w.f_centre, "bw_sub_mhz": w.bw,
         "ndm": len(w.dms), "dm_range": [w.dms[0], w.dms[-1]], "nchan": w.nchan, "nint": w.nint, "nbin": w.nbin,
         "pulses": len(w.pulses)}
    if info:
        d.update({"nd": info["nd"], "nseg": info["nseg"], "nout": info["nout"], "dm_tile": info["dm_tile"]})
    return d


# ---------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus_id = bus_id
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 10:
                    continue
                if self.bus_id and self.bus_id.lower() not in p[1].lower():
                    continue
                rows.append(p)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        busy = [v for v in sm if v > 0.5 * max(sm)] if sm else []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        pw = [float(r[4]) for r in rows if r[4].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(busy)) if busy else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------- oracle leg


def oracle_sample(w, x, nd, n_sub, n_seg, nthreads=0):
    """Time the FP64 oracle on the first n_sub subbands x n_seg segments x all DMs."""
    import oracle
    oracle.build()
    S = w.nbin - nd * w.nchan
    span = (n_seg - 1) * S + w.nbin
    xs = np.ascontiguousarray(x[:n_sub, :span])
    fc = w.f_centre - 0.5 * (w.nsub - n_sub) * w.bw
    t0 = time.perf_counter()
    oracle.filterbank(xs, fc, w.bw, w.dms, w.nchan, w.nint, w.nbin, nd, nthreads)
    dt = time.perf_counter() - t0
    units = len(w.dms) * n_sub * n_seg * S
    return units, dt, oracle.max_threads() if nthreads <= 0 else nthreads


def reference_arm(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    nd = w.nd if w.nd >= 0 else oracle.overlap(w.nsub, w.f_centre, w.bw, w.dms, w.nchan, w.nint, w.nbin)
    n_sub, n_seg = [int(v) for v in args.cpu_sample.split("x")]
    log(f"reference arm: FP64 oracle, {n_sub} subbands x {n_seg} segments x {len(w.dms)} DMs per step")
    x = w.voltages(threads=16)
    for _ in range(args.warmup):
        oracle_sample(w, x, nd, n_sub, n_seg)
    tot_u, tot_t, cores = 0, 0.0, 1
    for _ in range(args.steps):
        u, dt, cores = oracle_sample(w, x, nd, n_sub, n_seg)
        tot_u += u
        tot_t += dt
    v = tot_u / tot_t / 1e9
    sample = f"{n_sub} of {w.nsub} subbands x {n_seg} of the segments x all {len(w.dms)} DMs per step"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(w),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU leg


def kernel_source_hash(form="fp16"):
    """Hash of the sources the form's DM-stage kernel is compiled from (the key of its traffic figure)."""
    files = ("kernels_fp32.cu", "kernels_fp32_pair.cu", "fft_core.cuh", "tc_ptx.cuh", "cdmt_internal.h") \
        if form == "fp32" else \
        ("kernels_tc.cu", "fft_core.cuh", "tc_ptx.cuh", "cdmt_internal.h")
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1607_00909_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM bytes per DM-trial x sample of the DM-stage kernel from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum per launch / units per launch), valid for the sources of that form's kernel
# whose hash is recorded (kernel_source_hash); null otherwise.
NCU_TRAFFIC = {
    # 8-subband workload, one launch of k_dedisperse_tc (FP16, persistent, nint 8): 547.4 MB read +
    # 2069.1 MB written for 4.253e9 units (ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,
    # 4th launch)
    "d561d216c3f24e5d:fp16": 0.6152,
    # 8-subband workload, one launch of k_dedisperse_pair (FP32, 16 channels): 543.2 MB read +
    # 2066.9 MB written for 4.253e9 units (same capture command with the FP32 form)
    "11fe8e4f74697758:fp32": 0.6137,
    # the paper's setup at 2^20 samples, one launch of k_dedisperse_pair at M = 8192 (FP32, 8
    # channels, nint 1): 232.3 MB read + 3241.0 MB written for 8.258e8 units
    "11fe8e4f74697758:fp32:m8192": 4.2062,
}

try:
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as _f:
        MEASURED = json.load(_f)
except (OSError, ValueError):
    MEASURED = {}


PREC = {"fp32": 0, "fp16": 1, "bf16": 2}
DTYPE = {"fp32": "f32", "fp16": "f16 (FP32 accumulate)", "bf16": "bf16 hi/lo (FP32 accumulate)"}


def max_over_ranks(v: float, world: int, device=None) -> float:
    """The largest v over the ranks of the process group (v itself on one rank):
    replicas are timed by their slowest member."""
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v: float, world: int, device=None) -> float:
    """The sum of v over the ranks of the process group (v itself on one rank)."""
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def subband_slice(nsub: int, world: int, rank: int) -> tuple[int, int]:
    """Subbands [lo, hi) of one rank when `world` ranks split one beam's nsub
    subbands as evenly as possible (the first nsub % world ranks take one more).
    Subbands are independent problems (Sec. 4 splits them across nodes), so the
    split needs no exchange of data."""
    base, extra = divmod(nsub, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def slice_view(w, lo: int, hi: int):
    """The workload's description restricted to subbands [lo, hi): the same subband
    frequencies (the centre moves to the slice's centre), DMs, channels and N."""
    import dataclasses
    fc = w.f_centre + (0.5 * (lo + hi - 1) - 0.5 * (w.nsub - 1)) * w.bw
    return dataclasses.replace(w, nsub=hi - lo, f_centre=fc, name=f"{w.name}[subbands {lo}:{hi}]")


def replica_value(units_per_rank: float, steps: int, ms_max: float, world: int) -> float:
    """Whole-job throughput of `world` independent replicas (one beam each, same
    shapes) in G units/s: every rank's units over the slowest rank's time."""
    return world * units_per_rank * steps / (ms_max / 1e3) / 1e9


def sampled_error(w, x, out, info, ntile=32, seed=5):
    """max |gpu - oracle| / mean(oracle) and the RMS ratio on ntile random
    (subband, segment, DM) tiles of this run's output."""
    import oracle
    g = np.random.default_rng(seed)
    sub = g.integers(0, w.nsub, ntile)
    seg = g.integers(0, info["nseg"], ntile)
    dmi = g.integers(0, len(w.dms), ntile)
    o = oracle.tiles(x, w.f_centre, w.bw, w.dms, w.nchan, w.nint, w.nbin, info["nd"], sub, seg, dmi)
    L = (info["mbin"] - info["nd"]) // w.nint
    gt = np.stack([out[dmi[t], sub[t] * w.nchan:(sub[t] + 1) * w.nchan, seg[t] * L:(seg[t] + 1) * L]
                   .cpu().numpy().astype(np.float64) for t in range(ntile)])
    d = gt - o
    return {"rel_max": float(np.max(np.abs(d)) / np.mean(o)),
            "rel_rms": float(np.linalg.norm(d) / np.linalg.norm(o)), "tiles": ntile}


def time_cufft_unfused(w, xin, out, info, dev, stream, args):
    """The paper's own design on the same GPU, as a timed comparison (not the product path):
    batched cuFFT transforms (torch.fft, unitary) with the chirp multiply, the per-channel swap and
    backward FFT, detection and integration as separate passes through device memory for every DM
    (Sec. 3, Algorithm 1 with cuFFT).  Chirp phases DM K are reduced modulo 1 in FP64 per DM.
    Returns throughput, time per step and the largest difference from the headline filterbank."""
    import torch
    nsub, nchan, nint = w.nsub, w.nchan, w.nint
    N, M, nd, S, nseg = info["nbin"], info["mbin"], info["nd"], info["nvalid"], info["nseg"]
    bw = w.bw
    seglen = (M - nd) // nint
    D = 4.148808e3
    # K [nsub][N] in cycles per unit DM (Eq. 1, per channel), FP64 on the host
    s_idx = np.arange(nsub)[:, None, None]
    c_idx = np.arange(nchan)[None, :, None]
    j = np.arange(M)[None, None, :]
    nu_s = w.f_centre + (s_idx - 0.5 * (nsub - 1)) * bw
    nu_c = nu_s - 0.5 * bw + (c_idx + 0.5) * bw / nchan
    nu = (j - M / 2) * bw / N
    K = torch.from_numpy((1e6 * D * nu * nu / (nu_c * nu_c * (nu_c + nu))).reshape(nsub, N)).to(dev)
    xc = torch.view_as_complex(xin.view(nsub, w.nsamp, 2, 2))            # [nsub][nsamp][pol]
    dms = [float(v) for v in w.dms]
    o = torch.empty((len(dms), nsub * nchan, nseg * seglen), dtype=torch.float32, device=dev)

    def step():
        seg = xc.transpose(1, 2).unfold(2, N, S)                           # [nsub][pol][nseg][N]
        X = torch.fft.fftshift(torch.fft.fft(seg, norm="ortho"), dim=-1)
        for d, dm in enumerate(dms):
            ph = dm * K
            ph = ph - torch.round(ph)
            H = torch.polar(torch.ones_like(ph, dtype=torch.float32), (-2.0 * np.pi * ph).to(torch.float32))
            Y = (X * H[:, None, None, :]).view(nsub, 2, nseg, nchan, M)
            y = torch.fft.ifft(torch.fft.ifftshift(Y, dim=-1), norm="ortho")
            P = (y.real * y.real + y.imag * y.imag).sum(dim=1)             # [nsub][nseg][nchan][M]
            I = P[..., nd // 2: M - nd // 2].reshape(nsub, nseg, nchan, seglen, nint).sum(dim=-1)
            o[d] = I.permute(0, 2, 1, 3).reshape(nsub * nchan, nseg * seglen)

    with torch.cuda.stream(stream):
        step()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nstep = 2
        for _ in range(nstep):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / nstep
    units = len(dms) * nsub * nseg * S
    diff = float((o - out).abs().max() / out.mean())
    del o, K
    torch.cuda.empty_cache()
    return {"value": units / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "max_rel_diff_vs_headline": diff,
            "note": "the paper's unfused design: cuFFT (torch.fft) forward and backward FFTs, chirp multiply, "
                    "detection and integration as separate device-memory passes per DM; a comparison, "
                    "not the product path"}


def time_form(cdmt, w, xin, out, prec, args, dev, stream, barrier, world, nd=-1):
    """Plan one precision form, warm up, time args.steps executes; returns a dict.
    nd >= 0 fixes the overlap (a slice of a band keeps the whole band's)."""
    import torch
    import torch.distributed as dist
    plan = cdmt.Plan(w.nsub, w.nsamp, w.f_centre, w.bw, w.dms, w.nchan, w.nint, nbin=w.nbin, precision=PREC[prec],
                     host_block=args.host_block, nd=nd)
    info = plan.info
    st = stream.cuda_stream
    for _ in range(args.warmup):
        plan.execute(xin.data_ptr(), out.data_ptr(), 0, st)
    torch.cuda.synchronize(dev)
    plan.device_status()
    cdmt.cdmt_set_timing(plan.handle, True)
    cdmt.cdmt_stage_times(plan.handle)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.execute(xin.data_ptr(), out.data_ptr(), 0, st)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    plan.device_status()
    ms = ev0.elapsed_time(ev1)
    (fwd_ms, dd_ms), (fwd_n, dd_n) = cdmt.cdmt_stage_times(plan.handle)
    cdmt.cdmt_set_timing(plan.handle, False)
    ms_max = max_over_ranks(ms, world, dev)
    units_all = sum_over_ranks(info["units"], world, dev)   # every rank's units (equal for replicas)
    return {"plan": plan, "info": info, "ms_max": ms_max, "fwd_ms": fwd_ms, "dd_ms": dd_ms, "fwd_n": fwd_n,
            "dd_n": dd_n, "steps": args.steps, "units_all": units_all,
            "value": units_all * args.steps / (ms_max / 1e3) / 1e9}


def dm_stage_roofline(form, r, props, sm_max):
    """Roofline of one form's DM-stage kernel: the slower of (a) the nominal FFT flops
    10 N log2(M) / S per unit (2 polarisations x n_c backward M-point FFTs per segment,
    5 M log2 M each, and the forward N-point FFT amortised over the DMs is left out as in
    the definition) at the form's peak (FP32: SMs x 128 lanes x 2 x SM clock, derived;
    FP16 / BF16: the measured sustained bf16 dense peak) and (b) the algorithmic bytes
    16 N / (S ndm) + 4 / nint per unit (the spectra read once per DM tile, the filterbank
    written once) at the measured HBM bandwidth, divided by the kernel's measured time
    per launch.  The tensor-core forms also report the GEMM work they issue (the
    64-point DFTs as dense real GEMMs) against the tensor peak, as a utilisation of the
    tensor pipe (not the roofline)."""
    info = r["info"]
    units = info["units"]
    nbin, mbin, S = info["nbin"], info["mbin"], info["nvalid"]
    t = r["dd_ms"] / max(1, r["dd_n"]) / 1e3          # seconds per DM-stage launch
    launches_per_step = r["dd_n"] / max(1, r["steps"])
    units_launch = units / launches_per_step
    flops_unit = 10.0 * nbin * np.log2(mbin) / S
    bytes_unit = 16.0 * nbin / (S * info["ndm"]) + 4.0 / info["nint"]
    hbm = MEASURED.get("hbm_gbs") or 6800.0
    if form == "fp32":
        fpeak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
        fbasis = f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz"
        kernel, fbound = ("k_dedisperse_pair" if mbin >= 4096 else "k_dedisperse"), "alu"
    else:
        fpeak = MEASURED.get("bf16_tflops_sustained") or 1700.0
        fbasis = "measured bf16 dense GEMM, sustained (MEASURED_PEAKS.json); the FP16 dense rate equals BF16"
        kernel, fbound = "k_dedisperse_tc", "tensor"
    t_flop = flops_unit * units_launch / (fpeak * 1e12)
    t_byte = bytes_unit * units_launch / (hbm * 1e9)
    if t_byte >= t_flop:
        rf = {"bound": "hbm", "achieved": bytes_unit * units_launch / t / 1e9, "peak": hbm, "unit": "GB/s",
              "peak_basis": "measured HBM copy bandwidth (MEASURED_PEAKS.json)"}
    else:
        rf = {"bound": fbound, "achieved": flops_unit * units_launch / t / 1e12, "peak": fpeak, "unit": "TFLOP/s",
              "peak_basis": fbasis}
    rf["frac"] = max(t_flop, t_byte) / t
    tr = NCU_TRAFFIC.get(kernel_source_hash(form) + ":" + form + (":m8192" if mbin == 8192 else ""))
    rf.update({"traffic": tr * units_launch if tr else None, "kernel": kernel,
               "definition": "slower of nominal FFT flops at the form's peak and algorithmic bytes at HBM bandwidth, "
                             "over the kernel's time per launch",
               "flops_per_unit": flops_unit, "bytes_per_unit": bytes_unit, "units_per_launch": units_launch,
               "flop_leg_ms": t_flop * 1e3, "byte_leg_ms": t_byte * 1e3, "flop_peak_tflops": fpeak,
               "flop_peak_basis": fbasis, "kernel_ms_per_launch": t * 1e3,
               "nominal_fft_tflops": flops_unit * units_launch / t / 1e12,
               "share_of_step": r["dd_ms"] / max(1e-9, r["dd_ms"] + r["fwd_ms"])})
    if form != "fp32":
        # the tensor-core GEMM work issued per (channel, DM), P = M / 64: pass A 128 x 2P x 2P and
        # pass B 128 x 2P x 128, 2 flops per multiply-add (x3 for the BF16 hi/lo products)
        mult = 3 if form == "bf16" else 1
        P_ = mbin // 64
        tc_unit = mult * 2 * 128 * (2 * P_) * (2 * P_ + 128) * info["nchan"] / S
        ach = tc_unit * units_launch / t / 1e12
        rf["tensor_pipe_issued"] = {"flops_per_unit": tc_unit, "achieved_tflops": ach, "peak_tflops": fpeak,
                                    "frac": ach / fpeak,
                                    "note": "dense real DFT GEMMs issued on the tensor cores (17x the nominal FFT "
                                            "flops at M = 4096): a utilisation of the tensor pipe, not the roofline"}
        # the multi-pipe bound of the form as built: the slowest of its pipes at their peaks -- the
        # issued GEMM flops (with the dense-DFT tax) on the tensor cores, the FP32 work around the
        # GEMMs (per bin and DM, both polarisations: chirp 12, twiddle 12, detection 7 flops) on the
        # FP32 lanes, and the algorithmic bytes on HBM; the chirp phase needs no FP64 per DM (the
        # fixed-point words are computed in FP64 once per plan)
        alu_unit = 31.0 * nbin / S
        alu_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
        legs = {"tensor": tc_unit * units_launch / (fpeak * 1e12) * 1e3,
                "fp32_alu": alu_unit * units_launch / (alu_peak * 1e12) * 1e3,
                "hbm": t_byte * 1e3}
        slow = max(legs, key=legs.get)
        rf["multi_pipe"] = {"bound": slow, "frac": legs[slow] / (t * 1e3), "legs_ms": legs,
                            "fp32_flops_per_unit": alu_unit, "fp32_peak_tflops": alu_peak,
                            "note": "the slowest pipe of the form as built at its peak over the kernel's time; "
                                    "the nominal roofline above counts the method's FFT flops only"}
    return rf


def gpu_arm(args, w):
    import torch
    import torch.distributed as dist

    import paper_1607_00909_gb300 as cdmt

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    head = forms[-1]
    shard = args.shard == "subbands" and world > 1
    nd_band = w.nd
    log(f"rank {rank}: generating {w.name} ...")
    t0 = time.perf_counter()
    if shard and w.nsub < world:
        raise SystemExit(f"--shard subbands needs at least one subband per rank ({w.nsub} subbands, {world} ranks)")
    if shard:   # one beam, its subbands split across the ranks; every rank keeps the band's overlap
        probe = cdmt.Plan(w.nsub, w.nbin, w.f_centre, w.bw, w.dms, w.nchan, w.nint, nbin=w.nbin, nd=w.nd)
        nd_band = probe.info["nd"]
        probe.close()
        lo, hi = subband_slice(w.nsub, world, rank)
        x = w.voltages(threads=16, sub=(lo, hi))
        w = slice_view(w, lo, hi)
    else:       # independent replicas: one beam per rank
        x = w.voltages(threads=16, beam=rank)
    log(f"rank {rank}: inputs ready in {time.perf_counter() - t0:.1f}s ({x.nbytes / 1e9:.2f} GB)")
    xin = torch.from_numpy(x).to(dev)
    stream = torch.cuda.current_stream(dev)
    props = torch.cuda.get_device_properties(dev)
    bus = None
    try:
        bus = f"{props.pci_domain_id:08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0"
    except AttributeError:
        pass

    results = {}
    out = None
    clocks = None
    for f in forms:
        if out is None:
            probe = cdmt.Plan(w.nsub, w.nsamp, w.f_centre, w.bw, w.dms, w.nchan, w.nint, nbin=w.nbin, nd=nd_band)
            out = torch.empty(probe.out_shape(), dtype=torch.float32, device=dev)
            probe.close()
        if f == head:
            with ClockSampler(bus) as clk:
                r = time_form(cdmt, w, xin, out, f, args, dev, stream, barrier, world, nd_band)
            clocks = clk.summary()
        else:
            r = time_form(cdmt, w, xin, out, f, args, dev, stream, barrier, world, nd_band)
        if rank == 0 and not args.no_error:
            r["error"] = sampled_error(w, x, out, r["info"])
        results[f] = r
        if f != head:
            r["plan"].close()
        log(f"rank {rank}: {f}: {r['value']:.2f} {UNIT}, {r['ms_max'] / args.steps:.2f} ms/step, "
            f"error {r.get('error')}")

    R = results[head]
    plan, info = R["plan"], R["info"]
    units = info["units"]
    units_all = R["units_all"]   # all ranks' units (world x units for replicas)

    # 8-bit redigitisation of the headline form's filterbank (Sec. 3), timed on its own:
    # a statistics pass reads the filterbank, a code pass reads it again and writes one byte per sample
    redig = None
    if not args.no_redigitise:
        ndm_, rows_, nout_ = plan.out_shape()
        u8 = torch.empty((ndm_, nout_, rows_), dtype=torch.uint8, device=dev)
        st_ = stream.cuda_stream
        for _ in range(max(3, args.warmup)):
            plan.redigitise(out, u8, stream=st_)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            plan.redigitise(out, u8, stream=st_)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        rms = e0.elapsed_time(e1) / args.steps
        nbytes = ndm_ * rows_ * nout_ * (4 + 4 + 1)
        hbm = MEASURED.get("hbm_gbs")
        redig = {"ms_per_launch": rms, "kernels": 2, "bytes_per_launch": nbytes,
                 "achieved_gbs": nbytes / rms / 1e6, "peak_gbs": hbm,
                 "frac": (nbytes / rms / 1e6) / hbm if hbm else None, "bound": "hbm",
                 "output_bytes": ndm_ * rows_ * nout_, "levels_per_sigma": cdmt.REDIG_LEVELS,
                 "note": "8-bit codes, per DM time-major spectra in decreasing frequency; not part of the step"}
        del u8
        log(f"rank {rank}: redigitise: {rms:.2f} ms per launch, {nbytes / rms / 1e6:.0f} GB/s")

    # incoherent dedispersion of the headline filterbank over 500 fine trials (-0.5 .. +0.498 in
    # steps of 0.002) around every coherent DM (Sec. 4), timed on its own
    incoh = None
    if not args.no_incoherent:
        lo_, step_, nk_ = -0.5, 0.002, 500
        nt_o, _ = cdmt.cdmt_incoherent_info(plan.handle, lo_, step_, nk_)
        ndm_, rows_, nout_ = plan.out_shape()
        io = torch.empty((ndm_, nk_, nt_o), dtype=torch.float32, device=dev)
        st_ = stream.cuda_stream
        plan.incoherent(out, lo_, step_, nk_, io, st_)   # uploads the shift table
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_inc = max(1, min(args.steps, 3))
        e0.record(stream)
        for _ in range(n_inc):
            plan.incoherent(out, lo_, step_, nk_, io, st_)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ims = e0.elapsed_time(e1) / n_inc
        adds = ndm_ * nk_ * nt_o * rows_
        peak_adds = torch.cuda.get_device_properties(dev).multi_processor_count * 128 * (
            (clocks or {}).get("sm_max_mhz") or MEASURED.get("sm_max_mhz") or 2070.0) * 1e6
        incoh = {"ms_per_launch": ims, "trials": nk_, "ddm": [lo_, step_], "nt_out": nt_o,
                 "adds_per_launch": adds, "g_adds_per_s": adds / ims / 1e6, "bound": "alu",
                 "peak_g_adds_per_s": peak_adds / 1e9, "frac": (adds / (ims / 1e3)) / peak_adds,
                 "output_bytes": io.numel() * 4,
                 "note": "FP32 adds of shifted channel rows; peak = SMs x 128 lanes x SM clock; not part of the step"}
        del io
        log(f"rank {rank}: incoherent: {ims:.2f} ms per launch, {adds / ims / 1e6:.0f} G adds/s")

    # the paper's unfused cuFFT design on the same GPU, beside the fused kernels (rank 0)
    cufft = None
    if rank == 0 and not args.no_cufft:
        cufft = time_cufft_unfused(w, xin, out, info, dev, stream, args)
        log(f"rank {rank}: cuFFT unfused comparison: {cufft['value']:.2f} {UNIT}, {cufft['ms_per_step']:.1f} ms/step, "
            f"max rel diff vs headline {cufft['max_rel_diff_vs_headline']:.2e}")

    # ---- roofline of the dominant kernel (the DM stage) of every form: the slower of the nominal
    #      FFT flops at the form's peak and the algorithmic bytes at HBM bandwidth
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    rooflines = {f: dm_stage_roofline(f, r, props, sm_max) for f, r in results.items()}
    roofline = rooflines[head]

    # ---- end to end through the host-memory entry points: each call timed on its own (host clock
    #      around the call, which returns once the result is in host memory), over args.e2e_calls calls
    e2e = None
    if not args.no_e2e:
        st = stream.cuda_stream

        def timed_calls(fn):
            fn()   # warm-up (allocates the staging)
            barrier()
            torch.cuda.synchronize(dev)
            ts = []
            for _ in range(args.e2e_calls):
                t0 = time.perf_counter()
                fn()
                torch.cuda.synchronize(dev)
                ts.append(time.perf_counter() - t0)
            med = max_over_ranks(float(np.median(ts)), world, dev)
            return med, {"calls": len(ts), "ms_median": med * 1e3, "ms_min": min(ts) * 1e3, "ms_max": max(ts) * 1e3}

        hin = torch.from_numpy(x).pin_memory()
        hout = torch.empty(plan.out_shape(), dtype=torch.float32, pin_memory=True)
        med, spread = timed_calls(lambda: plan.execute_host(hin.data_ptr(), hout.data_ptr(), 0, st))
        plan.device_status()
        e2e = {"value": units_all / med / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(hin.numel() * 4), "d2h_bytes_per_step": int(hout.numel() * 4),
               "ms_per_step": med * 1e3, "spread": spread, "output": "float32 filterbank",
               "timing": "median of single calls, host clock around each call (inputs in pinned host memory, "
                         "result back in pinned host memory)"}
        del hout
        # the paper's pipeline (Algorithm 1): each block redigitised to 8 bits on the device, codes to host
        hu8 = torch.empty((plan.out_shape()[0], plan.out_shape()[2], plan.out_shape()[1]), dtype=torch.uint8,
                          pin_memory=True)
        kb = [0]

        def call_u8():
            kb[0] = plan.execute_host_u8(hin.data_ptr(), hu8.data_ptr(), st)
        med, spread = timed_calls(call_u8)
        plan.device_status()
        e2e["u8"] = {"value": units_all / med / 1e9, "unit": UNIT,
                     "h2d_bytes_per_step": int(hin.numel() * 4), "d2h_bytes_per_step": int(hu8.numel()),
                     "ms_per_step": med * 1e3, "spread": spread, "block_segments": kb[0],
                     "output": "8-bit filterbank (statistics per block), decreasing frequency, time-major"}
        del hin
        # the paper's own I/O: 8-bit voltages in (4 bytes per dual-polarisation sample, one scale per
        # subband, sigma at 16 levels), 8-bit filterbank out
        xs = xin.view(w.nsub, -1)
        sc = (xs.std(dim=1) / 16.0).clamp_min(1e-30).to(torch.float32)
        hin8 = torch.clamp(torch.round(xs / sc[:, None]), -127, 127).to(torch.int8).view(xin.shape).cpu().pin_memory()
        hsc = sc.cpu().pin_memory()
        plan8 = cdmt.Plan(w.nsub, w.nsamp, w.f_centre, w.bw, w.dms, w.nchan, w.nint, nbin=w.nbin,
                          precision=PREC[head], in_dtype=cdmt.CDMT_IN_I8, host_block=args.host_block, nd=nd_band)

        def call_i8():
            kb[0] = plan8.execute_host_u8(hin8.data_ptr(), hu8.data_ptr(), st, hsc.data_ptr())
        med, spread = timed_calls(call_i8)
        plan8.device_status()
        e2e["i8_u8"] = {"value": units_all / med / 1e9, "unit": UNIT,
                        "h2d_bytes_per_step": int(hin8.numel() + hsc.numel() * 4), "d2h_bytes_per_step": int(hu8.numel()),
                        "ms_per_step": med * 1e3, "spread": spread, "block_segments": kb[0],
                        "output": "int8 voltages in (per-subband scale), 8-bit filterbank out"}
        plan8.close()
        del plan8, hin8, hsc, hu8

    # ---- serving: one beam of the serving workload (288 subbands, blocks of 2^16 samples, 1024 DMs)
    serving = None
    if not args.no_serving and rank == 0:
        serving = serving_probe(cdmt, dev, args)

    cpu = None
    if rank == 0 and not args.no_cpu:
        n_sub, n_seg = [int(v) for v in args.cpu_sample.split("x")]
        u, dt, cores = oracle_sample(w, x, info["nd"], n_sub, n_seg)
        cpu = {"value": u / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n_sub} of {w.nsub} subbands x {n_seg} of {info['nseg']} segments x all {len(w.dms)} DMs "
                         f"({u:.3g} units in {dt:.1f} s)"}

    if rank == 0:
        cfg = describe(w, info)
        cfg.update({"l2": f"inputs ({x.nbytes / 1e9:.2f} GB) larger than L2; no flush", "precision": head,
                    "parallelism": (f"subbands split over {world} GPUs" if shard else f"replicas x{world}")
                    if world > 1 else "single GPU"})
        if shard:
            cfg.update({"workload": describe(workload(args.workload))["workload"], "nsub": w.nsub * world,
                        "subbands_per_rank": w.nsub, "nd": nd_band})
        launches = (R["fwd_n"] + R["dd_n"])
        line = {"metric": METRIC, "value": R["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": R["ms_max"] / args.steps, "higher_is_better": True,
                "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": DTYPE[head],
                "data": "synthetic", "config": cfg, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": int(launches),
                "error_vs_oracle": R.get("error"),
                "redigitise": redig,
                "incoherent": incoh,
                "comparisons": {"cufft_unfused": cufft},
                "serving": serving,
                "forms": {f: {"value": r["value"], "ms_per_step": r["ms_max"] / args.steps,
                              "dedisperse_ms_per_step": r["dd_ms"] / args.steps,
                              "forward_ms_per_step": r["fwd_ms"] / args.steps, "error_vs_oracle": r.get("error"),
                              "dtype": DTYPE[f], "roofline": rooflines[f]}
                          for f, r in results.items()}}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- batch of uneven beams

BATCH4 = [  # (nsub, log2 nsamp, ndm, nchan, nint): DMs k * 100 / ndm, k < ndm; 195.3125 kHz subbands at 135 MHz
    (288, 23, 1024, 16, 8),
    (160, 22, 512, 8, 4),
    (96, 22, 512, 32, 16),
    (32, 21, 256, 16, 8),
]


def batch_arm(args):
    """Four beams of uneven shapes through the batch API: one graph launch per
    round (forward stage of every beam + one persistent tensor-core launch).
    A step = every round = the whole input of every beam."""
    import torch

    import paper_1607_00909_gb300 as cdmt
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    g = torch.Generator(device=dev)
    ins, beams, units = [], [], 0.0
    t0 = time.perf_counter()
    for i, (nsub, lg, ndm, nchan, nint) in enumerate(BATCH4):
        g.manual_seed(1000 + i)
        x = torch.randn((nsub, 1 << lg, 4), generator=g, device=dev, dtype=torch.float32)
        x.mul_(float(np.sqrt(0.5)))
        ins.append(x)
        beams.append(dict(nsub=nsub, nsamp=1 << lg, f_centre=135.0, bw_sub=0.1953125, dm_first=0.0,
                          dm_step=100.0 / ndm, ndm=ndm, nchan=nchan, nint=nint, d_in=x.data_ptr()))
    torch.cuda.synchronize(dev)
    log(f"batch inputs ready in {time.perf_counter() - t0:.1f}s ({sum(x.numel() * 4 for x in ins) / 1e9:.1f} GB)")
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    batch = cdmt.Batch(beams, out_budget=24 << 30, autotune=args.autotune, stream=stream.cuda_stream)
    log(f"batch planned in {time.perf_counter() - t0:.1f}s: {batch.nround} rounds")
    per_beam = []
    for b, inf in zip(beams, batch.infos):
        units += inf.plan.units
        per_beam.append({"nsub": b["nsub"], "nsamp": b["nsamp"], "ndm": b["ndm"], "nchan": b["nchan"],
                         "nint": b["nint"], "nbin": inf.plan.nbin, "nd": inf.plan.nd, "nseg": inf.plan.nseg,
                         "precision": ["fp32", "fp16", "bf16"][inf.tune.precision], "dm_tile": inf.tune.dm_tile,
                         "tuned_units_per_s": inf.tune.units_per_s, "seg_per_round": inf.seg_per_round})
    for _ in range(args.warmup):
        batch.run_round(0, stream.cuda_stream)
    torch.cuda.synchronize(dev)
    batch.status()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    props = torch.cuda.get_device_properties(dev)
    bus = None
    try:
        bus = f"{props.pci_domain_id:08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0"
    except AttributeError:
        pass
    with ClockSampler(bus) as clk:
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for _ in range(args.steps):
            batch.run(stream.cuda_stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    clocks = clk.summary()
    batch.status()
    ms = ev0.elapsed_time(ev1)
    value = units * args.steps / (ms / 1e3) / 1e9
    n_fp32 = sum(1 for p in per_beam if p["precision"] == "fp32")
    launches_per_round = 1 + 2 * len(beams) + 1 + n_fp32
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16 (FP32 accumulate)", "data": "synthetic",
            "config": {"workload": "batch of 4 uneven beams (288/160/96/32 subbands, 2^23/2^22/2^22/2^21 samples, "
                                   "1024/512/512/256 DMs over 0-100, 16/8/32/16 channels, nint 8/4/16/8)",
                       "rounds": batch.nround, "beams": per_beam, "autotune": bool(args.autotune),
                       "l2": "inputs (57 GB) larger than L2; no flush",
                       "output": "each round's filterbanks are written to the batch's round buffers "
                                 f"({batch.infos[0].out_bytes_total / 1e9:.1f} GB) and overwritten by the next round"},
            "gpu_launches": launches_per_round * batch.nround * args.steps, "clocks": clocks,
            "graph_launches_per_step": batch.nround}
    print(json.dumps(line), flush=True)
    batch.close()
    return 0


SERVE = dict(nsub=288, block_len=1 << 16, ndm=1024, dm_max=100.0, nchan=16, nint=8, f_centre=135.0, bw=0.1953125)


def _serve_run(cdmt, srv, beams, host_blocks, scale, nblk, pace_s=0.0, hist=None, probe=None):
    """Submit nblk blocks per beam (round-robin over beams; every pace_s seconds a
    round when pacing), wait for each in submission order, release its slot.
    hist[b] records the host block index of every block beam b received;
    probe(b, block number, result) sees each result before its release."""
    reqs = []
    t0 = time.perf_counter()

    def finish(item):
        b, kb, rid = item
        res = srv.wait(rid, 600.0)
        if probe is not None:
            probe(b, kb, res)
        srv.release(rid)

    for k in range(nblk):
        if pace_s > 0:
            dt = t0 + k * pace_s - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
        for b in beams:
            i = (k + b) % len(host_blocks)
            hist.setdefault(b, []).append(i)
            reqs.append((b, len(hist[b]) - 1,
                         srv.submit(b, host_blocks[i].data_ptr(), scale.data_ptr() if scale is not None else 0)))
        if pace_s > 0:  # under pacing, drain what is done before the next round arrives
            while reqs and srv.stats().blocks_running + srv.stats().blocks_queued < len(reqs):
                finish(reqs.pop(0))
    for item in reqs:
        finish(item)


def serving_probe(cdmt, dev, args, nblk=8, npaced=6):
    """One beam of the serving workload through the streaming server (SERVE: 288
    subbands at 135 MHz, blocks of 2^16 complex64 samples from pinned host memory,
    1024 DMs 0-100, 16 channels, nint 8, FP16 form, float32 filterbank in device
    slots): its real-time factor with blocks queued back to back, and its block
    latency (submit to GPU completion) when blocks arrive at the data rate; four
    sampled (subband, DM) tiles of two blocks against the FP64 oracle."""
    import torch
    c = SERVE
    shape = (c["nsub"], c["block_len"], 4)
    g = torch.Generator(device=dev)
    host_blocks = []
    for i in range(4):
        g.manual_seed(5000 + i)
        d = torch.randn(shape, generator=g, device=dev, dtype=torch.float32)
        h = torch.empty(shape, dtype=d.dtype, pin_memory=True)
        h.copy_(d)
        host_blocks.append(h)
        del d
    srv = cdmt.Server(hbm_budget=120 << 30)
    beam = srv.add_beam(c["nsub"], c["block_len"], c["f_centre"], c["bw"], 0.0, c["dm_max"] / c["ndm"], c["ndm"],
                        c["nchan"], c["nint"], precision=cdmt.CDMT_PREC_FP16)
    hist, samples = {}, []
    _serve_run(cdmt, srv, [beam], host_blocks, None, 3, hist=hist)
    torch.cuda.synchronize(dev)
    srv.reset_stats()
    rng = np.random.default_rng(8)
    rows = c["nsub"] * c["nchan"]
    pick = {4, 3 + nblk - 1}

    def probe(b, kb, res):
        if args.no_error or kb not in pick or res.nseg < 1:
            return
        view = cdmt.Server.block_view(res, c["ndm"], rows)
        seglen = res.samples // res.nseg
        for _ in range(2):
            s_, d_ = int(rng.integers(0, c["nsub"])), int(rng.integers(0, c["ndm"]))
            samples.append((res.first_sample // seglen, s_, d_,
                            view[d_, s_ * c["nchan"]:(s_ + 1) * c["nchan"], :seglen].cpu().numpy()))
    _serve_run(cdmt, srv, [beam], host_blocks, None, nblk, hist=hist, probe=probe)
    sat = srv.stats()
    srv.reset_stats()
    block_s = c["block_len"] / (c["bw"] * 1e6)
    _serve_run(cdmt, srv, [beam], host_blocks, None, npaced, pace_s=block_s, hist=hist)
    paced = srv.stats()
    srv.close()
    err = _serve_error(c, host_blocks, None, hist[beam], samples, False) if samples else None
    del host_blocks
    torch.cuda.empty_cache()
    log(f"serving, one beam: {sat.realtime_factor:.2f}x real time, {sat.units_per_s / 1e9:.1f} {UNIT}; paced latency "
        f"p50 {paced.latency_p50_ms:.1f} ms, p99 {paced.latency_p99_ms:.1f} ms")
    return {"workload": f"one beam of {c['nsub']} subbands, blocks of 2^16 complex64 samples ({block_s * 1e3:.1f} ms "
                        f"of data) from pinned host memory, {c['ndm']} DMs 0-{c['dm_max']:g}, {c['nchan']} channels, "
                        f"nint {c['nint']}, FP16 form, float32 filterbank kept in device slots",
            "realtime_factor": sat.realtime_factor, "value": sat.units_per_s / 1e9, "unit": UNIT,
            "blocks": sat.blocks_done, "latency_p50_ms": sat.latency_p50_ms, "latency_p99_ms": sat.latency_p99_ms,
            "paced": {"blocks": paced.blocks_done, "latency_p50_ms": paced.latency_p50_ms,
                      "latency_p99_ms": paced.latency_p99_ms, "latency_max_ms": paced.latency_max_ms,
                      "note": "blocks submitted every 335.5 ms (the data rate)"},
            "target_realtime_factor": 10.0, "error_vs_oracle": err}


def _serve_error(c, host_blocks, scale, hist0, samples, i8):
    """Sampled (subband, DM) tiles of beam 0's first segment in two blocks against
    the FP64 oracle, from the same stream rebuilt from the host blocks."""
    import oracle
    dms = [i * c["dm_max"] / c["ndm"] for i in range(c["ndm"])]
    nbin, nchan, nint, L = 4096 * c["nchan"], c["nchan"], c["nint"], c["block_len"]
    nd = oracle.overlap(c["nsub"], c["f_centre"], c["bw"], dms, nchan, nint, nbin)
    S = nbin - nd * nchan
    gs, os_ = [], []
    for (seg0, s, dmi, g) in samples:
        t0 = seg0 * S
        x = np.empty((1, nbin, 4), dtype=np.float32)
        pos = t0
        while pos < t0 + nbin:   # gather the segment from the blocks the beam received
            blk, off = divmod(pos, L)
            n = min(L - off, t0 + nbin - pos)
            src = host_blocks[hist0[blk]][s, off:off + n].numpy()
            x[0, pos - t0:pos - t0 + n] = (src.astype(np.float32) * np.float32(scale[s].item())) if i8 else src
            pos += n
        fc = c["f_centre"] + (s - (c["nsub"] - 1) / 2) * c["bw"]
        o = oracle.tiles(x, fc, c["bw"], dms, nchan, nint, nbin, nd, [0], [0], [dmi])[0]
        gs.append(g.astype(np.float64))
        os_.append(o)
    g, o = np.stack(gs), np.stack(os_)
    d = g - o
    return {"rel_max": float(np.max(np.abs(d)) / np.mean(o)), "rel_rms": float(np.linalg.norm(d) / np.linalg.norm(o)),
            "tiles": len(samples), "beam": 0}


# the serving band planned as one long input with the subband-wide chirp, whose overlap
# holds the lowest subband's sweep (n_d = 1624 of M = 4096 at DM 100)
GROUPS = dict(nsub=288, nsamp=1 << 19, f_centre=135.0, bw=0.1953125, ndm=1024, dm_max=100.0, nchan=16, nint=8,
              nbin=1 << 16)
# the same lowest subband (so the same overlaps) over a quarter of the band, four times as long:
# 48 segments instead of 12, so rounding each group up to whole segments costs less
GROUPS_LONG = dict(GROUPS, nsub=72, nsamp=1 << 21, f_centre=135.0 - 108 * 0.1953125)


def groups_arm(args):
    """DM groups with their own overlap (cdmt_opts.dm_groups; with --group-nbin 1 also
    their own FFT length) against one overlap for the whole list, in the last of --forms.  A step = one execute over the whole input; units are
    those of the ungrouped plan (the same filterbank is delivered).  One sampled
    (subband, segment, DM) tile per group is checked against the oracle."""
    import torch

    import oracle
    import paper_1607_00909_gb300 as cdmt
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    c = GROUPS_LONG if args.workload == "groups-long" else GROUPS
    g = torch.Generator(device=dev)
    g.manual_seed(7000)
    x = torch.randn((c["nsub"], c["nsamp"], 4), generator=g, device=dev, dtype=torch.float32)
    x.mul_(float(np.sqrt(0.5)))
    dms = [i * c["dm_max"] / c["ndm"] for i in range(c["ndm"])]
    stream = torch.cuda.current_stream(dev)
    props = torch.cuda.get_device_properties(dev)
    bus = None
    try:
        bus = f"{props.pci_domain_id:08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0"
    except AttributeError:
        pass
    rng = np.random.default_rng(7001)
    form = [f.strip() for f in args.forms.split(",") if f.strip()][-1]
    out, res, clocks = None, {}, None
    for ng in [int(v) for v in args.dm_groups.split(",")]:
        plan = cdmt.Plan(c["nsub"], c["nsamp"], c["f_centre"], c["bw"], dms, c["nchan"], c["nint"], nbin=c["nbin"],
                         precision=PREC[form], chirp=cdmt.CDMT_CHIRP_SUBBAND, dm_groups=ng,
                         group_nbin=args.group_nbin)
        if out is None:
            out = torch.empty(plan.out_shape(), dtype=torch.float32, device=dev)
        st = stream.cuda_stream
        for _ in range(args.warmup):
            plan.execute(x.data_ptr(), out.data_ptr(), 0, st)
        torch.cuda.synchronize(dev)
        plan.device_status()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(bus) as clk:
            ev0.record(stream)
            for _ in range(args.steps):
                plan.execute(x.data_ptr(), out.data_ptr(), 0, st)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
        clocks = clk.summary()
        plan.device_status()
        ms = ev0.elapsed_time(ev1) / args.steps
        info, layout = plan.info, plan.groups()
        errs = []
        for gr in layout:
            nb = gr["nbin"]
            m = nb // c["nchan"]
            s = int(rng.integers(c["nsub"]))
            k = int(rng.integers(gr["nseg"]))
            di = gr["dm_first"] + int(rng.integers(gr["ndm"]))
            sv = nb - gr["nd"] * c["nchan"]
            xs = x[s:s + 1, gr["offset"] + k * sv:gr["offset"] + k * sv + nb].cpu().numpy()
            fc_s = c["f_centre"] + (s - 0.5 * (c["nsub"] - 1)) * c["bw"]
            o = oracle.tiles(xs, fc_s, c["bw"], [dms[di]], c["nchan"], c["nint"], nb, gr["nd"], [0], [0],
                             [0], chirp=1)[0]
            seglen = (m - gr["nd"]) // c["nint"]
            t0, t1 = k * seglen, min((k + 1) * seglen, info["nout"])
            gv = out[di, s * c["nchan"]:(s + 1) * c["nchan"], t0:t1].cpu().numpy()
            errs.append(float(np.max(np.abs(gv - o[:, :t1 - t0])) / np.mean(o[:, :t1 - t0])))
        res[ng] = {"value": info["units"] / (ms / 1e3) / 1e9, "ms_per_step": ms,
                   "overlaps": [gr["nd"] for gr in layout], "segments": [gr["nseg"] for gr in layout],
                   "channel_lengths": [gr["nbin"] // c["nchan"] for gr in layout],
                   "workspace_gb": info["workspace_bytes"] / 1e9, "sampled_rel_max_vs_oracle": max(errs),
                   "clocks": clocks}
        log(f"dm_groups {ng}: {res[ng]['value']:.1f} G/s, {ms:.1f} ms/step, overlaps {res[ng]['overlaps']}, "
            f"lengths {res[ng]['channel_lengths']}, sampled error {max(errs):.2e}")
        plan.close()
    best = max(res, key=lambda k: res[k]["value"])
    line = {"metric": METRIC, "value": res[best]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res[best]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[form], "data": "synthetic",
            "config": {"workload": f"{c['nsub']} subbands x {c['nsamp']} samples at {c['f_centre']} MHz, {c['ndm']} DMs "
                                   f"0-{c['dm_max']:g}, {c['nchan']} channels, nint {c['nint']}, N 2^16, one "
                                   f"transfer function per subband", "dm_groups": best,
                       "group_lengths": bool(args.group_nbin),
                       "l2": f"inputs ({x.numel() * 4 / 1e9:.1f} GB) larger than L2; no flush"},
            "dm_groups": {str(k): v for k, v in res.items()}, "roofline": None, "clocks": clocks,
            "gpu_launches": 3 * best * args.steps}
    print(json.dumps(line), flush=True)
    return 0


def serve_arm(args):
    """Streaming server: SERVE-shaped beams, blocks from pinned host memory.

    Three runs through one server: every beam saturated (blocks queued ahead:
    throughput and aggregate real-time factor), one beam saturated (its real-time
    factor), one beam paced at the data rate (its latency when blocks arrive in
    real time)."""
    import torch

    import paper_1607_00909_gb300 as cdmt
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    c = SERVE
    i8 = args.int8
    shape = (c["nsub"], c["block_len"], 4)
    g = torch.Generator(device=dev)
    host_blocks = []
    for i in range(4):
        g.manual_seed(5000 + i)
        if i8:
            d = torch.randint(-24, 25, shape, generator=g, device=dev, dtype=torch.int8)
        else:
            d = torch.randn(shape, generator=g, device=dev, dtype=torch.float32)
        h = torch.empty(shape, dtype=d.dtype, pin_memory=True)
        h.copy_(d)
        host_blocks.append(h)
    scale = torch.full((c["nsub"],), 0.05, dtype=torch.float32).pin_memory() if i8 else None
    srv = cdmt.Server(hbm_budget=120 << 30)
    t0 = time.perf_counter()
    beams = [srv.add_beam(c["nsub"], c["block_len"], c["f_centre"], c["bw"], 0.0, c["dm_max"] / c["ndm"], c["ndm"],
                          c["nchan"], c["nint"], precision=cdmt.CDMT_PREC_FP16,
                          in_dtype=cdmt.CDMT_IN_I8 if i8 else cdmt.CDMT_IN_C64,
                          out_dtype=cdmt.CDMT_OUT_U8 if args.u8 else cdmt.CDMT_OUT_F32) for _ in range(args.beams)]
    st0 = srv.stats()
    log(f"{args.beams} beams admitted in {time.perf_counter() - t0:.1f}s: {st0.hbm_bytes / 1e9:.1f} GB, "
        f"{st0.slots} output slots")
    hist, samples = {}, []
    _serve_run(cdmt, srv, beams, host_blocks, scale, args.warmup, hist=hist)
    torch.cuda.synchronize(dev)
    srv.reset_stats()
    rng = np.random.default_rng(7)
    pick = {args.warmup + 1, args.warmup + args.steps - 1}
    rows = c["nsub"] * c["nchan"]

    def probe(b, kb, res):   # copy a few tiles of beam 0's results before their slots are released
        if args.no_error or args.u8 or b != 0 or kb not in pick or res.nseg < 1:
            return
        view = cdmt.Server.block_view(res, c["ndm"], rows)
        seglen = res.samples // res.nseg
        for _ in range(4):
            s_, d_ = int(rng.integers(0, c["nsub"])), int(rng.integers(0, c["ndm"]))
            g = view[d_, s_ * c["nchan"]:(s_ + 1) * c["nchan"], :seglen].cpu().numpy()
            samples.append((res.first_sample // seglen, s_, d_, g))
    props = torch.cuda.get_device_properties(dev)
    bus = None
    try:
        bus = f"{props.pci_domain_id:08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0"
    except AttributeError:
        pass
    with ClockSampler(bus) as clk:
        _serve_run(cdmt, srv, beams, host_blocks, scale, args.steps, hist=hist, probe=probe)
    clocks = clk.summary()
    sat = srv.stats()
    block_s = c["block_len"] / (c["bw"] * 1e6)
    srv.reset_stats()
    _serve_run(cdmt, srv, beams[:1], host_blocks, scale, max(4, args.steps), hist=hist)
    one = srv.stats()
    srv.reset_stats()
    _serve_run(cdmt, srv, beams[:1], host_blocks, scale, max(8, args.steps), pace_s=block_s, hist=hist)
    paced = srv.stats()
    srv.close()
    err = _serve_error(c, host_blocks, scale, hist[0], samples, i8) if samples else None
    value = sat.units_per_s / 1e9
    in_bytes = (4 if i8 else 16) * c["nsub"] * c["block_len"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sat.wall_s * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16 (FP32 accumulate)", "data": "synthetic",
            "config": {"workload": f"streaming server, {args.beams} beams x {c['nsub']} subbands, blocks of "
                                   f"2^16 samples ({block_s * 1e3:.1f} ms of data), {c['ndm']} DMs 0-{c['dm_max']:g}, "
                                   f"{c['nchan']} channels, nint {c['nint']}, "
                                   + ("int8 input" if i8 else "complex64 input")
                                   + (", 8-bit output (redigitised per block)" if args.u8 else ", float32 output"),
                       "step": "one block of every beam, from pinned host memory",
                       "l2": "per-block inputs and outputs larger than L2; no flush",
                       "hbm_bytes": sat.hbm_bytes, "output_slots": sat.slots},
            "serving": {"all_beams": {"realtime_factor": sat.realtime_factor, "latency_p50_ms": sat.latency_p50_ms,
                                      "latency_p99_ms": sat.latency_p99_ms, "blocks": sat.blocks_done,
                                      "note": "blocks queued ahead (saturated); latency includes queueing"},
                        "one_beam": {"realtime_factor": one.realtime_factor, "units_per_s": one.units_per_s,
                                     "latency_p50_ms": one.latency_p50_ms, "latency_p99_ms": one.latency_p99_ms},
                        "one_beam_paced": {"latency_p50_ms": paced.latency_p50_ms,
                                           "latency_p99_ms": paced.latency_p99_ms,
                                           "latency_max_ms": paced.latency_max_ms, "blocks": paced.blocks_done}},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": in_bytes * args.beams,
                    "d2h_bytes_per_step": 0,
                    "note": "host blocks in; the filterbanks stay in device slots for the consumer"},
            "roofline": None, "gpu_launches": (6 if args.u8 else 4) * args.beams * args.steps, "clocks": clocks,
            "error_vs_oracle": err}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cdmt", choices=["cdmt", "reference"])
    ap.add_argument("--workload", default="lofar64", choices=["lofar64", "lofar8", "lofar64c32", "tiny", "paper", "batch4", "serve8",
                                                              "groups", "groups-long"])
    ap.add_argument("--dm-groups", default="1,2,4,8", help="groups: DM group counts to time")
    ap.add_argument("--group-nbin", type=int, default=0, help="groups: 1 = each group picks its own FFT length")
    ap.add_argument("--beams", type=int, default=8, help="serve8: beams served at once")
    ap.add_argument("--int8", action="store_true", help="serve8: int8 blocks (4 bytes per sample)")
    ap.add_argument("--u8", action="store_true", help="serve8: blocks redigitised to 8 bits on the device")
    ap.add_argument("--autotune", action="store_true", help="batch4: time candidates per beam")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--host-block", type=int, default=0,
                    help="segments per block of the host pipeline (e2e; 0: the plan's choice)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", default="4x8", help="oracle sample: SUBBANDSxSEGMENTS")
    ap.add_argument("--nsamp", type=int, default=0, help="input samples per subband (0: the workload's own)")
    ap.add_argument("--forms", default="fp32,bf16,fp16",
                    help="precision forms to time, comma-separated (fp32, fp16, bf16); the last is the headline")
    ap.add_argument("--no-error", action="store_true", help="skip the sampled error check against the oracle")
    ap.add_argument("--no-redigitise", action="store_true", help="skip timing the 8-bit redigitisation")
    ap.add_argument("--no-incoherent", action="store_true", help="skip timing the incoherent stage")
    ap.add_argument("--no-cufft", action="store_true", help="skip timing the unfused cuFFT comparison pipeline")
    ap.add_argument("--no-serving", action="store_true", help="skip the one-beam serving figures in the default run")
    ap.add_argument("--e2e-calls", type=int, default=10, help="host-memory calls timed per end-to-end leg")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "subbands"],
                    help="N > 1: one beam per rank (replicas, weak scaling) or one beam's subbands split across "
                         "the ranks (subbands, strong scaling)")
    args = ap.parse_args()
    if args.warmup < 3:
        log("note: fewer than 3 warm-up steps")
    if args.workload == "batch4" and args.impl != "reference":
        return batch_arm(args)
    if args.workload == "serve8" and args.impl != "reference":
        return serve_arm(args)
    if args.workload in ("groups", "groups-long") and args.impl != "reference":
        return groups_arm(args)
    w = workload(args.workload, args.nsamp)
    if args.workload == "paper" and args.forms != "fp32":
        log("paper workload: channels of 8192 bins run in the FP32 form only (--forms fp32)")
        args.forms = "fp32"
    if args.impl == "reference":
        return reference_arm(args, w)
    return gpu_arm(args, w)


if __name__ == "__main__":
    sys.exit(main())
