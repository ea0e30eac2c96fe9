"""Python binding of libcdmt.so (the C ABI declared in include/cdmt.h).

Argument marshalling only: every step of the coherent-dedispersion path runs in
the library's CUDA kernels.  Function names mirror the C entry points
(cdmt_plan, cdmt_plan_ex, cdmt_plan_info, cdmt_execute, cdmt_execute_host,
cdmt_destroy, cdmt_strerror, cdmt_last_error); :class:`Plan` wraps them.
Device buffers are passed as raw pointers (for example ``tensor.data_ptr()``
of a CUDA tensor) and streams as ``cudaStream_t`` integers
(``torch.cuda.current_stream().cuda_stream``).

Importing this module loads the compiled library and raises if it is missing:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcdmt.so")

CDMT_OK, CDMT_EINVAL, CDMT_ENOMEM, CDMT_ECUDA, CDMT_ETIMEOUT, CDMT_EBUDGET, CDMT_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
CDMT_CHIRP_CHANNEL, CDMT_CHIRP_SUBBAND = 0, 1
CDMT_PREC_FP32, CDMT_PREC_FP16, CDMT_PREC_BF16 = 0, 1, 2
CDMT_IN_C64, CDMT_IN_I8 = 0, 1
CDMT_OUT_F32, CDMT_OUT_U8 = 0, 1
CDMT_STATIC_SCRATCH_BYTES = 64 * 1024 * 1024   # size of the array behind cdmt_execute_static


class cdmt_opts(ctypes.Structure):
    _fields_ = [("nbin", ctypes.c_int64), ("nd", ctypes.c_int64), ("dm_tile", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("in_dtype", ctypes.c_int32), ("chirp", ctypes.c_int32),
                ("seg_chunk", ctypes.c_int64), ("mem_budget", ctypes.c_int64), ("host_block", ctypes.c_int64),
                ("sk_nsigma", ctypes.c_double), ("dm_groups", ctypes.c_int32), ("group_nbin", ctypes.c_int32),
                ("reserved", ctypes.c_int64 * 3)]


class cdmt_info(ctypes.Structure):
    _fields_ = [("nsamp", ctypes.c_int64), ("nbin", ctypes.c_int64), ("mbin", ctypes.c_int64),
                ("nd", ctypes.c_int64), ("nvalid", ctypes.c_int64), ("nseg", ctypes.c_int64),
                ("nout", ctypes.c_int64), ("seg_chunk", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("in_bytes", ctypes.c_int64), ("out_bytes", ctypes.c_int64), ("units", ctypes.c_double),
                ("nsub", ctypes.c_int32), ("nchan", ctypes.c_int32), ("nint", ctypes.c_int32),
                ("ndm", ctypes.c_int32), ("dm_tile", ctypes.c_int32), ("uniform_dm", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("in_dtype", ctypes.c_int32), ("device", ctypes.c_int32),
                ("dm_groups", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


class cdmt_beam(ctypes.Structure):
    _fields_ = [("nsub", ctypes.c_int32), ("ndm", ctypes.c_int32), ("nsamp", ctypes.c_int64),
                ("f_centre_mhz", ctypes.c_double), ("bw_sub_mhz", ctypes.c_double), ("dm_first", ctypes.c_double),
                ("dm_step", ctypes.c_double), ("nchan", ctypes.c_int32), ("nint", ctypes.c_int32),
                ("d_in", ctypes.c_void_p)]


class cdmt_batch_opts(ctypes.Structure):
    _fields_ = [("out_budget", ctypes.c_int64), ("autotune", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("tune_cache", ctypes.c_char_p), ("reserved", ctypes.c_int64 * 6)]


class cdmt_batch_tune(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("dm_tile", ctypes.c_int32), ("nbin", ctypes.c_int64),
                ("units_per_s", ctypes.c_double), ("from_cache", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class cdmt_batch_beam_info(ctypes.Structure):
    _fields_ = [("plan", cdmt_info), ("tune", cdmt_batch_tune), ("nround", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("seg_per_round", ctypes.c_int64), ("d_out", ctypes.c_void_p),
                ("out_row_stride", ctypes.c_int64), ("out_bytes_total", ctypes.c_int64)]


class cdmt_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_int64), ("max_slots", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("reserved", ctypes.c_int64 * 6)]


class cdmt_stream_desc(ctypes.Structure):
    _fields_ = [("nsub", ctypes.c_int32), ("ndm", ctypes.c_int32), ("block_len", ctypes.c_int64),
                ("f_centre_mhz", ctypes.c_double), ("bw_sub_mhz", ctypes.c_double), ("dm_first", ctypes.c_double),
                ("dm_step", ctypes.c_double), ("nchan", ctypes.c_int32), ("nint", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("in_dtype", ctypes.c_int32), ("nbin", ctypes.c_int64),
                ("dm_tile", ctypes.c_int32), ("out_dtype", ctypes.c_int32), ("sk_nsigma", ctypes.c_double),
                ("reserved", ctypes.c_int64 * 3)]


class cdmt_block_result(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("index", ctypes.c_int64),
                ("d_out", ctypes.c_void_p), ("nseg", ctypes.c_int64), ("first_sample", ctypes.c_int64),
                ("samples", ctypes.c_int64), ("row_stride", ctypes.c_int64), ("latency_ms", ctypes.c_double),
                ("d_u8", ctypes.c_void_p), ("d_stats", ctypes.c_void_p), ("d_flags", ctypes.c_void_p)]


class cdmt_server_stats(ctypes.Structure):
    _fields_ = [("blocks_done", ctypes.c_int64), ("blocks_queued", ctypes.c_int64), ("blocks_running", ctypes.c_int64),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("latency_max_ms", ctypes.c_double), ("wall_s", ctypes.c_double), ("data_s", ctypes.c_double),
                ("realtime_factor", ctypes.c_double), ("units_per_s", ctypes.c_double), ("hbm_bytes", ctypes.c_int64),
                ("slots", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


class CdmtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} [status {status}]")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1607_00909_gb300.build.build() "
                          "(nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    lib.cdmt_plan.argtypes = [ctypes.POINTER(P), ctypes.c_int, i64, ctypes.c_double, ctypes.c_double, dp,
                              ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.cdmt_plan_ex.argtypes = lib.cdmt_plan.argtypes + [ctypes.POINTER(cdmt_opts)]
    lib.cdmt_plan_info.argtypes = [P, ctypes.POINTER(cdmt_info)]
    lib.cdmt_selftest_wait.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_double)]
    lib.cdmt_inject_timeout.argtypes = [P]
    lib.cdmt_plan_group.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_int64)]
    lib.cdmt_plan_group_nbin.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
    lib.cdmt_execute.argtypes = [P, P, P, P, P]
    lib.cdmt_execute_host.argtypes = [P, P, P, P, P]
    lib.cdmt_destroy.argtypes = [P]
    lib.cdmt_set_timing.argtypes = [P, ctypes.c_int]
    lib.cdmt_device_status.argtypes = [P]
    lib.cdmt_server_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(cdmt_server_opts)]
    lib.cdmt_server_destroy.argtypes = [P]
    lib.cdmt_server_add_beam.argtypes = [P, ctypes.POINTER(cdmt_stream_desc), ctypes.POINTER(ctypes.c_int)]
    lib.cdmt_server_submit.argtypes = [P, ctypes.c_int, P, P, ctypes.POINTER(ctypes.c_int64)]
    lib.cdmt_server_wait.argtypes = [P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(cdmt_block_result)]
    lib.cdmt_server_release.argtypes = [P, ctypes.c_int64]
    lib.cdmt_server_get_stats.argtypes = [P, ctypes.POINTER(cdmt_server_stats)]
    lib.cdmt_server_reset_stats.argtypes = [P]
    lib.cdmt_server_save_beam.argtypes = [P, ctypes.c_int, P, ctypes.POINTER(ctypes.c_int64)]
    lib.cdmt_server_restore_beam.argtypes = [P, ctypes.c_int, P, ctypes.c_int64]
    lib.cdmt_server_last_error.argtypes = [P]
    lib.cdmt_server_last_error.restype = ctypes.c_char_p
    lib.cdmt_batch_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(cdmt_beam),
                                      ctypes.POINTER(cdmt_batch_opts), P]
    lib.cdmt_batch_info.argtypes = [P, ctypes.c_int, ctypes.POINTER(cdmt_batch_beam_info)]
    lib.cdmt_batch_run_round.argtypes = [P, ctypes.c_int, P]
    lib.cdmt_batch_run.argtypes = [P, P]
    lib.cdmt_batch_status.argtypes = [P]
    lib.cdmt_batch_copy_out.argtypes = [P, ctypes.c_int, P, P]
    lib.cdmt_batch_destroy.argtypes = [P]
    lib.cdmt_batch_last_error.argtypes = [P]
    lib.cdmt_batch_last_error.restype = ctypes.c_char_p
    lib.cdmt_execute_static.argtypes = [ctypes.c_int, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, i64, P, P, P]
    lib.cdmt_stage_times.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    lib.cdmt_redigitise.argtypes = [P, P, P, P, P]
    lib.cdmt_redigitise_sk.argtypes = [P, P, P, P, ctypes.c_double, P, P]
    lib.cdmt_execute_host_u8.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_int64), P]
    lib.cdmt_execute_host_u8_ex.argtypes = [P, P, P, P, ctypes.POINTER(ctypes.c_int64), P]
    lib.cdmt_incoherent_info.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int64), P]
    lib.cdmt_incoherent.argtypes = [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int, P, P]
    lib.cdmt_strerror.argtypes = [ctypes.c_int]
    lib.cdmt_strerror.restype = ctypes.c_char_p
    lib.cdmt_last_error.argtypes = [P]
    lib.cdmt_last_error.restype = ctypes.c_char_p
    for f in ("cdmt_plan", "cdmt_plan_ex", "cdmt_plan_info", "cdmt_execute", "cdmt_execute_host", "cdmt_destroy",
              "cdmt_set_timing", "cdmt_stage_times", "cdmt_device_status", "cdmt_execute_static",
              "cdmt_batch_create", "cdmt_batch_info", "cdmt_batch_run_round", "cdmt_batch_run", "cdmt_batch_status",
              "cdmt_batch_destroy", "cdmt_batch_copy_out", "cdmt_server_create", "cdmt_server_destroy",
              "cdmt_server_add_beam", "cdmt_server_submit", "cdmt_server_wait", "cdmt_server_release",
              "cdmt_server_get_stats", "cdmt_server_reset_stats", "cdmt_redigitise", "cdmt_incoherent_info",
              "cdmt_incoherent", "cdmt_execute_host_u8", "cdmt_redigitise_sk", "cdmt_execute_host_u8_ex"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


_lib = _load()

EXPORTED = ("cdmt_plan", "cdmt_plan_ex", "cdmt_plan_info", "cdmt_plan_group", "cdmt_plan_group_nbin",
            "cdmt_selftest_wait",
            "cdmt_inject_timeout", "cdmt_execute", "cdmt_execute_host", "cdmt_destroy",
            "cdmt_strerror", "cdmt_last_error", "cdmt_set_timing", "cdmt_stage_times", "cdmt_device_status",
            "cdmt_redigitise", "cdmt_redigitise_sk", "cdmt_incoherent_info", "cdmt_incoherent",
            "cdmt_execute_host_u8", "cdmt_execute_host_u8_ex", "cdmt_execute_static", "cdmt_batch_create", "cdmt_batch_info", "cdmt_batch_run_round", "cdmt_batch_run",
            "cdmt_batch_status", "cdmt_batch_last_error", "cdmt_batch_destroy", "cdmt_batch_copy_out",
            "cdmt_server_create", "cdmt_server_destroy", "cdmt_server_add_beam", "cdmt_server_submit",
            "cdmt_server_wait", "cdmt_server_release", "cdmt_server_get_stats", "cdmt_server_reset_stats",
            "cdmt_server_last_error", "cdmt_server_save_beam", "cdmt_server_restore_beam")


def lib():
    return _lib


def cdmt_strerror(status: int) -> str:
    return _lib.cdmt_strerror(status).decode()


def cdmt_last_error(plan=None) -> str:
    return _lib.cdmt_last_error(plan).decode()


def _check(rc: int, plan=None):
    if rc != CDMT_OK:
        raise CdmtError(rc, f"{cdmt_strerror(rc)}: {cdmt_last_error(plan)}")


def cdmt_plan_ex(nsub, nsamp, f_centre, bw_sub, dm_list, nchan, nint, opts: cdmt_opts | None = None):
    """Create a plan; returns the opaque handle (int)."""
    dms = (ctypes.c_double * len(dm_list))(*[float(d) for d in dm_list])
    h = ctypes.c_void_p()
    rc = _lib.cdmt_plan_ex(ctypes.byref(h), int(nsub), int(nsamp), float(f_centre), float(bw_sub), dms,
                           len(dm_list), int(nchan), int(nint), ctypes.byref(opts) if opts is not None else None)
    _check(rc)
    return h.value


def cdmt_plan(nsub, nsamp, f_centre, bw_sub, dm_list, nchan, nint):
    return cdmt_plan_ex(nsub, nsamp, f_centre, bw_sub, dm_list, nchan, nint, None)


def cdmt_plan_info(plan) -> dict:
    info = cdmt_info()
    _check(_lib.cdmt_plan_info(plan, ctypes.byref(info)), plan)
    return {name: (list(getattr(info, name)) if name == "reserved" else getattr(info, name))
            for name, _ in cdmt_info._fields_ if name != "reserved"}


def cdmt_plan_group(plan, g: int) -> dict:
    """Layout of DM group g (cdmt_opts.dm_groups): first DM, DM count, overlap nd_g,
    input offset in samples and the segments its DM stage runs on."""
    first, n = ctypes.c_int(), ctypes.c_int()
    nd, off, nseg = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.cdmt_plan_group(plan, g, ctypes.byref(first), ctypes.byref(n), ctypes.byref(nd), ctypes.byref(off),
                                ctypes.byref(nseg)), plan)
    return {"dm_first": first.value, "ndm": n.value, "nd": nd.value, "offset": off.value, "nseg": nseg.value,
            "nbin": cdmt_plan_group_nbin(plan, g)}


def cdmt_plan_group_nbin(plan, g: int) -> int:
    """Forward FFT length N_g of DM group g (cdmt_opts.group_nbin)."""
    nbin = ctypes.c_int64()
    _check(_lib.cdmt_plan_group_nbin(plan, g, ctypes.byref(nbin)), plan)
    return nbin.value


def cdmt_selftest_wait(limit_ms: float, arrive: bool = False) -> tuple[bool, float]:
    """The tensor-core kernels' bounded mbarrier wait on a barrier nothing arrives on
    (arrive: one arrival first).  Returns (gave_up, waited_ms)."""
    g, w = ctypes.c_int(), ctypes.c_double()
    _check(_lib.cdmt_selftest_wait(limit_ms, 1 if arrive else 0, ctypes.byref(g), ctypes.byref(w)), None)
    return bool(g.value), w.value


def cdmt_inject_timeout(plan) -> None:
    """Mark the plan's device status as a tensor-core wait that gave up (host-side injection)."""
    _check(_lib.cdmt_inject_timeout(plan), plan)


def cdmt_execute(plan, d_in: int, d_out: int, d_scale: int = 0, stream: int = 0):
    _check(_lib.cdmt_execute(plan, d_in, d_out, d_scale or None, stream or None), plan)


def cdmt_execute_host(plan, h_in: int, h_out: int, h_scale: int = 0, stream: int = 0):
    _check(_lib.cdmt_execute_host(plan, h_in, h_out, h_scale or None, stream or None), plan)


def cdmt_destroy(plan):
    _check(_lib.cdmt_destroy(plan))


def cdmt_execute_static(nsub, nsamp, f_centre, bw_sub, dm_first, dm_step, ndm, nchan, nint, nbin, nd,
                        d_in: int, d_out: int, stream: int = 0):
    """The allocation-free entry point: filterbank of one block for the DMs
    dm_first + i dm_step, using the library's fixed device scratch array."""
    _check(_lib.cdmt_execute_static(int(nsub), int(nsamp), float(f_centre), float(bw_sub), float(dm_first),
                                    float(dm_step), int(ndm), int(nchan), int(nint), int(nbin), int(nd),
                                    d_in, d_out, stream or None))


def cdmt_batch_last_error(batch=None) -> str:
    return _lib.cdmt_batch_last_error(batch).decode()


def _bcheck(rc: int, batch=None):
    if rc != CDMT_OK:
        raise CdmtError(rc, f"{cdmt_strerror(rc)}: {cdmt_batch_last_error(batch)}")


def cdmt_batch_create(beams, opts: cdmt_batch_opts | None = None, stream: int = 0):
    arr = (cdmt_beam * len(beams))(*beams)
    h = ctypes.c_void_p()
    _bcheck(_lib.cdmt_batch_create(ctypes.byref(h), len(beams), arr, ctypes.byref(opts) if opts else None,
                                   stream or None))
    return h.value


def cdmt_batch_info(batch, beam: int) -> cdmt_batch_beam_info:
    info = cdmt_batch_beam_info()
    _bcheck(_lib.cdmt_batch_info(batch, beam, ctypes.byref(info)), batch)
    return info


def cdmt_batch_run_round(batch, r: int, stream: int = 0):
    _bcheck(_lib.cdmt_batch_run_round(batch, r, stream or None), batch)


def cdmt_batch_run(batch, stream: int = 0):
    _bcheck(_lib.cdmt_batch_run(batch, stream or None), batch)


def cdmt_batch_copy_out(batch, beam: int, dst: int, stream: int = 0):
    _bcheck(_lib.cdmt_batch_copy_out(batch, beam, dst, stream or None), batch)


def cdmt_batch_status(batch):
    _bcheck(_lib.cdmt_batch_status(batch), batch)


def cdmt_batch_destroy(batch):
    _bcheck(_lib.cdmt_batch_destroy(batch))


class Batch:
    """Owning wrapper of a batch of beams.  beams: list of dicts with nsub, nsamp,
    f_centre, bw_sub, dm_first, dm_step, ndm, nchan, nint and d_in (device
    pointer, kept valid by the caller)."""

    def __init__(self, beams, *, out_budget=0, autotune=False, tune_cache=None, stream=0):
        bs = [cdmt_beam(int(b["nsub"]), int(b["ndm"]), int(b["nsamp"]), float(b["f_centre"]), float(b["bw_sub"]),
                        float(b["dm_first"]), float(b["dm_step"]), int(b["nchan"]), int(b["nint"]), int(b["d_in"]))
              for b in beams]
        o = cdmt_batch_opts()
        o.out_budget = int(out_budget)
        o.autotune = 1 if autotune else 0
        self._cache = tune_cache.encode() if tune_cache else None
        o.tune_cache = self._cache
        self.handle = cdmt_batch_create(bs, o, stream)
        self.nbeam = len(bs)
        self.infos = [cdmt_batch_info(self.handle, i) for i in range(self.nbeam)]
        self.nround = self.infos[0].nround

    def run_round(self, r, stream=0):
        cdmt_batch_run_round(self.handle, r, stream)

    def run(self, stream=0):
        cdmt_batch_run(self.handle, stream)

    def status(self):
        cdmt_batch_status(self.handle)

    def round_output(self, beam, stream=None):
        """The beam's round output as a new CUDA tensor [ndm][nsub*nchan][out_row_stride]."""
        import torch
        inf = self.infos[beam]
        shape = (inf.plan.ndm, inf.plan.nsub * inf.plan.nchan, inf.out_row_stride)
        t = torch.empty(shape, dtype=torch.float32, device="cuda")
        st = (stream or torch.cuda.current_stream()).cuda_stream
        cdmt_batch_copy_out(self.handle, beam, t.data_ptr(), st)
        return t

    def close(self):
        if getattr(self, "handle", None):
            cdmt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cdmt_server_last_error(server=None) -> str:
    return _lib.cdmt_server_last_error(server).decode()


def _scheck(rc: int, server=None):
    if rc != CDMT_OK:
        raise CdmtError(rc, f"{cdmt_strerror(rc)}: {cdmt_server_last_error(server)}")


def cdmt_server_create(opts: cdmt_server_opts | None = None):
    h = ctypes.c_void_p()
    _scheck(_lib.cdmt_server_create(ctypes.byref(h), ctypes.byref(opts) if opts else None))
    return h.value


def cdmt_server_destroy(server):
    _scheck(_lib.cdmt_server_destroy(server))


def cdmt_server_save_beam(server, beam: int):
    """Checkpoint of a beam's stream (its overlap tail and counters) as a numpy uint8 array."""
    import numpy as np
    n = ctypes.c_int64()
    _scheck(_lib.cdmt_server_save_beam(server, beam, None, ctypes.byref(n)), server)
    buf = np.empty(n.value, dtype=np.uint8)
    _scheck(_lib.cdmt_server_save_beam(server, beam, buf.ctypes.data, ctypes.byref(n)), server)
    return buf[:n.value]


def cdmt_server_restore_beam(server, beam: int, ckpt) -> None:
    """Continue a beam's stream from a checkpoint of cdmt_server_save_beam."""
    import numpy as np
    buf = np.ascontiguousarray(ckpt, dtype=np.uint8)
    _scheck(_lib.cdmt_server_restore_beam(server, beam, buf.ctypes.data, buf.size), server)


def cdmt_server_add_beam(server, desc: cdmt_stream_desc) -> int:
    b = ctypes.c_int()
    _scheck(_lib.cdmt_server_add_beam(server, ctypes.byref(desc), ctypes.byref(b)), server)
    return b.value


def cdmt_server_submit(server, beam: int, block: int, scale: int = 0) -> int:
    r = ctypes.c_int64()
    _scheck(_lib.cdmt_server_submit(server, beam, block, scale or None, ctypes.byref(r)), server)
    return r.value


def cdmt_server_wait(server, request: int, timeout_s: float = 60.0) -> cdmt_block_result:
    res = cdmt_block_result()
    _scheck(_lib.cdmt_server_wait(server, request, timeout_s, ctypes.byref(res)), server)
    return res


def cdmt_server_release(server, request: int):
    _scheck(_lib.cdmt_server_release(server, request), server)


def cdmt_server_get_stats(server) -> cdmt_server_stats:
    st = cdmt_server_stats()
    _scheck(_lib.cdmt_server_get_stats(server, ctypes.byref(st)), server)
    return st


def cdmt_server_reset_stats(server):
    _scheck(_lib.cdmt_server_reset_stats(server), server)


class Server:
    """Owning wrapper of a streaming server."""

    def __init__(self, hbm_budget=0, max_slots=0):
        o = cdmt_server_opts()
        o.hbm_budget, o.max_slots = int(hbm_budget), int(max_slots)
        self.handle = cdmt_server_create(o)

    def add_beam(self, nsub, block_len, f_centre, bw_sub, dm_first, dm_step, ndm, nchan, nint,
                 precision=CDMT_PREC_FP16, in_dtype=CDMT_IN_C64, nbin=0, dm_tile=0, out_dtype=CDMT_OUT_F32,
                 sk_nsigma=0.0) -> int:
        d = cdmt_stream_desc(int(nsub), int(ndm), int(block_len), float(f_centre), float(bw_sub), float(dm_first),
                             float(dm_step), int(nchan), int(nint), int(precision), int(in_dtype), int(nbin),
                             int(dm_tile), int(out_dtype), float(sk_nsigma))
        return cdmt_server_add_beam(self.handle, d)

    def submit(self, beam, block_ptr, scale_ptr=0) -> int:
        return cdmt_server_submit(self.handle, beam, block_ptr, scale_ptr)

    def wait(self, request, timeout_s=60.0):
        return cdmt_server_wait(self.handle, request, timeout_s)

    def release(self, request):
        cdmt_server_release(self.handle, request)

    def stats(self):
        return cdmt_server_get_stats(self.handle)

    def save_beam(self, beam):
        return cdmt_server_save_beam(self.handle, beam)

    def restore_beam(self, beam, ckpt):
        cdmt_server_restore_beam(self.handle, beam, ckpt)

    @staticmethod
    def block_view(res: cdmt_block_result, ndm: int, rows: int):
        """Zero-copy torch view [ndm][rows][samples] of a finished block's output slot (valid until release)."""
        import torch

        class _Slot:
            __cuda_array_interface__ = {"shape": (ndm, rows, res.row_stride), "typestr": "<f4",
                                        "data": (res.d_out, False), "version": 3, "strides": None}
        return torch.as_tensor(_Slot(), device="cuda")[:, :, :res.samples]

    @staticmethod
    def block_u8_view(res: cdmt_block_result, ndm: int, rows: int):
        """Zero-copy torch views of an 8-bit block (valid until release): codes [ndm][samples][rows]
        (spectra in decreasing frequency), statistics [ndm][rows][2] (mean, sigma) and
        spectral-kurtosis flags [ndm][rows]."""
        import torch
        if not res.d_u8:
            raise CdmtError(CDMT_EINVAL, "the block has no 8-bit output (float32 beam)")

        def view(ptr, shape, typestr):
            class _A:
                __cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3,
                                            "strides": None}
            return torch.as_tensor(_A(), device="cuda")
        return (view(res.d_u8, (ndm, res.samples, rows), "|u1"), view(res.d_stats, (ndm, rows, 2), "<f4"),
                view(res.d_flags, (ndm, rows), "|u1"))

    def reset_stats(self):
        cdmt_server_reset_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            cdmt_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cdmt_device_status(plan):
    """Raise CdmtError(CDMT_ETIMEOUT) if a tensor-core wait of the plan gave up."""
    _check(_lib.cdmt_device_status(plan), plan)


def cdmt_set_timing(plan, on: bool):
    _check(_lib.cdmt_set_timing(plan, 1 if on else 0), plan)


def cdmt_stage_times(plan):
    """((forward_ms, dedisperse_ms), (forward_launches, dedisperse_launches))
    summed since the previous call."""
    ms = (ctypes.c_double * 2)()
    n = (ctypes.c_int64 * 2)()
    _check(_lib.cdmt_stage_times(plan, ms, n), plan)
    return (ms[0], ms[1]), (n[0], n[1])


def cdmt_execute_host_u8_ex(plan, h_in: int, h_scale: int, h_u8: int, stream: int = 0) -> int:
    """8-bit codes of every block to host memory (Algorithm 1's redigitize + copy to host);
    h_scale: host nsub floats for int8 input (0 for complex64).  Returns the segments per block."""
    n = ctypes.c_int64()
    _check(_lib.cdmt_execute_host_u8_ex(plan, h_in, h_scale or None, h_u8, ctypes.byref(n), stream or None), plan)
    return n.value


def cdmt_execute_host_u8(plan, h_in: int, h_u8: int, stream: int = 0, h_scale: int = 0) -> int:
    """As cdmt_execute_host_u8_ex (h_scale for int8 input)."""
    n = ctypes.c_int64()
    _check(_lib.cdmt_execute_host_u8_ex(plan, h_in, h_scale or None, h_u8, ctypes.byref(n), stream or None), plan)
    return n.value


def cdmt_redigitise(plan, d_fb: int, d_u8: int, d_stats: int = 0, stream: int = 0):
    _check(_lib.cdmt_redigitise(plan, d_fb, d_u8, d_stats or None, stream or None), plan)


def cdmt_redigitise_sk(plan, d_fb: int, d_u8: int, d_stats: int = 0, sk_nsigma: float = 0.0, d_flags: int = 0,
                       stream: int = 0):
    _check(_lib.cdmt_redigitise_sk(plan, d_fb, d_u8, d_stats or None, float(sk_nsigma), d_flags or None,
                                   stream or None), plan)


REDIG_LEVELS = 16.0


def cdmt_incoherent_info(plan, ddm_lo: float, ddm_step: float, nk: int, delays: bool = False):
    """(nt_out, shifts int32 [ndm][nk][rows] or None) of the fine-trial grid."""
    n = ctypes.c_int64()
    tab = None
    ptr = None
    if delays:
        import numpy as np
        info = cdmt_plan_info(plan)
        tab = np.empty((info["ndm"], nk, info["nsub"] * info["nchan"]), dtype=np.int32)
        ptr = tab.ctypes.data
    _check(_lib.cdmt_incoherent_info(plan, ddm_lo, ddm_step, nk, ctypes.byref(n), ptr), plan)
    return n.value, tab


def cdmt_incoherent(plan, d_fb: int, ddm_lo: float, ddm_step: float, nk: int, d_out: int, stream: int = 0):
    _check(_lib.cdmt_incoherent(plan, d_fb, ddm_lo, ddm_step, nk, d_out, stream or None), plan)


class Plan:
    """Owning wrapper of a cdmt plan."""

    def __init__(self, nsub, nsamp, f_centre, bw_sub, dm_list, nchan, nint, *, nbin=0, nd=-1, dm_tile=0,
                 seg_chunk=0, mem_budget=0, precision=CDMT_PREC_FP32, in_dtype=CDMT_IN_C64, chirp=0, host_block=0,
                 sk_nsigma=0.0, dm_groups=0, group_nbin=0):
        o = cdmt_opts()
        o.nbin, o.nd, o.dm_tile, o.seg_chunk, o.mem_budget = nbin, nd, dm_tile, seg_chunk, mem_budget
        o.precision, o.in_dtype, o.chirp, o.host_block, o.sk_nsigma = precision, in_dtype, chirp, host_block, sk_nsigma
        o.dm_groups, o.group_nbin = dm_groups, group_nbin
        self.handle = cdmt_plan_ex(nsub, nsamp, f_centre, bw_sub, list(dm_list), nchan, nint, o)
        self.info = cdmt_plan_info(self.handle)

    def execute(self, d_in: int, d_out: int, d_scale: int = 0, stream: int = 0):
        cdmt_execute(self.handle, d_in, d_out, d_scale, stream)

    def execute_host(self, h_in: int, h_out: int, h_scale: int = 0, stream: int = 0):
        cdmt_execute_host(self.handle, h_in, h_out, h_scale, stream)

    def execute_host_u8(self, h_in: int, h_u8: int, stream: int = 0, h_scale: int = 0) -> int:
        """8-bit codes [ndm][nout][nsub*nchan] to host memory (h_scale: host nsub floats for int8
        input); returns the segments per block."""
        return cdmt_execute_host_u8(self.handle, h_in, h_u8, stream, h_scale)

    def device_status(self):
        cdmt_device_status(self.handle)

    def groups(self) -> list[dict]:
        """Layout of the plan's DM groups: dm_first, ndm, nd, offset (input samples), nseg, nbin."""
        return [cdmt_plan_group(self.handle, g) for g in range(self.info["dm_groups"])]

    def out_shape(self):
        i = self.info
        return (i["ndm"], i["nsub"] * i["nchan"], i["nout"])

    def incoherent(self, fb, ddm_lo=-0.5, ddm_step=0.002, nk=500, out=None, stream=None):
        """Incoherent dedispersion of the filterbank fb (device tensor of out_shape()) over
        nk fine trials around every coherent DM: float32 [ndm][nk][nt_out]."""
        import torch
        nt_out, _ = cdmt_incoherent_info(self.handle, ddm_lo, ddm_step, nk)
        if out is None:
            out = torch.empty((self.info["ndm"], nk, nt_out), dtype=torch.float32, device=fb.device)
        assert fb.is_contiguous() and tuple(fb.shape) == self.out_shape() and out.is_contiguous()
        st = torch.cuda.current_stream(fb.device).cuda_stream if stream is None else stream
        cdmt_incoherent(self.handle, fb.data_ptr(), ddm_lo, ddm_step, nk, out.data_ptr(), st)
        return out

    def redigitise(self, fb, out=None, stats=None, stream=None, sk_nsigma=0.0, flags=None):
        """8-bit codes uint8 [ndm][nout][nsub*nchan] (decreasing frequency) of the
        filterbank fb (a device tensor of out_shape()); stats, if given, receives
        float32 [ndm][nsub*nchan][2] (mean, sigma).  sk_nsigma > 0 flags rows by
        spectral kurtosis (codes 128; flags, if given, uint8 [ndm][nsub*nchan])."""
        import torch
        ndm, rows, nout = self.out_shape()
        assert tuple(fb.shape) == (ndm, rows, nout) and fb.dtype == torch.float32 and fb.is_contiguous()
        if out is None:
            out = torch.empty((ndm, nout, rows), dtype=torch.uint8, device=fb.device)
        st = torch.cuda.current_stream(fb.device).cuda_stream if stream is None else stream
        cdmt_redigitise_sk(self.handle, fb.data_ptr(), out.data_ptr(), stats.data_ptr() if stats is not None else 0,
                           sk_nsigma, flags.data_ptr() if flags is not None else 0, st)
        return out

    def close(self):
        if getattr(self, "handle", None):
            cdmt_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run(plan: Plan, x, out=None, stream=None, scale=None):
    """Convenience for torch CUDA tensors: x float32 [nsub][nsamp][4] on the
    plan's device (int8 [nsub][nsamp][4] with scale float32 [nsub] for a
    CDMT_IN_I8 plan), out float32 [ndm][nsub*nchan][nout] (allocated if None).
    Enqueues on `stream` (default: torch's current stream) and returns out."""
    import torch
    i8 = plan.info["in_dtype"] == CDMT_IN_I8
    want = torch.int8 if i8 else torch.float32
    if not (x.is_cuda and x.dtype == want and x.is_contiguous()):
        raise ValueError(f"x must be a contiguous {want} CUDA tensor [nsub][nsamp][4]")
    if i8 and (scale is None or not (scale.is_cuda and scale.dtype == torch.float32 and scale.numel() == x.shape[0])):
        raise ValueError("an int8 plan needs scale, a float32 CUDA tensor of nsub values")
    i = plan.info
    if tuple(x.shape) != (i["nsub"], i["nsamp"], 4):
        raise ValueError(f"x has shape {tuple(x.shape)}, plan wants {(i['nsub'], i['nsamp'], 4)}")
    if out is None:
        out = torch.empty(plan.out_shape(), dtype=torch.float32, device=x.device)
    if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and tuple(out.shape) == plan.out_shape()):
        raise ValueError("out must be a contiguous float32 CUDA tensor of the plan's output shape")
    st = (stream or torch.cuda.current_stream(x.device)).cuda_stream
    plan.execute(x.data_ptr(), out.data_ptr(), scale.data_ptr() if i8 else 0, st)
    return out
