// cdmt_execute_static: the whole filterbank of one input block without any
// device-memory allocation, for callers that must not call cudaMalloc.
//
// Who needs it: a caller whose device memory belongs to another framework's
// pool (so a cudaMalloc here would compete with, or fail under, that pool), or
// a real-time loop that cannot afford the device-wide synchronisation and
// latency of cudaMalloc / cudaFree between blocks.  Such a caller still owns
// and passes the input and the output; every other byte this call touches
// (twiddle tables, chirp-phase words, the forward spectrum of a chunk of
// segments) lives in one file-scope __device__ array of
// CDMT_STATIC_SCRATCH_BYTES, which the CUDA runtime reserves on each GPU that
// loads this part of the library and keeps until the process exits.
//
// The computation is the same as cdmt_plan + cdmt_execute in the FP32 form with
// an evenly spaced DM list (the same arithmetic, bit for bit; the forward stage
// runs as two launches, which need no work queue, and the scratch lives in a
// different place).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/cdmt.h"
#include "cdmt_internal.h"

namespace cdmt {

void set_thread_error(const char *msg);

namespace {

__device__ __align__(256) unsigned char g_static_scratch[CDMT_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
void *g_scratch_addr[kMaxDevices];  // device address of g_static_scratch, per device
std::mutex g_scratch_mu;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_thread_error(buf);
    return code;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace
}  // namespace cdmt

using namespace cdmt;

extern "C" int cdmt_execute_static(int nsub, int64_t nsamp, double f_centre_mhz, double bw_sub_mhz,
                                   double dm_first, double dm_step, int ndm, int nchan, int nint, int64_t nbin,
                                   int64_t nd, const void *d_in, float *d_out, void *cuda_stream)
{
    // ---- arguments (same rules as cdmt_plan_ex)
    if (nsub < 1 || ndm < 1 || nint < 1) return fail(CDMT_EINVAL, "need nsub, ndm, nint >= 1");
    if (!(bw_sub_mhz > 0) || !std::isfinite(bw_sub_mhz)) return fail(CDMT_EINVAL, "bw_sub must be > 0");
    if (!std::isfinite(dm_first) || !std::isfinite(dm_step)) return fail(CDMT_EINVAL, "DMs must be finite");
    if (!is_pow2(nchan) || nchan < 2 || nchan > 32) return fail(CDMT_EINVAL, "nchan must be a power of two in 2..32");
    const double band_lo = f_centre_mhz - 0.5 * nsub * bw_sub_mhz;
    if (!(band_lo > 0)) return fail(CDMT_EINVAL, "lowest frequency %.6g MHz must be > 0", band_lo);
    if (!is_pow2(nbin) || nbin % nchan) return fail(CDMT_EINVAL, "nbin must be a power of two divisible by nchan");
    const int64_t m = nbin / nchan;
    if (m < 512 || m > 8192) return fail(CDMT_ENOTSUP, "M_bin = %lld outside 512..8192", (long long)m);
    if (nsamp < nbin) return fail(CDMT_EINVAL, "nsamp (%lld) < nbin (%lld)", (long long)nsamp, (long long)nbin);
    if (!d_in || !d_out) return fail(CDMT_EINVAL, "NULL input or output pointer");
    if (reinterpret_cast<uintptr_t>(d_in) % 16) return fail(CDMT_EINVAL, "input must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(d_out) % 4) return fail(CDMT_EINVAL, "output must be 4-byte aligned");
    if (nd < 0) {   // the planner's overlap rule (Sec. 2) for the largest |DM| of the list
        const double dmax = std::fmax(std::fabs(dm_first), std::fabs(dm_first + (ndm - 1) * dm_step));
        nd = overlap_for(nsub, f_centre_mhz, bw_sub_mhz, dmax, nchan, nint, nbin);
        if (nd < 0) return fail(CDMT_EINVAL, "the overlap for DM %.6g does not fit M=%lld", dmax, (long long)m);
    }
    if (nd % 2 || nd >= m || (m - nd) % nint)
        return fail(CDMT_EINVAL, "overlap nd=%lld invalid for M=%lld, nint=%d", (long long)nd, (long long)m, nint);
    const int r = (int)(m / 256);
    const int64_t nvalid = nbin - nd * nchan;
    const int64_t nseg = (nsamp - nbin) / nvalid + 1;
    const int64_t seglen = (m - nd) / nint;
    const int64_t nout = nseg * seglen;

    // ---- scratch map inside the static array; refuse what does not fit
    const size_t ntw = (size_t)15 * (16 * r + r);
    const size_t off_twn = 0;
    const size_t off_twf = align256(off_twn + sizeof(float2) * (size_t)nbin);
    const size_t off_twi = align256(off_twf + sizeof(float2) * ntw);
    const size_t off_nco = align256(off_twi + sizeof(float2) * ntw);
    const size_t off_spec = align256(off_nco + sizeof(uint2) * (size_t)nsub * (size_t)nbin);
    const size_t per_seg = sizeof(float4) * (size_t)nsub * (size_t)nbin;
    if (off_spec + per_seg > (size_t)CDMT_STATIC_SCRATCH_BYTES)
        return fail(CDMT_EBUDGET,
                    "nsub=%d, nbin=%lld need %zu bytes of scratch for one segment; the static scratch holds %zu "
                    "(about 24 * nsub * nbin bytes are needed)",
                    nsub, (long long)nbin, off_spec + per_seg, (size_t)CDMT_STATIC_SCRATCH_BYTES);
    const int64_t kc_max = std::min<int64_t>(nseg, (int64_t)(((size_t)CDMT_STATIC_SCRATCH_BYTES - off_spec) / per_seg));

    // ---- once per device: the device address of the static array
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(CDMT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(CDMT_EINVAL, "device %d out of range", dev);
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p) return fail(CDMT_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_scratch_addr[dev] = p;
        }
        base = static_cast<unsigned char *>(g_scratch_addr[dev]);
    }
    e = fp32_prepare(r);
    if (e != cudaSuccess) return fail(CDMT_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));

    // ---- tables (every byte read later is written here first: nothing needs clearing)
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    float2 *twn = reinterpret_cast<float2 *>(base + off_twn);
    float2 *twf = reinterpret_cast<float2 *>(base + off_twf);
    float2 *twi = reinterpret_cast<float2 *>(base + off_twi);
    uint2 *nco = reinterpret_cast<uint2 *>(base + off_nco);
    float4 *spec = reinterpret_cast<float4 *>(base + off_spec);
    e = enqueue_fp32_tables(twn, twf, twi, nbin, r, st);
    if (e == cudaSuccess)
        e = enqueue_nco_table(nco, nullptr, dm_first, dm_step, f_centre_mhz, bw_sub_mhz, nsub, nchan, nbin, 1, 0,
                              CDMT_CHIRP_CHANNEL, st);
    if (e != cudaSuccess) return fail(CDMT_ECUDA, "table kernels: %s", cudaGetErrorString(e));

    // ---- segment chunks: forward stage into the scratch spectrum, then the DM stage
    for (int64_t k0 = 0; k0 < nseg; k0 += kc_max) {
        const int kc = (int)std::min<int64_t>(kc_max, nseg - k0);
        ForwardArgs fa{};
        fa.in = static_cast<const float4 *>(d_in);
        fa.spec = spec;
        fa.tw_a = twf;
        fa.tw_b = twf + 15 * 16 * r;
        fa.tw_n = twn;
        fa.nsamp = nsamp;
        fa.nvalid = nvalid;
        fa.nbin = nbin;
        fa.k0 = k0;
        fa.nchan = nchan;
        fa.kc = kc;
        fa.nsub = nsub;
        fa.r = r;
        e = fp32_forward(fa, st);
        if (e != cudaSuccess) return fail(CDMT_ECUDA, "forward stage: %s", cudaGetErrorString(e));
        DedispArgs da{};
        da.spec = spec;
        da.nco = nco;
        da.ktab = nullptr;
        da.dm_list = nullptr;
        da.tw_a = twi;
        da.tw_b = twi + 15 * 16 * r;
        da.out = d_out;
        da.k0 = k0;
        da.nout = nout;
        da.nsub = nsub;
        da.kc = kc;
        da.nchan = nchan;
        da.ndm = ndm;
        da.dm_tile = ndm;
        da.nd = (int)nd;
        da.nint = nint;
        da.r = r;
        da.uniform = true;
        da.scale = (float)(1.0 / ((double)nbin * (double)m));
        e = fp32_dedisperse(da, st);
        if (e != cudaSuccess) return fail(CDMT_ECUDA, "DM stage: %s", cudaGetErrorString(e));
    }
    return CDMT_OK;
}
