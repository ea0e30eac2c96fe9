// Host side of the C ABI declared in include/cdmt.h: validation, planning
// (Sec. 2 overlap rule, Sec. 3 fixed N_bin / n_d), FP64 table construction on
// the device (Algorithm 1: "compute transfer function for DM[idm]"), and the
// execute paths.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/cdmt.h"
#include "cdmt_internal.h"
#include "cdmt_plan_impl.h"

using namespace cdmt;

namespace {

constexpr double kD = 4.148808e3;  // MHz^2 pc^-1 cm^3 s

thread_local std::string g_thread_error;

}  // namespace

namespace {

int fail(cdmt_plan_s *p, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (p) p->last_error = buf;
    else g_thread_error = buf;
    return code;
}

#define CK(p, call)                                                                                       \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail(p, e_ == cudaErrorMemoryAllocation ? CDMT_ENOMEM : CDMT_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                               \
    } while (0)

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Eq. 2
double sweep(double lo, double hi, double dm) { return kD * dm * (1.0 / (lo * lo) - 1.0 / (hi * hi)); }

// Overlap n_d of Sec. 2 for the lowest channel of the band at the largest |DM|,
// rounded up to an even number with (M - n_d) % nint == 0.  -1 if none < M.
int64_t overlap_rule(const cdmt_plan_s &p, int64_t nbin)
{
    double dmax = 0;
    for (double d : p.dms) dmax = std::max(dmax, std::fabs(d));
    const double band_lo = p.f_centre - 0.5 * p.nsub * p.bw;
    // the overlap holds the chirp of the lowest channel, or of the lowest subband
    // when one transfer function spans the subband
    const double span = p.chirp == CDMT_CHIRP_SUBBAND ? p.bw : p.bw / p.nchan;
    const double td = sweep(band_lo, band_lo + span, dmax);
    const double want = p.bw * 1e6 * td / p.nchan;
    int64_t nd = (int64_t)std::ceil(want);
    nd += nd & 1;
    const int64_t m = nbin / p.nchan;
    while (nd < m && (m - nd) % p.nint) nd += 2;
    return nd < m ? nd : -1;
}

// ---- FP64 table kernels (run once per plan) ---------------------------------

// tw[k] = exp(sign 2 pi i k / n), k < n
__global__ void k_twiddle_line(float2 *tw, int64_t n, int sign)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)n, &s, &c);
    tw[k] = make_float2((float)c, (float)(sign * s));
}

// pass-A twiddles W_M^{t m0} at [m0-1][t] and pass-B twiddles W_M^{16 j0 m1} at [m1-1][j0]
__global__ void k_twiddle_passes(float2 *ta, float2 *tb, int r, int sign)
{
    const int m = 256 * r, t_n = 16 * r;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 15 * t_n + 15 * r; i += gridDim.x * blockDim.x) {
        int64_t p;
        float2 *dst;
        if (i < 15 * t_n) {
            const int m0 = i / t_n + 1, t = i % t_n;
            p = (int64_t)t * m0;
            dst = ta + i;
        } else {
            const int q = i - 15 * t_n, m1 = q / r + 1, j0 = q % r;
            p = 16LL * j0 * m1;
            dst = tb + q;
        }
        double s, c;
        sincospi(2.0 * (double)(p % m) / (double)m, &s, &c);
        *dst = make_float2((float)c, (float)(sign * s));
    }
}

// K = 1e6 D nu^2 / (nu_c^2 (nu_c + nu)) in cycles per unit DM for shifted bin
// i = c M + j of subband s (Eq. 1 per channel; nu = (j - M/2) bw / N).
__device__ __forceinline__ double chirp_k(double f_centre, double bw, int nsub, int nchan, int64_t nbin, int s, int64_t i,
                                          int chirp)
{
    const double nu_s = f_centre + ((double)s - 0.5 * (double)(nsub - 1)) * bw;
    if (chirp == CDMT_CHIRP_SUBBAND) {   // Eq. 1 about the subband centre: bin i at (i - N/2) bw / N
        const double nu = ((double)i - 0.5 * (double)nbin) * bw / (double)nbin;
        return 1e6 * 4.148808e3 * nu * nu / (nu_s * nu_s * (nu_s + nu));
    }
    const int64_t m = nbin / nchan;
    const int c = (int)(i / m);
    const int64_t j = i % m;
    const double nu_c = nu_s - 0.5 * bw + ((double)c + 0.5) * bw / (double)nchan;
    const double nu = ((double)j - 0.5 * (double)m) * bw / (double)nbin;
    return 1e6 * 4.148808e3 * nu * nu / (nu_c * nu_c * (nu_c + nu));
}

// 32-bit fixed-point fraction of x cycles (x * 2^32 rounded, modulo 2^32)
__device__ __forceinline__ uint32_t fix32(double x) { return (uint32_t)(unsigned long long)llrint(x * 4294967296.0); }

// shift != 0 (tensor-core form): the start words also carry a phase ramp of
// shift * j / M cycles on bin j of each channel, which delays the channel's
// backward DFT output by `shift` samples (exact: shift * j * 2^32 / M is an
// integer for M a power of two <= 2^32).
__global__ void k_nco_table(uint2 *nco, const double *dm_tile0, double dm0, double ddm, double f_centre, double bw,
                            int nsub, int nchan, int64_t nbin, int ntile, int shift, int chirp)
{
    const int64_t mbin = nbin / nchan;
    const int64_t total = (int64_t)ntile * nsub * nbin;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q % nbin;
        const int s = (int)((q / nbin) % nsub);
        const int tile = (int)(q / ((int64_t)nbin * nsub));
        const double k = chirp_k(f_centre, bw, nsub, nchan, nbin, s, i, chirp);
        const int lm = 31 - __clz((int)mbin);   // shift * j * 2^32 / M = (shift * j) << (32 - log2 M)
        const uint32_t ramp = shift ? (uint32_t)((i % mbin) * shift) << (32 - lm) : 0u;
        const double first = dm_tile0 ? dm_tile0[tile] : dm0;
        nco[q] = make_uint2(fix32(-first * k) + ramp, fix32(-ddm * k));
    }
}

__global__ void k_k_table(double *kt, double f_centre, double bw, int nsub, int nchan, int64_t nbin, int chirp)
{
    const int64_t total = (int64_t)nsub * nbin;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
        kt[q] = chirp_k(f_centre, bw, nsub, nchan, nbin, (int)(q / nbin), q % nbin, chirp);
}

// 2P x 2P real form of the backward P-point DFT (W = exp(+2 pi i / P)) in the
// K-major canonical layout (SBO 32P B, LBO 128 B): output n = P ro + m (real
// parts, then imaginary parts), input k = 2 j + (re, im).  ab = 0: FP16; ab = 1:
// BF16 hi in the first (2P)^2 elements and the BF16 rounding residue (lo) in the
// next (2P)^2 (16-bit elements).
__global__ void k_tc_bmat(uint16_t *out, int ab, int P)
{
    const int n2 = 4 * P * P;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n2; idx += gridDim.x * blockDim.x) {
        const int n = idx / (2 * P), k = idx % (2 * P);
        const int m = n % P, ro = n / P, j = k >> 1, ri = k & 1;
        double sn, cs;
        sincospi(2.0 * (double)((j * m) % P) / (double)P, &sn, &cs);
        const double v = ro == 0 ? (ri == 0 ? cs : -sn) : (ri == 0 ? sn : cs);
        const int off = (n / 8) * (16 * P) + (k / 8) * 64 + (n % 8) * 8 + (k % 8);
        if (ab == 0) {
            out[off] = __half_as_ushort(__double2half(v));
        } else {
            const __nv_bfloat16 hi = __double2bfloat16(v);
            const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
            out[off] = __bfloat16_as_ushort(hi);
            out[n2 + off] = __bfloat16_as_ushort(lo);
        }
    }
}

// W_M^{j_lo m0} = exp(+2 pi i j_lo m0 / M), m0 < M / 64, for consecutive pairs of
// m0: [m0 / 2][j_lo] = (cos, cos', sin, sin') of m0 = 2i, 2i + 1
__global__ void k_tc_twq(float2 *tw, int mbin)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= mbin / 2) return;
    const int i = idx / 64, jlo = idx % 64;
    double s0, c0, s1, c1;
    sincospi(2.0 * (double)(jlo * (2 * i)) / (double)mbin, &s0, &c0);
    sincospi(2.0 * (double)(jlo * (2 * i + 1)) / (double)mbin, &s1, &c1);
    reinterpret_cast<float4 *>(tw)[idx] = make_float4((float)c0, (float)c1, (float)s0, (float)s1);
}

// Frees a buffer from dalloc and gives its bytes back to the plan's count.
template <class T> void dfree(cdmt_plan_s *p, T *&ptr, size_t count)
{
    if (!ptr) return;
    cudaFree(ptr);
    p->bytes -= (int64_t)(sizeof(T) * count);
    ptr = nullptr;
}

template <class T> int dalloc(cdmt_plan_s *p, T **ptr, size_t count)
{
    size_t b = sizeof(T) * count;
    if (p->mem_budget > 0 && p->bytes + (int64_t)b > p->mem_budget)
        return fail(p, CDMT_EBUDGET, "device memory budget of %lld bytes exceeded (need %lld more)",
                    (long long)p->mem_budget, (long long)b);
    cudaError_t e = cudaMalloc((void **)ptr, b);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(p, CDMT_ENOMEM, "cudaMalloc(%zu): %s", b, cudaGetErrorString(e));
    }
    p->bytes += (int64_t)b;
    return CDMT_OK;
}

void release(cdmt_plan_s *p)
{
    if (!p) return;
    for (auto &g : p->groups) cdmt_destroy(g.plan);
    p->groups.clear();
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    // tw_bf / tw_bi point inside the tw_af / tw_ai allocations
    void *ptrs[] = {p->tw_n, p->tw_af, p->tw_ai, p->nco, p->ktab, p->d_dm, p->spec, p->tc_bmat, p->tc_twq,
                    p->d_status, p->fwd_sync, p->redig_mg, p->tc_bmat64 != p->tc_bmat ? p->tc_bmat64 : nullptr, p->inc_tab,
                    p->d_scale_buf, p->grp_in, p->grp_out, p->grp_u8};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (auto &st : p->stage) {
        if (st.in) cudaFree(st.in);
        if (st.out) cudaFree(st.out);
        if (st.u8) cudaFree(st.u8);
        cudaEvent_t evs[] = {st.in_free, st.in_ready, st.out_ready, st.out_free};
        for (auto ev : evs)
            if (ev) cudaEventDestroy(ev);
    }
    if (p->s_h2d) cudaStreamDestroy(p->s_h2d);
    if (p->s_d2h) cudaStreamDestroy(p->s_d2h);
    for (auto ev : p->ev_pool) cudaEventDestroy(ev);
    for (auto ev : p->ev_marks) cudaEventDestroy(ev);
    cudaGetLastError();  // leave no error of the teardown behind for a later call to pick up
    cudaSetDevice(cur);
}

int mark(cdmt_plan_s *p, cudaStream_t st)
{
    cudaEvent_t ev;
    if (p->ev_pool.empty()) {
        CK(p, cudaEventCreate(&ev));
    } else {
        ev = p->ev_pool.back();
        p->ev_pool.pop_back();
    }
    p->ev_marks.push_back(ev);
    CK(p, cudaEventRecord(ev, st));
    return CDMT_OK;
}

}  // namespace

namespace cdmt {
// Forward stage and DM stage of kc segments of `in` (segment kk at
// in + (in_k0 + kk) * S, subbands in_stride samples apart) into `out`
// (rows out_stride floats apart, segment kk at (out_k0 + kk) * seglen).
// The forward stage of kc segments (segment in_k0 of `in` first) into the plan's spectra.
int enqueue_forward(cdmt_plan_s *p, const void *in, int64_t in_stride, int64_t in_k0, int kc, cudaStream_t st)
{
    const Range range("cdmt forward stage");
    ForwardArgs fa{};
    fa.in = in;
    fa.spec = p->spec;
    fa.tw_a = p->tw_af;
    fa.tw_b = p->tw_bf;
    fa.tw_n = p->tw_n;
    fa.nsamp = in_stride;
    fa.nvalid = p->nvalid;
    fa.nbin = p->nbin;
    fa.k0 = in_k0;
    fa.nchan = p->nchan;
    fa.kc = kc;
    fa.nsub = p->nsub;
    fa.r = p->r;
    fa.i8 = p->in_dtype == CDMT_IN_I8;
    fa.scale = p->scale_dev;
    fa.status = p->d_status;
    fa.sync = p->fwd_sync;
    fa.sync_n = p->fwd_sync_n;
    fa.nsm = p->nsm;
    CK(p, fp32_forward(fa, st));
    return CDMT_OK;
}

// The DM stage of the kc segments in the plan's spectra, for DMs dm_off .. dm_off + dm_cnt - 1
// of every DM tile (dm_cnt 0: all), into out (row stride out_stride floats; segment kk at
// (out_k0 + kk) * seglen; DM j of tile t's range at row block t * dm_cnt + j).
int enqueue_dm(cdmt_plan_s *p, float *out, int64_t out_stride, int64_t out_k0, int kc, int dm_off, int dm_cnt,
               cudaStream_t st)
{
    const Range range("cdmt DM stage");
    if (p->precision != CDMT_PREC_FP32) {
        TcArgs ta{};
        ta.spec = p->spec;
        ta.nco = p->nco;
        ta.ktab = p->ktab;
        ta.dm_list = p->d_dm;
        ta.bmat = p->tc_bmat;
        ta.bmat64 = p->tc_bmat64;
        ta.twq = p->tc_twq;
        ta.lm = p->mbin == 2048 ? 11 : 12;
        ta.out = out;
        ta.status = p->d_status;
        ta.k0 = out_k0;
        ta.nout = out_stride;
        ta.nsub = p->nsub;
        ta.kc = kc;
        ta.nchan = p->nchan;
        ta.ndm = p->ndm;
        ta.dm_tile = p->dm_tile;
        ta.nd = (int)p->nd;
        ta.nint = p->nint;
        ta.ab = p->precision == CDMT_PREC_BF16 ? 1 : 0;
        ta.uniform = p->uniform;
        ta.scale = (float)(1.0 / ((double)p->nbin * (double)p->mbin));
        ta.nsm = p->nsm;
        ta.dm_off = dm_off;
        ta.dm_cnt = dm_cnt;
        ta.tlim = p->out_tlim;
        CK(p, tc_dedisperse(ta, st));
        return CDMT_OK;
    }
    DedispArgs da{};
    da.spec = p->spec;
    da.nco = p->nco;
    da.ktab = p->ktab;
    da.dm_list = p->d_dm;
    da.tw_a = p->tw_ai;
    da.tw_b = p->tw_bi;
    da.out = out;
    da.k0 = out_k0;
    da.nout = out_stride;
    da.nsub = p->nsub;
    da.kc = kc;
    da.nchan = p->nchan;
    da.ndm = p->ndm;
    da.dm_tile = p->dm_tile;
    da.nd = (int)p->nd;
    da.nint = p->nint;
    da.r = p->r;
    da.uniform = p->uniform;
    da.scale = (float)(1.0 / ((double)p->nbin * (double)p->mbin));
    da.dm_off = dm_off;
    da.dm_cnt = dm_cnt;
    da.tlim = p->out_tlim;
    CK(p, fp32_dedisperse(da, st));
    return CDMT_OK;
}

int enqueue_chunk(cdmt_plan_s *p, const void *in, int64_t in_stride, int64_t in_k0, float *out,
                  int64_t out_stride, int64_t out_k0, int kc, cudaStream_t st)
{
    int rc;
    if (p->timing && (rc = mark(p, st)) != CDMT_OK) return rc;
    if ((rc = enqueue_forward(p, in, in_stride, in_k0, kc, st)) != CDMT_OK) return rc;
    if (p->timing && (rc = mark(p, st)) != CDMT_OK) return rc;
    if ((rc = enqueue_dm(p, out, out_stride, out_k0, kc, 0, 0, st)) != CDMT_OK) return rc;
    if (p->timing && (rc = mark(p, st)) != CDMT_OK) return rc;
    return CDMT_OK;
}


// DM groups (cdmt_opts.dm_groups): child plans over contiguous parts of the DM
// list, each with the smallest overlap that holds its own largest |DM| (Sec. 2's
// rule) and whose segments, started (nd - nd_g) * nchan / 2 input samples in,
// still cover the parent's nout: the parent's time axis and length are kept.
// Steps along the overlaps the rule allows (even, (M - nd_g) % nint == 0) end
// at the parent's nd, which covers nout with no offset.
int make_groups(cdmt_plan_s *p, const cdmt_opts &o, const double *dm_list)
{
    const int G = o.dm_groups;
    const int64_t ndm = p->ndm;
    // A group's overlap at channel length m: its own rule at N = nchan m, grown (even, (m - ndg)
    // divisible by nint) until its segments from offset (nd - ndg) nchan / 2 cover nout.  At the
    // plan's own m the whole list's nd always covers; at another m, -1 when that needs more than nd
    // or one segment does not fit the input.
    auto fit = [&](const cdmt_plan_s &part, int64_t m) -> int64_t {
        const int64_t n = m * p->nchan;
        int64_t ndg = overlap_rule(part, n);
        if (ndg < 0 || ndg > p->nd) {
            if (m != p->mbin) return -1;
            ndg = p->nd;
        }
        for (;;) {
            if (ndg > p->nd) return -1;
            const int64_t off = (p->nd - ndg) * p->nchan / 2;
            if (p->nsamp - off >= n) {
                const int64_t nseg = (p->nsamp - off - n) / (n - ndg * p->nchan) + 1;
                if (nseg * ((m - ndg) / p->nint) >= p->nout) return ndg;
            }
            ndg += 2;
            while ((m - ndg) % p->nint) ndg += 2;
        }
    };
    // channel lengths a group may take: the plan's, or (group_nbin) every length its precision runs
    std::vector<int64_t> lengths;
    if (o.group_nbin) {
        for (int64_t m = 512; m <= (p->precision == CDMT_PREC_FP32 ? 8192 : 4096); m *= 2)
            if (p->precision == CDMT_PREC_FP32 || m == 2048 || m == 4096) lengths.push_back(m);
    } else {
        lengths.push_back(p->mbin);
    }
    for (int g = 0; g < G; g++) {
        const int first = (int)(g * ndm / G), count = (int)((g + 1) * ndm / G) - first;
        cdmt_plan_s part;
        part.nsub = p->nsub;
        part.f_centre = p->f_centre;
        part.bw = p->bw;
        part.nchan = p->nchan;
        part.nint = p->nint;
        part.chirp = p->chirp;
        part.dms.assign(dm_list + first, dm_list + first + count);
        // the length with the least nominal FFT work per unit, 10 N log2(M) / S_g (Sec. 5: digifil
        // picks the FFT size per DM); the plan's own length on a tie
        int64_t mg = p->mbin, ndg = fit(part, p->mbin);
        double best = (double)mg * std::log2((double)mg) / (double)(mg - ndg);
        for (int64_t m : lengths) {
            if (m == p->mbin) continue;
            const int64_t nd_m = fit(part, m);
            if (nd_m < 0) continue;
            const double cost = (double)m * std::log2((double)m) / (double)(m - nd_m);
            if (cost < best * (1.0 - 1e-12)) {
                best = cost;
                mg = m;
                ndg = nd_m;
            }
        }
        const int64_t off = (p->nd - ndg) * p->nchan / 2;
        cdmt_opts co = o;
        co.nbin = mg * p->nchan;
        co.nd = ndg;
        co.dm_groups = 0;
        co.mem_budget = o.mem_budget > 0 ? o.mem_budget / G : 0;
        cdmt_plan_s *child = nullptr;
        const int rc = cdmt_plan_ex(&child, p->nsub, p->nsamp - off, p->f_centre, p->bw, dm_list + first, count,
                                    p->nchan, p->nint, &co);
        if (rc != CDMT_OK) {
            p->last_error = g_thread_error;
            return rc;
        }
        const int64_t seglen = (mg - ndg) / p->nint;
        child->out_tlim = p->nout;
        p->groups.push_back({child, first, off, (p->nout + seglen - 1) / seglen});
    }
    p->dm_tile = p->groups.back().plan->dm_tile;
    p->seg_chunk = p->groups.back().plan->seg_chunk;
    p->ntile = 0;
    return CDMT_OK;
}

cudaError_t enqueue_fp32_tables(float2 *tw_n, float2 *tw_af, float2 *tw_ai, int64_t nbin, int r, cudaStream_t st)
{
    const int tn = 16 * r;
    k_twiddle_line<<<(unsigned)((nbin + 255) / 256), 256, 0, st>>>(tw_n, nbin, -1);
    k_twiddle_passes<<<64, 256, 0, st>>>(tw_af, tw_af + 15 * tn, r, -1);
    k_twiddle_passes<<<64, 256, 0, st>>>(tw_ai, tw_ai + 15 * tn, r, +1);
    return cudaGetLastError();
}

cudaError_t enqueue_nco_table(uint2 *nco, const double *d_tile0, double dm0, double ddm, double f_centre, double bw,
                              int nsub, int nchan, int64_t nbin, int ntile, int shift, int chirp, cudaStream_t st)
{
    k_nco_table<<<1024, 256, 0, st>>>(nco, d_tile0, dm0, ddm, f_centre, bw, nsub, nchan, nbin, ntile, shift, chirp);
    return cudaGetLastError();
}

// lets other translation units of the library report an error before a plan exists
void set_thread_error(const char *msg) { g_thread_error = msg; }

int64_t overlap_for(int nsub, double f_centre, double bw, double dm_abs_max, int nchan, int nint, int64_t nbin)
{
    cdmt_plan_s p;
    p.nsub = nsub;
    p.f_centre = f_centre;
    p.bw = bw;
    p.nchan = nchan;
    p.nint = nint;
    p.dms.assign(1, dm_abs_max);
    return overlap_rule(p, nbin);
}
}  // namespace cdmt

extern "C" {

const char *cdmt_strerror(int status)
{
    switch (status) {
    case CDMT_OK: return "success";
    case CDMT_EINVAL: return "invalid argument";
    case CDMT_ENOMEM: return "out of memory";
    case CDMT_ECUDA: return "CUDA error";
    case CDMT_ETIMEOUT: return "device wait timed out";
    case CDMT_EBUDGET: return "memory budget exceeded";
    case CDMT_ENOTSUP: return "unsupported size combination";
    default: return "unknown status";
    }
}

const char *cdmt_last_error(cdmt_plan_t plan)
{
    return plan ? plan->last_error.c_str() : g_thread_error.c_str();
}

int cdmt_plan(cdmt_plan_t *plan, int nsub, int64_t nsamp, double f_centre_mhz, double bw_sub_mhz,
              const double *dm_list, int ndm, int nchan, int nint)
{
    return cdmt_plan_ex(plan, nsub, nsamp, f_centre_mhz, bw_sub_mhz, dm_list, ndm, nchan, nint, nullptr);
}

int cdmt_plan_ex(cdmt_plan_t *plan, int nsub, int64_t nsamp, double f_centre_mhz, double bw_sub_mhz,
                 const double *dm_list, int ndm, int nchan, int nint, const cdmt_opts *opts)
{
    if (!plan) return fail(nullptr, CDMT_EINVAL, "plan pointer is NULL");
    *plan = nullptr;
    cdmt_opts o{};
    if (opts) o = *opts;
    if (nsub < 1) return fail(nullptr, CDMT_EINVAL, "nsub must be >= 1 (got %d)", nsub);
    if (ndm < 1 || !dm_list) return fail(nullptr, CDMT_EINVAL, "need ndm >= 1 and a DM list");
    if (!(bw_sub_mhz > 0) || !std::isfinite(bw_sub_mhz)) return fail(nullptr, CDMT_EINVAL, "bw_sub must be > 0");
    if (!is_pow2(nchan) || nchan < 2 || nchan > 32)
        return fail(nullptr, CDMT_EINVAL, "nchan must be a power of two in 2..32 (got %d)", nchan);
    if (nint < 1) return fail(nullptr, CDMT_EINVAL, "nint must be >= 1 (got %d)", nint);
    for (int i = 0; i < ndm; i++)
        if (!std::isfinite(dm_list[i])) return fail(nullptr, CDMT_EINVAL, "DM %d is not finite", i);
    const double band_lo = f_centre_mhz - 0.5 * nsub * bw_sub_mhz;
    if (!(band_lo > 0)) return fail(nullptr, CDMT_EINVAL, "lowest frequency %.6g MHz must be > 0", band_lo);
    if (o.precision != CDMT_PREC_FP32 && o.precision != CDMT_PREC_FP16 && o.precision != CDMT_PREC_BF16)
        return fail(nullptr, CDMT_ENOTSUP, "precision %d not available", o.precision);
    if (o.in_dtype != CDMT_IN_C64 && o.in_dtype != CDMT_IN_I8)
        return fail(nullptr, CDMT_ENOTSUP, "input dtype %d not available", o.in_dtype);
    if (o.chirp != CDMT_CHIRP_CHANNEL && o.chirp != CDMT_CHIRP_SUBBAND)
        return fail(nullptr, CDMT_EINVAL, "chirp %d is neither per channel nor per subband", o.chirp);
    if (o.dm_groups < 0 || o.dm_groups > ndm)
        return fail(nullptr, CDMT_EINVAL, "dm_groups must be in 0..ndm (got %d)", o.dm_groups);

    auto *p = new cdmt_plan_s();
    cudaGetDevice(&p->device);
    p->nsub = nsub;
    p->nsamp = nsamp;
    p->f_centre = f_centre_mhz;
    p->bw = bw_sub_mhz;
    p->dms.assign(dm_list, dm_list + ndm);
    p->ndm = ndm;
    p->nchan = nchan;
    p->nint = nint;
    p->precision = o.precision;
    p->in_dtype = o.in_dtype;
    p->chirp = o.chirp;
    p->mem_budget = o.mem_budget;
    p->host_block_opt = o.host_block;
    p->sk_nsigma = o.sk_nsigma > 0.0 ? o.sk_nsigma : 0.0;

    // N_bin: explicit, or the largest M in 512..4096 whose overlap wastes <= 1/4
    int64_t nbin = o.nbin;
    if (nbin > 0) {
        if (!is_pow2(nbin) || nbin % nchan) {
            delete p;
            return fail(nullptr, CDMT_EINVAL, "nbin must be a power of two divisible by nchan");
        }
    } else {
        nbin = 0;
        for (int64_t m = 4096; m >= 512; m /= 2) {
            int64_t n = m * nchan;
            if (n > nsamp) continue;
            int64_t nd = o.nd >= 0 ? o.nd : overlap_rule(*p, n);
            if (nd < 0) continue;
            if (!nbin) nbin = n;  // largest that fits at all
            if (nd * 4 <= m) { nbin = n; break; }
        }
        if (!nbin) {
            delete p;
            return fail(nullptr, CDMT_EINVAL, "no FFT length in 512*nchan..4096*nchan fits nsamp=%lld with its overlap",
                        (long long)nsamp);
        }
    }
    p->nbin = nbin;
    p->mbin = nbin / nchan;
    if (p->mbin < 512 || p->mbin > (p->precision == CDMT_PREC_FP32 ? 8192 : 4096)) {
        const long long mb = (long long)p->mbin;
        delete p;
        return fail(nullptr, CDMT_ENOTSUP, "M_bin = %lld outside 512..4096 (512..8192 in the FP32 form)", mb);
    }
    p->r = (int)(p->mbin / 256);
    if (p->precision != CDMT_PREC_FP32 && 32 % nint != 0) {
        delete p;
        return fail(nullptr, CDMT_ENOTSUP, "tensor-core precisions need nint dividing 32 (got %d)", nint);
    }
    if (p->precision != CDMT_PREC_FP32 && p->mbin != 4096 && p->mbin != 2048) {
        const long long mb = (long long)p->mbin;
        delete p;
        return fail(nullptr, CDMT_ENOTSUP, "tensor-core precisions need M_bin = 2048 or 4096 (got %lld)", mb);
    }
    if (nsamp < nbin) {
        delete p;
        return fail(nullptr, CDMT_EINVAL, "nsamp (%lld) < N_bin (%lld)", (long long)nsamp, (long long)nbin);
    }
    p->nd = o.nd >= 0 ? o.nd : overlap_rule(*p, nbin);
    if (p->nd < 0 || p->nd % 2 || p->nd >= p->mbin || (p->mbin - p->nd) % nint) {
        const long long nd = (long long)p->nd, mb = (long long)p->mbin;
        delete p;
        return fail(nullptr, CDMT_EINVAL, "overlap nd=%lld invalid for M=%lld, nint=%d (need even, < M, (M-nd) %% nint == 0)",
                    nd, mb, nint);
    }
    p->nvalid = nbin - p->nd * nchan;
    p->nseg = (nsamp - nbin) / p->nvalid + 1;
    p->seglen = (p->mbin - p->nd) / nint;
    p->nout = p->nseg * p->seglen;

    // DM list spacing
    p->ddm = ndm > 1 ? (dm_list[ndm - 1] - dm_list[0]) / (ndm - 1) : 0.0;
    p->uniform = true;
    for (int i = 0; i < ndm; i++) {
        double want = dm_list[0] + i * p->ddm;
        if (std::fabs(dm_list[i] - want) > 1e-9 * std::max(1.0, std::fabs(dm_list[i]))) p->uniform = false;
    }

    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
    p->nsm = nsm;
    if (o.dm_groups > 1) {
        const int rc = make_groups(p, o, dm_list);
        if (rc != CDMT_OK) {
            release(p);
            delete p;
            return rc;
        }
        *plan = p;
        return CDMT_OK;
    }
    // DM tile: all DMs, unless that leaves too few work items to fill the GPU
    const int64_t items = (int64_t)nsub * p->nseg * nchan;
    const int64_t want_items = 4LL * nsm;
    int tiles = 1;
    if (o.dm_tile > 0) tiles = (ndm + o.dm_tile - 1) / o.dm_tile;
    else if (items < want_items) tiles = (int)std::min<int64_t>(ndm, (want_items + items - 1) / items);
    p->dm_tile = (ndm + tiles - 1) / tiles;
    p->ntile = (ndm + p->dm_tile - 1) / p->dm_tile;

    // workspace chunk: all segments unless the budget / a request says otherwise
    p->seg_chunk = o.seg_chunk > 0 ? std::min<int64_t>(o.seg_chunk, p->nseg) : p->nseg;
    const int64_t spec_bytes_per_seg = (int64_t)nsub * nbin * 16;
    if (o.seg_chunk <= 0 && p->mem_budget > 0) {
        int64_t room = p->mem_budget / 2 / spec_bytes_per_seg;
        p->seg_chunk = std::max<int64_t>(1, std::min<int64_t>(room, p->nseg));
    }

    int rc;
    cudaError_t e = fp32_prepare(p->r);
    if (e == cudaSuccess && p->precision != CDMT_PREC_FP32) e = tc_prepare(p->precision == CDMT_PREC_BF16 ? 1 : 0);
    if (e != cudaSuccess) {
        release(p);
        delete p;
        return fail(nullptr, CDMT_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
    }
#define TRY(x)                          \
    do {                                \
        if ((rc = (x)) != CDMT_OK) {    \
            g_thread_error = p->last_error; \
            release(p);                 \
            delete p;                   \
            return rc;                  \
        }                               \
    } while (0)
    const int tn = 16 * p->r;
    TRY(dalloc(p, &p->tw_n, (size_t)nbin));
    TRY(dalloc(p, &p->tw_af, (size_t)15 * (tn + p->r)));
    TRY(dalloc(p, &p->tw_ai, (size_t)15 * (tn + p->r)));
    p->tw_bf = p->tw_af + 15 * tn;
    p->tw_bi = p->tw_ai + 15 * tn;
    TRY(dalloc(p, &p->d_dm, (size_t)ndm));
    if (p->uniform) TRY(dalloc(p, &p->nco, (size_t)p->ntile * nsub * nbin));
    else TRY(dalloc(p, &p->ktab, (size_t)nsub * nbin));
    TRY(dalloc(p, &p->spec, (size_t)p->seg_chunk * nsub * nbin));
    TRY(dalloc(p, &p->d_status, 1));
    p->fwd_sync_n = 1 + (nsub * p->seg_chunk + 1) / 2;
    TRY(dalloc(p, &p->fwd_sync, (size_t)p->fwd_sync_n));
    if (p->precision != CDMT_PREC_FP32) {
        const int P = (int)(p->mbin / 64), planes = p->precision == CDMT_PREC_BF16 ? 2 : 1;
        TRY(dalloc(p, &p->tc_bmat, (size_t)planes * P * P / 2));   // (2P)^2 halves per plane, 8 per uint4
        if (P != 64) TRY(dalloc(p, &p->tc_bmat64, (size_t)planes * 2048));
        else p->tc_bmat64 = p->tc_bmat;
        TRY(dalloc(p, &p->tc_twq, (size_t)p->mbin));
    }

    std::vector<double> tile0(p->ntile);
    for (int t = 0; t < p->ntile; t++) tile0[t] = dm_list[t * p->dm_tile];
    double *d_tile0 = nullptr;
#define TRYC(x)                                                                            \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) {                                                           \
            fail(nullptr, CDMT_ECUDA, "%s: %s", #x, cudaGetErrorString(e_));               \
            if (d_tile0) cudaFree(d_tile0);                                                \
            release(p);                                                                    \
            delete p;                                                                      \
            return CDMT_ECUDA;                                                             \
        }                                                                                  \
    } while (0)
    TRYC(cudaMemcpy(p->d_dm, dm_list, sizeof(double) * ndm, cudaMemcpyHostToDevice));
    TRYC(cudaMemset(p->d_status, 0, sizeof(int)));
    if (p->precision != CDMT_PREC_FP32) {
        const int ab = p->precision == CDMT_PREC_BF16 ? 1 : 0;
        k_tc_bmat<<<64, 256>>>(reinterpret_cast<uint16_t *>(p->tc_bmat), ab, (int)(p->mbin / 64));
        if (p->tc_bmat64 != p->tc_bmat) k_tc_bmat<<<64, 256>>>(reinterpret_cast<uint16_t *>(p->tc_bmat64), ab, 64);
        k_tc_twq<<<(unsigned)((p->mbin / 2 + 255) / 256), 256>>>(p->tc_twq, (int)p->mbin);
    }
    TRYC(enqueue_fp32_tables(p->tw_n, p->tw_af, p->tw_ai, nbin, p->r, 0));
    if (p->uniform) {
        TRYC(cudaMalloc(&d_tile0, sizeof(double) * p->ntile));
        TRYC(cudaMemcpy(d_tile0, tile0.data(), sizeof(double) * p->ntile, cudaMemcpyHostToDevice));
        TRYC(enqueue_nco_table(p->nco, d_tile0, 0.0, p->ddm, f_centre_mhz, bw_sub_mhz, nsub, nchan, nbin, p->ntile,
                               p->precision != CDMT_PREC_FP32 ? (int)(p->nd / 2) : 0, p->chirp, 0));
    } else {
        k_k_table<<<1024, 256>>>(p->ktab, f_centre_mhz, bw_sub_mhz, nsub, nchan, nbin, p->chirp);
    }
    TRYC(cudaGetLastError());
    TRYC(cudaDeviceSynchronize());
    if (d_tile0) cudaFree(d_tile0);
#undef TRY
#undef TRYC
    *plan = p;
    return CDMT_OK;
}

int cdmt_plan_info(cdmt_plan_t p, cdmt_info *info)
{
    if (!p || !info) return fail(p, CDMT_EINVAL, "NULL plan or info");
    std::memset(info, 0, sizeof *info);
    info->nsamp = p->nsamp;
    info->nbin = p->nbin;
    info->mbin = p->mbin;
    info->nd = p->nd;
    info->nvalid = p->nvalid;
    info->nseg = p->nseg;
    info->nout = p->nout;
    info->seg_chunk = p->seg_chunk;
    info->workspace_bytes = p->bytes;
    info->in_bytes = (int64_t)p->nsub * p->nsamp * (p->in_dtype == CDMT_IN_I8 ? 4 : 16);
    info->out_bytes = (int64_t)p->ndm * p->nsub * p->nchan * p->nout * 4;
    info->units = (double)p->ndm * p->nsub * p->nseg * p->nvalid;
    info->nsub = p->nsub;
    info->nchan = p->nchan;
    info->nint = p->nint;
    info->ndm = p->ndm;
    info->dm_tile = p->dm_tile;
    info->uniform_dm = p->uniform ? 1 : 0;
    info->precision = p->precision;
    info->in_dtype = p->in_dtype;
    info->device = p->device;
    info->dm_groups = p->groups.empty() ? 1 : (int32_t)p->groups.size();
    for (auto &g : p->groups) info->workspace_bytes += g.plan->bytes;
    return CDMT_OK;
}

int cdmt_plan_group(cdmt_plan_t p, int g, int *dm_first, int *ndm, int64_t *nd, int64_t *offset, int64_t *nseg)
{
    if (!p) return fail(nullptr, CDMT_EINVAL, "NULL plan");
    const int ng = p->groups.empty() ? 1 : (int)p->groups.size();
    if (g < 0 || g >= ng) return fail(p, CDMT_EINVAL, "group %d outside 0..%d", g, ng - 1);
    if (p->groups.empty()) {
        if (dm_first) *dm_first = 0;
        if (ndm) *ndm = p->ndm;
        if (nd) *nd = p->nd;
        if (offset) *offset = 0;
        if (nseg) *nseg = p->nseg;
        return CDMT_OK;
    }
    const auto &q = p->groups[g];
    if (dm_first) *dm_first = q.first;
    if (ndm) *ndm = q.plan->ndm;
    if (nd) *nd = q.plan->nd;
    if (offset) *offset = q.off;
    if (nseg) *nseg = q.kneed;
    return CDMT_OK;
}

int cdmt_plan_group_nbin(cdmt_plan_t p, int g, int64_t *nbin)
{
    if (!p || !nbin) return fail(p, CDMT_EINVAL, "NULL plan or nbin");
    const int ng = p->groups.empty() ? 1 : (int)p->groups.size();
    if (g < 0 || g >= ng) return fail(p, CDMT_EINVAL, "group %d outside 0..%d", g, ng - 1);
    *nbin = p->groups.empty() ? p->nbin : p->groups[g].plan->nbin;
    return CDMT_OK;
}

int cdmt_execute(cdmt_plan_t p, const void *d_in, float *d_out, const float *d_scale, void *cuda_stream)
{
    if (!p) return fail(nullptr, CDMT_EINVAL, "NULL plan");
    if (!d_in || !d_out) return fail(p, CDMT_EINVAL, "NULL input or output pointer");
    const bool i8 = p->in_dtype == CDMT_IN_I8;
    if (i8 && !d_scale) return fail(p, CDMT_EINVAL, "int8 input needs the per-subband scales");
    if (reinterpret_cast<uintptr_t>(d_in) % (i8 ? 4 : 16))
        return fail(p, CDMT_EINVAL, "input must be %d-byte aligned", i8 ? 4 : 16);
    p->scale_dev = d_scale;
    if (reinterpret_cast<uintptr_t>(d_out) % 4) return fail(p, CDMT_EINVAL, "output must be 4-byte aligned");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) CK(p, cudaSetDevice(p->device));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int rc = CDMT_OK;
    // DM groups: each child reads the input from its offset on (subbands p->nsamp samples apart)
    // and writes its DMs' rows of the common filterbank, only the segments that cover nout
    const int64_t rows = (int64_t)p->nsub * p->nchan;
    for (auto &g : p->groups) {
        cdmt_plan_s *c = g.plan;
        c->scale_dev = d_scale;
        c->timing = p->timing;
        const void *in = static_cast<const char *>(d_in) + g.off * (i8 ? 4 : 16);
        float *out = d_out + (int64_t)g.first * rows * p->nout;
        for (int64_t k0 = 0; k0 < g.kneed && rc == CDMT_OK; k0 += c->seg_chunk) {
            const int kc = (int)std::min<int64_t>(c->seg_chunk, g.kneed - k0);
            rc = enqueue_chunk(c, in, p->nsamp, k0, out, p->nout, k0, kc, st);
        }
        if (rc != CDMT_OK) {
            p->last_error = c->last_error;
            break;
        }
    }
    for (int64_t k0 = 0; k0 < p->nseg && rc == CDMT_OK && p->groups.empty(); k0 += p->seg_chunk) {
        const int kc = (int)std::min<int64_t>(p->seg_chunk, p->nseg - k0);
        rc = enqueue_chunk(p, d_in, p->nsamp, k0, d_out, p->nout, k0, kc, st);
    }
    if (cur != p->device) cudaSetDevice(cur);
    return rc;
}

namespace {

// Segments per block of the host pipeline: the caller's choice, else by output
// type.  The first block's copy-in and compute are not hidden, and the link to
// the host moves 2D rows of a float32 block faster the longer they are (16 KB
// rows ~170 GB/s, 64 KB ~194 GB/s on GB300): float32 output takes about 4
// blocks, 8-bit output (4x fewer bytes back) about 16.  Every block holds at
// least 16 work items per SM.
int64_t host_block(const cdmt_plan_s *p, bool u8)
{
    int64_t kc;
    if (p->host_block_opt > 0) {
        kc = p->host_block_opt;
    } else {
        const int64_t ntile = (p->ndm + p->dm_tile - 1) / p->dm_tile;
        const int64_t per_seg = std::max<int64_t>(1, ntile * p->nsub * p->nchan);
        const int64_t fill = (16 * std::max(1, p->nsm) + per_seg - 1) / per_seg;
        const int64_t nblk = u8 ? 16 : 4;
        kc = std::max<int64_t>((p->nseg + nblk - 1) / nblk, fill);
    }
    return std::max<int64_t>(1, std::min<int64_t>(kc, std::min<int64_t>(p->seg_chunk, p->nseg)));
}

// Staging buffers (grown when a call needs more: input spans of kc segments,
// out_floats per output slot), events and copy streams of the host pipeline.
int host_setup(cdmt_plan_s *p, int64_t kc, int64_t out_floats, cudaStream_t st)
{
    if (!p->s_h2d) {
        for (auto &sg : p->stage) {
            CK(p, cudaEventCreateWithFlags(&sg.in_free, cudaEventDisableTiming));
            CK(p, cudaEventCreateWithFlags(&sg.in_ready, cudaEventDisableTiming));
            CK(p, cudaEventCreateWithFlags(&sg.out_ready, cudaEventDisableTiming));
            CK(p, cudaEventCreateWithFlags(&sg.out_free, cudaEventDisableTiming));
        }
        CK(p, cudaStreamCreateWithFlags(&p->s_h2d, cudaStreamNonBlocking));
        CK(p, cudaStreamCreateWithFlags(&p->s_d2h, cudaStreamNonBlocking));
    }
    // (the previous call ended with both copy streams drained, so the buffers are idle)
    if (p->host_chunk < kc) {
        for (auto &sg : p->stage) dfree(p, sg.in, (size_t)p->nsub * p->span_max);
        p->host_chunk = 0;
        p->span_max = (kc - 1) * p->nvalid + p->nbin;
        for (auto &sg : p->stage) {
            const int rc = dalloc(p, &sg.in, (size_t)p->nsub * p->span_max);
            if (rc != CDMT_OK) return rc;
        }
        p->host_chunk = kc;
    }
    if (p->host_out_cap < out_floats) {
        for (auto &sg : p->stage) {
            dfree(p, sg.out, (size_t)p->host_out_cap);
            dfree(p, sg.u8, (size_t)p->host_out_cap);
        }
        p->host_out_cap = 0;
        for (auto &sg : p->stage) {
            const int rc = dalloc(p, &sg.out, (size_t)out_floats);
            if (rc != CDMT_OK) return rc;
        }
        p->host_out_cap = out_floats;
    }
    for (auto &sg : p->stage) {
        CK(p, cudaEventRecord(sg.in_free, st));
        CK(p, cudaEventRecord(sg.out_free, st));
    }
    return CDMT_OK;
}

// The host pipeline: per block of segments, H2D of its input span (copy stream),
// the forward and DM stages (st), then D2H of its filterbank (copy stream); with
// u8, the block is redigitised on the device and its codes are copied instead.
// Three input spans and three output slots are in flight.  For float32 output of
// a plan with one DM tile, each block's DM stage runs in up to 4 DM ranges with
// an output slot each, so the copy back of a block starts after a quarter of its
// compute (the first one is the pipeline's fill) while its rows stay long.
// *kc_used receives the segments per block.
int host_pipeline(cdmt_plan_s *p, const void *h_in, const float *h_scale, float *h_out, uint8_t *h_u8,
                  int64_t *kc_used, cudaStream_t st);

// Plans with DM groups from and to host memory: the whole input to the device, the grouped
// execute, and the whole filterbank back, or its 8-bit codes with the whole input as one data
// block (Sec. 3 statistics over all of it).  Copies and compute do not overlap: the groups
// segment the input differently, so there is no common block of segments to pipeline.
int grouped_host(cdmt_plan_s *p, const void *h_in, const float *h_scale, float *h_out, uint8_t *h_u8,
                 int64_t *kc_used, cudaStream_t st)
{
    int rc;
    const bool i8 = p->in_dtype == CDMT_IN_I8;
    if (i8 && !h_scale) return fail(p, CDMT_EINVAL, "int8 input needs the per-subband scales");
    const size_t in_bytes = (size_t)p->nsub * p->nsamp * (i8 ? 4 : 16);
    const size_t fb = (size_t)p->ndm * p->nsub * p->nchan * p->nout;
    if (!p->grp_in && (rc = dalloc(p, &p->grp_in, in_bytes)) != CDMT_OK) return rc;
    if (!p->grp_out && (rc = dalloc(p, &p->grp_out, fb)) != CDMT_OK) return rc;
    if (h_u8 && !p->grp_u8 && (rc = dalloc(p, &p->grp_u8, fb)) != CDMT_OK) return rc;
    CK(p, cudaMemcpyAsync(p->grp_in, h_in, in_bytes, cudaMemcpyHostToDevice, st));
    const float *d_scale = nullptr;
    if (i8) {
        if (!p->d_scale_buf && (rc = dalloc(p, &p->d_scale_buf, (size_t)p->nsub)) != CDMT_OK) return rc;
        CK(p, cudaMemcpyAsync(p->d_scale_buf, h_scale, sizeof(float) * p->nsub, cudaMemcpyHostToDevice, st));
        d_scale = p->d_scale_buf;
    }
    if ((rc = cdmt_execute(p, p->grp_in, p->grp_out, d_scale, st)) != CDMT_OK) return rc;
    if (h_u8) {
        if ((rc = redig_enqueue(p, p->grp_out, p->nout, p->nout, p->grp_u8, nullptr, st, p->sk_nsigma)) != CDMT_OK)
            return rc;
        CK(p, cudaMemcpyAsync(h_u8, p->grp_u8, fb, cudaMemcpyDeviceToHost, st));
    } else {
        CK(p, cudaMemcpyAsync(h_out, p->grp_out, fb * sizeof(float), cudaMemcpyDeviceToHost, st));
    }
    CK(p, cudaStreamSynchronize(st));
    if (kc_used) *kc_used = p->nseg;
    return CDMT_OK;
}

int host_pipeline(cdmt_plan_s *p, const void *h_in, const float *h_scale, float *h_out, uint8_t *h_u8,
                  int64_t *kc_used, cudaStream_t st)
{
    int rc;
    const bool u8 = h_u8 != nullptr;
    const bool i8 = p->in_dtype == CDMT_IN_I8;
    const size_t es = i8 ? 4 : 16;   // bytes per input sample
    if (i8 && !h_scale) return fail(p, CDMT_EINVAL, "int8 input needs the per-subband scales");
    const int64_t kcm = host_block(p, u8);
    const int64_t nrow = (int64_t)p->nsub * p->nchan;
    const int64_t ntile = (p->ndm + p->dm_tile - 1) / p->dm_tile;
    const int nq = (!u8 && ntile == 1) ? (int)std::max<int64_t>(1, std::min<int64_t>(4, p->ndm / 32)) : 1;
    const int qdm = (p->ndm + nq - 1) / nq;   // DMs per range
    if ((rc = host_setup(p, kcm, (int64_t)qdm * nrow * kcm * p->seglen, st)) != CDMT_OK) return rc;
    if (u8)
        for (auto &sg : p->stage)
            if (!sg.u8 && (rc = dalloc(p, &sg.u8, (size_t)p->host_out_cap)) != CDMT_OK) return rc;
    const auto *src = static_cast<const char *>(h_in);
    if (i8) {   // the scales go first on the copy stream, so block 0's copy event covers them
        if (!p->d_scale_buf && (rc = dalloc(p, &p->d_scale_buf, (size_t)p->nsub)) != CDMT_OK) return rc;
        CK(p, cudaMemcpyAsync(p->d_scale_buf, h_scale, sizeof(float) * p->nsub, cudaMemcpyHostToDevice, p->s_h2d));
        p->scale_dev = p->d_scale_buf;
    }
    const int64_t ostride = kcm * p->seglen;   // floats per row of an output slot
    int bi = 0, bo = 0;
    // float32 output chosen by the plan: the first block is a quarter of the others (at least the
    // 16 items per SM of a full GPU), so the pipeline fills after a short copy-in and compute
    int64_t first = kcm;
    if (!u8 && p->host_block_opt <= 0) {
        const int64_t per_seg = std::max<int64_t>(1, ntile * p->nsub * p->nchan);
        const int64_t fill = (16 * std::max(1, p->nsm) + per_seg - 1) / per_seg;
        first = std::max<int64_t>(1, std::min<int64_t>(kcm, std::max<int64_t>(kcm / 4, fill)));
    }
    for (int64_t k0 = 0; k0 < p->nseg; k0 += (k0 == 0 ? first : kcm), bi = (bi + 1) % 3) {
        const Range range("cdmt host block");
        Staging &si = p->stage[bi];
        const int kc = (int)std::min<int64_t>(k0 == 0 ? first : kcm, p->nseg - k0);
        const int64_t span = (kc - 1) * p->nvalid + p->nbin;
        CK(p, cudaStreamWaitEvent(p->s_h2d, si.in_free, 0));
        CK(p, cudaMemcpy2DAsync(si.in, p->span_max * es, src + k0 * p->nvalid * es, p->nsamp * es, span * es,
                                p->nsub, cudaMemcpyHostToDevice, p->s_h2d));
        CK(p, cudaEventRecord(si.in_ready, p->s_h2d));
        CK(p, cudaStreamWaitEvent(st, si.in_ready, 0));
        if ((rc = enqueue_forward(p, si.in, p->span_max, 0, kc, st)) != CDMT_OK) return rc;
        CK(p, cudaEventRecord(si.in_free, st));
        for (int q = 0; q < nq; q++, bo = (bo + 1) % 3) {
            Staging &so = p->stage[bo];
            const int dm_lo = q * qdm, cnt = std::min(qdm, p->ndm - dm_lo);
            CK(p, cudaStreamWaitEvent(st, so.out_free, 0));
            if ((rc = enqueue_dm(p, so.out, ostride, 0, kc, nq > 1 ? dm_lo : 0, nq > 1 ? cnt : 0, st)) != CDMT_OK)
                return rc;
            if (u8 && (rc = redig_enqueue(p, so.out, kc * p->seglen, ostride, so.u8, nullptr, st, p->sk_nsigma)) !=
                          CDMT_OK)
                return rc;
            CK(p, cudaEventRecord(so.out_ready, st));
            CK(p, cudaStreamWaitEvent(p->s_d2h, so.out_ready, 0));
            if (u8)   // [ndm][kc * seglen][nrow] -> rows of [ndm][nout][nrow] from sample k0 * seglen
                CK(p, cudaMemcpy2DAsync(h_u8 + k0 * p->seglen * nrow, p->nout * nrow, so.u8, kc * p->seglen * nrow,
                                        kc * p->seglen * nrow, p->ndm, cudaMemcpyDeviceToHost, p->s_d2h));
            else   // DMs dm_lo .. dm_lo + cnt - 1: cnt * nrow rows of the host filterbank
                CK(p, cudaMemcpy2DAsync(h_out + (int64_t)dm_lo * nrow * p->nout + k0 * p->seglen, p->nout * 4,
                                        so.out, ostride * 4, kc * p->seglen * 4, (int64_t)cnt * nrow,
                                        cudaMemcpyDeviceToHost, p->s_d2h));
            CK(p, cudaEventRecord(so.out_free, p->s_d2h));
        }
    }
    CK(p, cudaStreamSynchronize(p->s_d2h));
    CK(p, cudaStreamSynchronize(st));
    if (kc_used) *kc_used = kcm;
    return CDMT_OK;
}

// After a host-memory call failed part-way, copies from or into the caller's host
// buffers may still be queued: wait for every stream the call used (ignoring their
// status), so that no copy touches those buffers once the call has returned.
void drain_after_error(cdmt_plan_s *p, cudaStream_t st)
{
    cudaStreamSynchronize(st);
    if (p->s_h2d) cudaStreamSynchronize(p->s_h2d);
    if (p->s_d2h) cudaStreamSynchronize(p->s_d2h);
}

}  // namespace

int cdmt_execute_host(cdmt_plan_t p, const void *h_in, float *h_out, const float *h_scale, void *cuda_stream)
{
    if (!p) return fail(nullptr, CDMT_EINVAL, "NULL plan");
    if (!h_in || !h_out) return fail(p, CDMT_EINVAL, "NULL input or output pointer");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) CK(p, cudaSetDevice(p->device));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int rc = p->groups.empty() ? host_pipeline(p, h_in, h_scale, h_out, nullptr, nullptr, st)
                                     : grouped_host(p, h_in, h_scale, h_out, nullptr, nullptr, st);
    if (rc != CDMT_OK) drain_after_error(p, st);
    if (cur != p->device) cudaSetDevice(cur);
    return rc;
}

int cdmt_execute_host_u8_ex(cdmt_plan_t p, const void *h_in, const float *h_scale, uint8_t *h_u8,
                            int64_t *block_segments, void *cuda_stream)
{
    if (!p) return fail(nullptr, CDMT_EINVAL, "NULL plan");
    if (!h_in || !h_u8) return fail(p, CDMT_EINVAL, "NULL input or output pointer");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) CK(p, cudaSetDevice(p->device));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int rc = p->groups.empty() ? host_pipeline(p, h_in, h_scale, nullptr, h_u8, block_segments, st)
                                     : grouped_host(p, h_in, h_scale, nullptr, h_u8, block_segments, st);
    if (rc != CDMT_OK) drain_after_error(p, st);
    if (cur != p->device) cudaSetDevice(cur);
    return rc;
}

int cdmt_execute_host_u8(cdmt_plan_t p, const void *h_in, uint8_t *h_u8, int64_t *block_segments, void *cuda_stream)
{
    return cdmt_execute_host_u8_ex(p, h_in, nullptr, h_u8, block_segments, cuda_stream);
}

int cdmt_device_status(cdmt_plan_t p)
{
    if (!p) return fail(nullptr, CDMT_EINVAL, "NULL plan");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) CK(p, cudaSetDevice(p->device));
    int flag = 0;
    for (auto &g : p->groups) {
        int f = 0;
        CK(p, cudaMemcpy(&f, g.plan->d_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (f) CK(p, cudaMemset(g.plan->d_status, 0, sizeof(int)));
        flag |= f;
    }
    if (p->d_status) {
        CK(p, cudaMemcpy(&flag, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) CK(p, cudaMemset(p->d_status, 0, sizeof(int)));
    }
    if (cur != p->device) cudaSetDevice(cur);
    if (flag) return fail(p, CDMT_ETIMEOUT, "a tensor-core wait gave up; outputs of that execute are incomplete");
    return CDMT_OK;
}

int cdmt_set_timing(cdmt_plan_t p, int on)
{
    if (!p) return fail(nullptr, CDMT_EINVAL, "NULL plan");
    p->timing = on != 0;
    for (auto &g : p->groups) g.plan->timing = p->timing;
    return CDMT_OK;
}

int cdmt_stage_times(cdmt_plan_t p, double *ms, int64_t *launches)
{
    if (!p || !ms) return fail(p, CDMT_EINVAL, "NULL plan or ms");
    ms[0] = ms[1] = 0.0;
    int64_t n = 0;
    for (auto &g : p->groups) {   // a grouped plan's stages are its children's
        double cm[2];
        int64_t cl[2];
        if (cdmt_stage_times(g.plan, cm, cl) != CDMT_OK) {
            p->last_error = g.plan->last_error;
            return CDMT_ECUDA;
        }
        ms[0] += cm[0];
        ms[1] += cm[1];
        n += cl[1];
    }
    for (size_t i = 0; i + 2 < p->ev_marks.size(); i += 3) {
        float a = 0.f, b = 0.f;
        CK(p, cudaEventSynchronize(p->ev_marks[i + 2]));
        CK(p, cudaEventElapsedTime(&a, p->ev_marks[i], p->ev_marks[i + 1]));
        CK(p, cudaEventElapsedTime(&b, p->ev_marks[i + 1], p->ev_marks[i + 2]));
        ms[0] += a;
        ms[1] += b;
        n++;
    }
    if (launches) {
        launches[0] = 2 * n;  // decimated FFTs + column DFTs per chunk
        launches[1] = n;
    }
    p->ev_pool.insert(p->ev_pool.end(), p->ev_marks.begin(), p->ev_marks.end());
    p->ev_marks.clear();
    return CDMT_OK;
}

int cdmt_destroy(cdmt_plan_t p)
{
    if (!p) return CDMT_OK;
    release(p);
    delete p;
    return CDMT_OK;
}

}  // extern "C"
