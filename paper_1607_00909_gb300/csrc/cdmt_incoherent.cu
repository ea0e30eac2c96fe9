// Incoherent dedispersion of a plan's coherent filterbanks over fine DM trials
// (Sec. 4: the semi-coherent search dedisperses each coherent filterbank
// incoherently at small DM steps around its coherent DM; Sec. 1: incoherent
// dedispersion shifts each channel's time series by its dispersive delay).
//
// The channels of a coherent filterbank keep the delays between their
// reference frequencies nu_r (channel centres, or subband centres for one
// transfer function per subband), so the shift of row r for the total DM
// DM_c + ddm_k, in output samples of t_samp = nint nchan / bw seconds, is
//     d(c, k, r) = rint(D (DM_c + ddm_k) (nu_r^-2 - nu_top^-2) / t_samp)
// and, with d_lo / d_hi the extreme shifts over every (c, k, r),
//     out[c][k][t] = sum_r fb[c][r][t + d(c, k, r) - d_lo],  t < nt - (d_hi - d_lo).
// The shifts are computed once on the host in FP64.
//
// Kernel: neighbouring fine trials differ only in the channels whose shift
// grows between them (a fraction of a sample per trial, so about one channel in
// ten), hence
//     out[c][k][t] = out[c][k-1][t] + sum over changed rows (fb[r][t + d_new] - fb[r][t + d_old]).
// One CTA takes a block of kKB consecutive trials, 2048 output samples and one
// coherent DM: thread i sums the first trial of the block over all rows for
// samples t0 + i + 256 q (q < 8), then steps through the block's trials with
// the host-built lists of changed rows, storing each trial.  Every block starts
// from a full sum, so rounding does not accumulate over more than kKB - 1
// steps.  Consecutive CTAs take the other trial blocks of the same samples, so
// the filterbank rows stay in L2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/cdmt.h"
#include "cdmt_plan_impl.h"

namespace {

constexpr int kKB = 32;     // trials per CTA (one full sum, then kKB - 1 difference steps)
constexpr int kT = 8;       // samples per thread
constexpr int kThreads = 256;
constexpr int kSpan = kT * kThreads;   // samples per CTA

// Shifts of every (coherent DM, trial, row) relative to the smallest, and nt_out.
int64_t shifts(const cdmt_plan_s *p, double ddm_lo, double ddm_step, int nk, std::vector<int32_t> *tab)
{
    const int rows = p->nsub * p->nchan;
    std::vector<double> nu(rows);
    double top = 0.0;
    for (int s = 0; s < p->nsub; s++) {
        const double nu_s = p->f_centre + ((double)s - 0.5 * (double)(p->nsub - 1)) * p->bw;
        for (int c = 0; c < p->nchan; c++) {
            const double f = p->chirp == CDMT_CHIRP_SUBBAND
                                 ? nu_s
                                 : nu_s - 0.5 * p->bw + ((double)c + 0.5) * p->bw / (double)p->nchan;
            nu[s * p->nchan + c] = f;
            top = std::max(top, f);
        }
    }
    const double tsamp = (double)p->nint * (double)p->nchan / (p->bw * 1e6);
    std::vector<int32_t> local;
    std::vector<int32_t> &d = tab ? *tab : local;
    d.resize((size_t)p->ndm * nk * rows);
    int64_t lo = 0, hi = 0;
    for (int i = 0; i < p->ndm; i++)
        for (int k = 0; k < nk; k++)
            for (int r = 0; r < rows; r++) {
                const double dm = p->dms[i] + ddm_lo + (double)k * ddm_step;
                const int64_t v = (int64_t)llrint(4.148808e3 * dm * (1.0 / (nu[r] * nu[r]) - 1.0 / (top * top)) / tsamp);
                d[((size_t)i * nk + k) * rows + r] = (int32_t)v;
                if ((i | k | r) == 0 || v < lo) lo = v;
                if ((i | k | r) == 0 || v > hi) hi = v;
            }
    for (auto &v : d) v -= (int32_t)lo;
    return p->nout - (hi - lo);
}

// Device tables of a trial grid, from the shifts d[c][k][r]:
//   first[(c, b)][r]       shifts of the block's first trial,
//   off[(c, b)][kk]        start of the changes of trial kk (kk = 1 .. kKB, exclusive end at kKB),
//   chg[...]               (row, old shift, new shift) of every row whose shift changes at that trial.
struct IncTables {
    std::vector<int32_t> first, off;
    std::vector<int4> chg;
};

void build_tables(const std::vector<int32_t> &d, int ndm, int nk, int rows, IncTables *t)
{
    const int nkb = (nk + kKB - 1) / kKB;
    t->first.resize((size_t)ndm * nkb * rows);
    t->off.resize((size_t)ndm * nkb * (kKB + 1));
    t->chg.clear();
    for (int c = 0; c < ndm; c++)
        for (int b = 0; b < nkb; b++) {
            const int k0 = b * kKB;
            const size_t cb = (size_t)c * nkb + b;
            for (int r = 0; r < rows; r++) t->first[cb * rows + r] = d[((size_t)c * nk + k0) * rows + r];
            t->off[cb * (kKB + 1)] = (int32_t)t->chg.size();
            for (int kk = 1; kk <= kKB; kk++) {
                t->off[cb * (kKB + 1) + kk] = (int32_t)t->chg.size();   // start of trial kk's changes
                if (kk == kKB || k0 + kk >= nk) continue;
                const int32_t *prev = &d[((size_t)c * nk + k0 + kk - 1) * rows];
                const int32_t *now = prev + rows;
                for (int r = 0; r < rows; r++)
                    if (now[r] != prev[r]) t->chg.push_back(make_int4(r, prev[r], now[r], 0));
            }
        }
}

__global__ void __launch_bounds__(kThreads) k_incoherent(const float *__restrict__ fb, const int32_t *__restrict__ first,
                                                        const int32_t *__restrict__ off, const int4 *__restrict__ chg,
                                                        float *__restrict__ out, int rows, int64_t nt, int nk,
                                                        int64_t nt_out)
{
    const int b = blockIdx.x;
    const int k0 = b * kKB;
    const int64_t t0 = (int64_t)blockIdx.y * kSpan;
    const int c = blockIdx.z;
    const int nkb = min(kKB, nk - k0);
    const int64_t cb = (int64_t)c * gridDim.x + b;
    const float *src = fb + (int64_t)c * rows * nt;
    const int32_t *fs = first + cb * rows;
    const int32_t *of = off + cb * (kKB + 1);
    int64_t t[kT];
    bool live[kT];
    #pragma unroll
    for (int q = 0; q < kT; q++) {
        t[q] = t0 + threadIdx.x + (int64_t)q * kThreads;
        live[q] = t[q] < nt_out;
    }
    // the block's first trial: the full sum over rows
    float acc[kT];
    #pragma unroll
    for (int q = 0; q < kT; q++) acc[q] = 0.f;
    #pragma unroll 4
    for (int r = 0; r < rows; r++) {
        const float *row = src + (int64_t)r * nt + __ldg(fs + r);
        #pragma unroll
        for (int q = 0; q < kT; q++)
            if (live[q]) acc[q] += __ldg(row + t[q]);
    }
    float *o = out + ((int64_t)c * nk + k0) * nt_out;
    #pragma unroll
    for (int q = 0; q < kT; q++)
        if (live[q]) o[t[q]] = acc[q];
    // the other trials: add the changed rows' new samples, remove their old ones
    for (int kk = 1; kk < nkb; kk++) {
        const int e0 = __ldg(of + kk), e1 = __ldg(of + kk + 1);
        #pragma unroll 2
        for (int e = e0; e < e1; e++) {
            const int4 ch = __ldg(chg + e);
            const float *row = src + (int64_t)ch.x * nt;
            #pragma unroll
            for (int q = 0; q < kT; q++)
                if (live[q]) acc[q] += __ldg(row + t[q] + ch.z) - __ldg(row + t[q] + ch.y);
        }
        o += nt_out;
        #pragma unroll
        for (int q = 0; q < kT; q++)
            if (live[q]) o[t[q]] = acc[q];
    }
}

int ifail(cdmt_plan_s *p, int code, const char *msg)
{
    p->last_error = msg;
    return code;
}

}  // namespace

extern "C" {

int cdmt_incoherent_info(cdmt_plan_t p, double ddm_lo, double ddm_step, int nk, int64_t *nt_out, int32_t *h_delays)
{
    if (!p) return CDMT_EINVAL;
    if (nk < 1 || !nt_out) return ifail(p, CDMT_EINVAL, "nk must be >= 1 and nt_out not NULL");
    std::vector<int32_t> tab;
    if (!h_delays && p->inc_key[0] == ddm_lo && p->inc_key[1] == ddm_step && p->inc_nk == nk) {
        *nt_out = p->inc_nt_out;   // the grid of the last cdmt_incoherent call
        return CDMT_OK;
    }
    *nt_out = shifts(p, ddm_lo, ddm_step, nk, h_delays ? &tab : nullptr);
    if (h_delays) std::copy(tab.begin(), tab.end(), h_delays);
    if (*nt_out < 1) return ifail(p, CDMT_EINVAL, "the shifts leave no output sample");
    return CDMT_OK;
}

int cdmt_incoherent(cdmt_plan_t p, const float *d_fb, double ddm_lo, double ddm_step, int nk, float *d_out,
                    void *cuda_stream)
{
    if (!p) return CDMT_EINVAL;
    if (!d_fb || !d_out || nk < 1) return ifail(p, CDMT_EINVAL, "NULL buffer or nk < 1");
    const cdmt::Range range("cdmt incoherent stage");
    const int rows = p->nsub * p->nchan;
    const bool same = p->inc_key[0] == ddm_lo && p->inc_key[1] == ddm_step && p->inc_nk == nk;
    std::vector<int32_t> tab;
    const int64_t nt_out = same ? p->inc_nt_out : shifts(p, ddm_lo, ddm_step, nk, &tab);
    if (nt_out < 1) return ifail(p, CDMT_EINVAL, "the shifts leave no output sample");
    if (p->ndm > 65535 || (nt_out + kSpan - 1) / kSpan > 65535)
        return ifail(p, CDMT_ENOTSUP, "more than 65535 coherent DMs or sample blocks");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device && cudaSetDevice(p->device) != cudaSuccess) return ifail(p, CDMT_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int rc = CDMT_OK;
    if (!same) {
        // the plan keeps the tables of the last trial grid in one device buffer:
        // first shifts, change offsets, changes (16-byte aligned)
        IncTables tb;
        build_tables(tab, p->ndm, nk, rows, &tb);
        const size_t b_first = sizeof(int32_t) * tb.first.size(), b_off = sizeof(int32_t) * tb.off.size();
        const size_t o_off = (b_first + 15) / 16 * 16, o_chg = (o_off + b_off + 15) / 16 * 16;
        const size_t bytes = o_chg + sizeof(int4) * std::max<size_t>(1, tb.chg.size());
        if (p->inc_bytes < bytes) {
            if (p->inc_tab) cudaFree(p->inc_tab);
            p->inc_tab = nullptr;
            p->inc_bytes = 0;
            if (cudaMalloc((void **)&p->inc_tab, bytes) != cudaSuccess) {
                cudaGetLastError();
                rc = ifail(p, CDMT_ENOMEM, "incoherent shift tables");
            } else {
                p->inc_bytes = bytes;
            }
        }
        // synchronous copies from pageable memory: the tables may not change under a running kernel
        uint8_t *base = reinterpret_cast<uint8_t *>(p->inc_tab);
        if (rc == CDMT_OK &&
            (cudaStreamSynchronize(st) != cudaSuccess ||
             cudaMemcpy(base, tb.first.data(), b_first, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(base + o_off, tb.off.data(), b_off, cudaMemcpyHostToDevice) != cudaSuccess ||
             (!tb.chg.empty() && cudaMemcpy(base + o_chg, tb.chg.data(), sizeof(int4) * tb.chg.size(),
                                            cudaMemcpyHostToDevice) != cudaSuccess))) {
            cudaGetLastError();
            rc = ifail(p, CDMT_ECUDA, "incoherent shift table upload");
        }
        if (rc == CDMT_OK) {
            p->inc_key[0] = ddm_lo;
            p->inc_key[1] = ddm_step;
            p->inc_nk = nk;
            p->inc_nt_out = nt_out;
            p->inc_off = o_off;
            p->inc_chg = o_chg;
        } else {
            p->inc_nk = 0;
        }
    }
    if (rc == CDMT_OK) {
        const dim3 grid((unsigned)((nk + kKB - 1) / kKB), (unsigned)((nt_out + kSpan - 1) / kSpan), (unsigned)p->ndm);
        const uint8_t *base = reinterpret_cast<const uint8_t *>(p->inc_tab);
        k_incoherent<<<grid, kThreads, 0, st>>>(d_fb, reinterpret_cast<const int32_t *>(base),
                                                reinterpret_cast<const int32_t *>(base + p->inc_off),
                                                reinterpret_cast<const int4 *>(base + p->inc_chg), d_out, rows,
                                                p->nout, nk, nt_out);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = ifail(p, CDMT_ECUDA, cudaGetErrorString(e));
    }
    if (cur != p->device) cudaSetDevice(cur);
    return rc;
}

}  // extern "C"
