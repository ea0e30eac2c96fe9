// Batches of beams of uneven shapes: one CUDA graph per batch runs, for one
// "round" (a chunk of consecutive overlap-save segments of every beam), the
// forward stage of every beam and then one persistent tensor-core launch that
// takes (beam, subband, segment, channel, DM tile) items from a device queue
// until all beams' items of the round are done.  The round number lives in
// device memory and the graph advances it, so the same graph is replayed for
// every round.
//
// This generalises the block loop of Algorithm 1 (Sec. 3): N_FFT segments of
// every subband per block, chosen to fit the GPU memory, with the transfer
// functions of every DM trial applied to each block.  Each beam keeps its own
// N_bin, n_d, channel count, integration and DM list; an autotuner chooses per
// beam the precision form and DM tile (and, for the FP32 form, N_bin) by timing
// candidates on a sample of that beam's own input.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/cdmt.h"
#include "cdmt_internal.h"
#include "cdmt_plan_impl.h"

namespace cdmt {
void set_thread_error(const char *msg);
}
using namespace cdmt;

struct cdmt_batch_s {
    int device = 0;
    int nsm = 0;
    std::vector<cdmt_beam> beams;
    std::vector<cdmt_plan_t> plans;
    std::vector<float *> out;
    std::vector<int64_t> kc, out_stride, rows;
    std::vector<cdmt_batch_tune> tune;
    int nround = 0;
    int64_t out_bytes = 0;
    TcBeam *d_beams = nullptr;
    int n_tc = 0;
    int *d_ctl = nullptr;  // [0] round, [1] next round, [2] queue, [3] status
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string last_error;
};

namespace {

int bfail(cdmt_batch_s *b, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->last_error = buf;
    else set_thread_error(buf);
    return code;
}

#define BCK(b, call)                                                                                      \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? CDMT_ENOMEM : CDMT_ECUDA, "%s: %s", #call, \
                         cudaGetErrorString(e_));                                                         \
    } while (0)

// round r: round = next; next = (round + 1) % nround; queue = 0
__global__ void k_batch_begin(int *ctl, int nround)
{
    ctl[0] = ctl[1];
    ctl[1] = (ctl[0] + 1) % nround;
    ctl[2] = 0;
}

__global__ void k_batch_set_next(int *ctl, int r) { ctl[1] = r; }

std::string tune_key(const cdmt_beam &bm)
{
    char k[256];
    snprintf(k, sizeof k, "v1 nchan=%d nint=%d ndm=%d dm0=%.6g ddm=%.6g fc=%.6g bw=%.6g nsub=%d", bm.nchan, bm.nint,
             bm.ndm, bm.dm_first, bm.dm_step, bm.f_centre_mhz, bm.bw_sub_mhz, bm.nsub);
    return k;
}

bool load_tune(const char *path, const std::string &key, cdmt_batch_tune *t)
{
    if (!path) return false;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        const size_t bar = line.find('|');
        if (bar == std::string::npos || line.substr(0, bar) != key) continue;
        std::istringstream is(line.substr(bar + 1));
        cdmt_batch_tune v{};
        if (is >> v.precision >> v.nbin >> v.dm_tile >> v.units_per_s) {
            *t = v;
            t->from_cache = 1;
            return true;
        }
    }
    return false;
}

void save_tune(const char *path, const std::string &key, const cdmt_batch_tune &t)
{
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    f << key << '|' << t.precision << ' ' << t.nbin << ' ' << t.dm_tile << ' ' << t.units_per_s << '\n';
}

// Time one candidate on a sample of the beam (its lowest nsub_s subbands, three
// segments); returns DM-trial samples per second, or -1 if the candidate is not
// valid for this beam.
double time_candidate(const cdmt_beam &bm, int precision, int64_t nbin, int dm_tile, int nsub_s, cudaStream_t st,
                      void *scratch_in, float *scratch_out, size_t scratch_out_bytes)
{
    const double dmax = std::max(std::fabs(bm.dm_first), std::fabs(bm.dm_first + (bm.ndm - 1) * bm.dm_step));
    const int64_t nd = overlap_for(bm.nsub, bm.f_centre_mhz, bm.bw_sub_mhz, dmax, bm.nchan, bm.nint, nbin);
    if (nd < 0) return -1;
    const int64_t sv = nbin - nd * bm.nchan;
    const int64_t nsamp_s = std::min<int64_t>(bm.nsamp, nbin + 2 * sv);
    if (nsamp_s < nbin) return -1;
    std::vector<double> dms(bm.ndm);
    for (int i = 0; i < bm.ndm; i++) dms[i] = bm.dm_first + i * bm.dm_step;
    cdmt_opts o{};
    o.nbin = nbin;
    o.nd = nd;
    o.dm_tile = dm_tile;
    o.precision = precision;
    const double fc_s = bm.f_centre_mhz - 0.5 * (bm.nsub - nsub_s) * bm.bw_sub_mhz;
    cdmt_plan_t p = nullptr;
    if (cdmt_plan_ex(&p, nsub_s, nsamp_s, fc_s, bm.bw_sub_mhz, dms.data(), bm.ndm, bm.nchan, bm.nint, &o) != CDMT_OK)
        return -1;
    cdmt_info inf;
    cdmt_plan_info(p, &inf);
    double rate = -1;
    if ((size_t)inf.out_bytes <= scratch_out_bytes &&
        cudaMemcpy2DAsync(scratch_in, (size_t)nsamp_s * 16, bm.d_in, (size_t)bm.nsamp * 16, (size_t)nsamp_s * 16,
                          nsub_s, cudaMemcpyDeviceToDevice, st) == cudaSuccess) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        bool ok = cdmt_execute(p, scratch_in, scratch_out, nullptr, st) == CDMT_OK;
        cudaEventRecord(e0, st);
        for (int i = 0; i < 2 && ok; i++) ok = cdmt_execute(p, scratch_in, scratch_out, nullptr, st) == CDMT_OK;
        cudaEventRecord(e1, st);
        if (ok && cudaEventSynchronize(e1) == cudaSuccess && cdmt_device_status(p) == CDMT_OK) {
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms > 0) rate = 2.0 * inf.units / (ms * 1e-3);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    cdmt_destroy(p);
    cudaGetLastError();
    return rate;
}

void release(cdmt_batch_s *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaDeviceSynchronize();
    for (float *o : b->out)
        if (o) cudaFree(o);
    for (cdmt_plan_t p : b->plans)
        if (p) cdmt_destroy(p);
    if (b->d_beams) cudaFree(b->d_beams);
    if (b->d_ctl) cudaFree(b->d_ctl);
    cudaGetLastError();
}

}  // namespace

extern "C" {

int cdmt_batch_create(cdmt_batch_t *out, int nbeam, const cdmt_beam *beams, const cdmt_batch_opts *opts, void *stream)
{
    if (!out) return bfail(nullptr, CDMT_EINVAL, "batch pointer is NULL");
    *out = nullptr;
    if (nbeam < 1 || !beams) return bfail(nullptr, CDMT_EINVAL, "need nbeam >= 1 beams");
    cdmt_batch_opts o{};
    if (opts) o = *opts;
    const int64_t budget = o.out_budget > 0 ? o.out_budget : (int64_t)16 << 30;
    auto *b = new cdmt_batch_s();
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
    b->beams.assign(beams, beams + nbeam);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < nbeam; i++) {
        const cdmt_beam &bm = beams[i];
        if (!bm.d_in || bm.nsub < 1 || bm.ndm < 1 || bm.nsamp < 1) {
            delete b;
            return bfail(nullptr, CDMT_EINVAL, "beam %d: need an input pointer, nsub, ndm, nsamp >= 1", i);
        }
    }

    // ---- choose form, N_bin and DM tile per beam
    b->tune.resize(nbeam);
    {
        // sample buffers large enough for 8 subbands x 3 segments of the largest candidate
        int64_t max_nbin = 0, max_out = 0;
        for (const cdmt_beam &bm : b->beams) {
            max_nbin = std::max<int64_t>(max_nbin, 4096LL * bm.nchan);
            max_out = std::max<int64_t>(max_out, (int64_t)bm.ndm * 8 * bm.nchan * 3 * 4096 * 4 / std::max(1, bm.nint));
        }
        void *s_in = nullptr;
        float *s_out = nullptr;
        const size_t in_bytes = (size_t)8 * 3 * max_nbin * 16, out_bytes = (size_t)max_out + (1 << 20);
        const bool measure = o.autotune != 0;
        if (measure) {
            if (cudaMalloc(&s_in, in_bytes) != cudaSuccess || cudaMalloc((void **)&s_out, out_bytes) != cudaSuccess) {
                cudaGetLastError();
                if (s_in) cudaFree(s_in);
                delete b;
                return bfail(nullptr, CDMT_ENOMEM, "autotuner sample buffers");
            }
        }
        for (int i = 0; i < nbeam; i++) {
            const cdmt_beam &bm = b->beams[i];
            cdmt_batch_tune &t = b->tune[i];
            const std::string key = tune_key(bm);
            if (load_tune(o.tune_cache, key, &t)) continue;
            // heuristic default: FP16 tensor-core form, all DMs in one tile
            t = cdmt_batch_tune{};
            t.precision = CDMT_PREC_FP16;
            t.nbin = 4096LL * bm.nchan;
            t.dm_tile = bm.ndm;
            t.units_per_s = 0;
            if (!measure) continue;
            const int nsub_s = std::min(bm.nsub, 8);
            double best = -1;
            struct Cand { int prec; int64_t nbin; int tile; };
            std::vector<Cand> cands;
            for (int div : {1, 2, 4})
                if (bm.ndm / div >= 1) cands.push_back({CDMT_PREC_FP16, 4096LL * bm.nchan, (bm.ndm + div - 1) / div});
            for (int64_t m : {4096, 2048, 1024}) cands.push_back({CDMT_PREC_FP32, m * bm.nchan, bm.ndm});
            for (const Cand &c : cands) {
                if (c.nbin > bm.nsamp) continue;
                const double r = time_candidate(bm, c.prec, c.nbin, c.tile, nsub_s, st, s_in, s_out, out_bytes);
                if (r > best) {
                    best = r;
                    t.precision = c.prec;
                    t.nbin = c.nbin;
                    t.dm_tile = c.tile;
                    t.units_per_s = r;
                }
            }
            if (best > 0) save_tune(o.tune_cache, key, t);
        }
        if (s_in) cudaFree(s_in);
        if (s_out) cudaFree(s_out);
    }

    // ---- per-beam plans with the chosen parameters (segment chunk fixed below)
    std::vector<int64_t> nseg(nbeam), seglen(nbeam), obps(nbeam);
    std::vector<cdmt_info> info(nbeam);
    for (int i = 0; i < nbeam; i++) {
        const cdmt_beam &bm = b->beams[i];
        std::vector<double> dms(bm.ndm);
        for (int k = 0; k < bm.ndm; k++) dms[k] = bm.dm_first + k * bm.dm_step;
        cdmt_opts po{};
        po.nbin = b->tune[i].nbin;
        po.nd = -1;
        po.dm_tile = b->tune[i].dm_tile;
        po.precision = b->tune[i].precision;
        po.seg_chunk = 1;  // placeholder: re-planned with the round's chunk below
        cdmt_plan_t p = nullptr;
        int rc = cdmt_plan_ex(&p, bm.nsub, bm.nsamp, bm.f_centre_mhz, bm.bw_sub_mhz, dms.data(), bm.ndm, bm.nchan,
                              bm.nint, &po);
        if (rc != CDMT_OK) {
            char msg[600];
            snprintf(msg, sizeof msg, "beam %d: %s", i, cdmt_last_error(nullptr));
            release(b);
            delete b;
            return bfail(nullptr, rc, "%s", msg);
        }
        cdmt_plan_info(p, &info[i]);
        cdmt_destroy(p);
        nseg[i] = info[i].nseg;
        seglen[i] = (info[i].mbin - info[i].nd) / bm.nint;
        obps[i] = (int64_t)bm.ndm * bm.nsub * bm.nchan * seglen[i] * 4;
    }
    // rounds: the fewest whose output chunks of all beams fit the budget
    int64_t maxseg = *std::max_element(nseg.begin(), nseg.end());
    int nround = 0;
    for (int64_t r = 1; r <= maxseg; r++) {
        int64_t need = 0;
        for (int i = 0; i < nbeam; i++) need += ((nseg[i] + r - 1) / r) * obps[i];
        if (need <= budget) { nround = (int)r; break; }
    }
    if (!nround) {
        release(b);
        delete b;
        return bfail(nullptr, CDMT_EBUDGET, "one segment of every beam needs more than the output budget of %lld bytes",
                     (long long)budget);
    }
    b->nround = nround;
    b->plans.assign(nbeam, nullptr);
    b->out.assign(nbeam, nullptr);
    b->kc.resize(nbeam);
    b->out_stride.resize(nbeam);
    b->rows.resize(nbeam);
    std::vector<TcBeam> tcb;
    for (int i = 0; i < nbeam; i++) {
        const cdmt_beam &bm = b->beams[i];
        std::vector<double> dms(bm.ndm);
        for (int k = 0; k < bm.ndm; k++) dms[k] = bm.dm_first + k * bm.dm_step;
        b->kc[i] = (nseg[i] + nround - 1) / nround;
        cdmt_opts po{};
        po.nbin = b->tune[i].nbin;
        po.nd = info[i].nd;
        po.dm_tile = b->tune[i].dm_tile;
        po.precision = b->tune[i].precision;
        po.seg_chunk = b->kc[i];
        int rc = cdmt_plan_ex(&b->plans[i], bm.nsub, bm.nsamp, bm.f_centre_mhz, bm.bw_sub_mhz, dms.data(), bm.ndm,
                              bm.nchan, bm.nint, &po);
        if (rc == CDMT_OK && !b->plans[i]->uniform) rc = CDMT_EINVAL;
        if (rc != CDMT_OK) {
            release(b);
            delete b;
            return bfail(nullptr, rc, "beam %d: plan failed", i);
        }
        b->rows[i] = (int64_t)bm.nsub * bm.nchan;
        b->out_stride[i] = b->kc[i] * seglen[i];
        const size_t ob = sizeof(float) * (size_t)bm.ndm * b->rows[i] * b->out_stride[i];
        if (cudaMalloc((void **)&b->out[i], ob) != cudaSuccess) {
            cudaGetLastError();
            release(b);
            delete b;
            return bfail(nullptr, CDMT_ENOMEM, "beam %d: round output of %zu bytes", i, ob);
        }
        b->out_bytes += (int64_t)ob;
        cdmt_plan_s *p = b->plans[i];
        if (p->precision == CDMT_PREC_FP16) {
            TcBeam t{};
            t.spec = p->spec;
            t.nco = p->nco;
            t.out = b->out[i];
            t.out_stride = b->out_stride[i];
            t.nseg = p->nseg;
            t.nsub = p->nsub;
            t.kc = (int)b->kc[i];
            t.nchan = p->nchan;
            t.ndm = p->ndm;
            t.dm_tile = p->dm_tile;
            t.ntile = p->ntile;
            t.nd = (int)p->nd;
            t.nint = p->nint;
            t.scale = (float)(1.0 / ((double)p->nbin * (double)p->mbin));
            tcb.push_back(t);
        }
    }
    b->n_tc = (int)tcb.size();
    BCK(nullptr, cudaMalloc((void **)&b->d_ctl, 4 * sizeof(int)));
    BCK(nullptr, cudaMemset(b->d_ctl, 0, 4 * sizeof(int)));
    if (b->n_tc) {
        BCK(nullptr, cudaMalloc((void **)&b->d_beams, sizeof(TcBeam) * tcb.size()));
        BCK(nullptr, cudaMemcpy(b->d_beams, tcb.data(), sizeof(TcBeam) * tcb.size(), cudaMemcpyHostToDevice));
    }

    // ---- capture one round into a graph
    BCK(nullptr, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    BCK(nullptr, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int rc = CDMT_OK;
    k_batch_begin<<<1, 1, 0, b->cap>>>(b->d_ctl, nround);
    const uint4 *bmat = nullptr;
    const float2 *twq = nullptr;
    for (int i = 0; i < nbeam && rc == CDMT_OK; i++) {
        cdmt_plan_s *p = b->plans[i];
        ForwardArgs fa{};
        fa.in = static_cast<const float4 *>(b->beams[i].d_in);
        fa.spec = p->spec;
        fa.tw_a = p->tw_af;
        fa.tw_b = p->tw_bf;
        fa.tw_n = p->tw_n;
        fa.nsamp = p->nsamp;
        fa.nvalid = p->nvalid;
        fa.nbin = p->nbin;
        fa.k0 = 0;
        fa.nchan = p->nchan;
        fa.kc = (int)b->kc[i];
        fa.nsub = p->nsub;
        fa.r = p->r;
        fa.round_dev = b->d_ctl;
        fa.nseg = p->nseg;
        if (fp32_forward(fa, b->cap) != cudaSuccess) rc = CDMT_ECUDA;
        if (p->precision == CDMT_PREC_FP16) {
            bmat = p->tc_bmat;
            twq = p->tc_twq;
        } else {
            DedispArgs da{};
            da.spec = p->spec;
            da.nco = p->nco;
            da.ktab = p->ktab;
            da.dm_list = p->d_dm;
            da.tw_a = p->tw_ai;
            da.tw_b = p->tw_bi;
            da.out = b->out[i];
            da.k0 = 0;
            da.nout = b->out_stride[i];
            da.nsub = p->nsub;
            da.kc = (int)b->kc[i];
            da.nchan = p->nchan;
            da.ndm = p->ndm;
            da.dm_tile = p->dm_tile;
            da.nd = (int)p->nd;
            da.nint = p->nint;
            da.r = p->r;
            da.uniform = true;
            da.scale = (float)(1.0 / ((double)p->nbin * (double)p->mbin));
            da.round_dev = b->d_ctl;
            da.nseg = p->nseg;
            if (fp32_dedisperse(da, b->cap) != cudaSuccess) rc = CDMT_ECUDA;
        }
    }
    if (rc == CDMT_OK && b->n_tc &&
        tc_batch_launch(b->d_beams, b->n_tc, b->d_ctl, b->d_ctl + 2, bmat, twq, b->d_ctl + 3, 0, b->nsm, b->cap) !=
            cudaSuccess)
        rc = CDMT_ECUDA;
    cudaError_t ce = cudaStreamEndCapture(b->cap, &b->graph);
    if (rc != CDMT_OK || ce != cudaSuccess || cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
        const char *why = cudaGetErrorString(cudaGetLastError());
        release(b);
        delete b;
        return bfail(nullptr, CDMT_ECUDA, "graph capture of a round failed: %s", why);
    }
    *out = b;
    return CDMT_OK;
}

int cdmt_batch_info(cdmt_batch_t b, int beam, cdmt_batch_beam_info *info)
{
    if (!b || !info || beam < 0 || beam >= (int)b->beams.size())
        return bfail(b, CDMT_EINVAL, "NULL batch / info or beam out of range");
    std::memset(info, 0, sizeof *info);
    cdmt_plan_info(b->plans[beam], &info->plan);
    info->tune = b->tune[beam];
    info->nround = b->nround;
    info->seg_per_round = b->kc[beam];
    info->d_out = b->out[beam];
    info->out_row_stride = b->out_stride[beam];
    info->out_bytes_total = b->out_bytes;
    return CDMT_OK;
}

int cdmt_batch_run_round(cdmt_batch_t b, int round, void *stream)
{
    if (!b || round < 0 || round >= b->nround) return bfail(b, CDMT_EINVAL, "NULL batch or round out of range");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_batch_set_next<<<1, 1, 0, st>>>(b->d_ctl, round);
    BCK(b, cudaGetLastError());
    BCK(b, cudaGraphLaunch(b->exec, st));
    return CDMT_OK;
}

int cdmt_batch_run(cdmt_batch_t b, void *stream)
{
    if (!b) return bfail(nullptr, CDMT_EINVAL, "NULL batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_batch_set_next<<<1, 1, 0, st>>>(b->d_ctl, 0);
    BCK(b, cudaGetLastError());
    for (int r = 0; r < b->nround; r++) BCK(b, cudaGraphLaunch(b->exec, st));
    return CDMT_OK;
}

int cdmt_batch_copy_out(cdmt_batch_t b, int beam, void *dst, void *stream)
{
    if (!b || !dst || beam < 0 || beam >= (int)b->beams.size())
        return bfail(b, CDMT_EINVAL, "NULL batch / destination or beam out of range");
    const size_t n = sizeof(float) * (size_t)b->beams[beam].ndm * (size_t)b->rows[beam] * (size_t)b->out_stride[beam];
    BCK(b, cudaMemcpyAsync(dst, b->out[beam], n, cudaMemcpyDefault, static_cast<cudaStream_t>(stream)));
    return CDMT_OK;
}

int cdmt_batch_status(cdmt_batch_t b)
{
    if (!b) return bfail(nullptr, CDMT_EINVAL, "NULL batch");
    int flag = 0;
    BCK(b, cudaMemcpy(&flag, b->d_ctl + 3, sizeof(int), cudaMemcpyDeviceToHost));
    for (cdmt_plan_t p : b->plans)
        if (cdmt_device_status(p) != CDMT_OK) flag = 1;
    if (flag) {
        BCK(b, cudaMemset(b->d_ctl + 3, 0, sizeof(int)));
        return bfail(b, CDMT_ETIMEOUT, "a tensor-core wait gave up; that round's outputs are incomplete");
    }
    return CDMT_OK;
}

const char *cdmt_batch_last_error(cdmt_batch_t b) { return b ? b->last_error.c_str() : cdmt_last_error(nullptr); }

int cdmt_batch_destroy(cdmt_batch_t b)
{
    if (!b) return CDMT_OK;
    release(b);
    delete b;
    return CDMT_OK;
}

}  // extern "C"
