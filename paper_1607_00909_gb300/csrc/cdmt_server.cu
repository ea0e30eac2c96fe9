// Streaming server: real-time voltage blocks from several beams, continuously
// batched on one GPU.
//
// Each beam keeps, resident on the device, its plan (chirp-phase words,
// twiddles, workspace), the overlap tail of its stream (Sec. 2: consecutive
// overlap-save segments share n_d n_c input samples; samples that do not yet
// complete a segment wait for the next block) and one block buffer.  A block
// of a beam is appended after its tail, every segment it completes is
// dedispersed into an output slot, and the unconsumed samples become the new
// tail (Algorithm 1's block loop, "read block" ... "copy to host", run per
// beam as blocks arrive).
//
// Output slots come from one pool whose size follows from the HBM budget left
// after the resident beam state.  A scheduler thread dispatches queued blocks
// in arrival order, across beams, whenever a slot is free (blocks of one beam
// stay in order on that beam's CUDA stream, blocks of different beams overlap
// on the device), watches completion events, and keeps latency statistics.
// The caller waits for a block, reads its filterbank in the slot, and
// releases the slot.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/cdmt.h"
#include "cdmt_internal.h"
#include "cdmt_plan_impl.h"

namespace cdmt {
void set_thread_error(const char *msg);
}
using namespace cdmt;

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// stage[s][tail + i] = block sample i of subband s, as float4; int8 input is
// (X re, X im, Y re, Y im) scaled by the subband's scale
__global__ void k_append(float4 *__restrict__ stage, int64_t cap, int64_t tail, const void *__restrict__ block,
                         const float *__restrict__ scale, int64_t blen, int nsub, int i8)
{
    const int64_t total = (int64_t)nsub * blen;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(q / blen);
        const int64_t i = q % blen;
        float4 v;
        if (i8) {
            const char4 c = reinterpret_cast<const char4 *>(block)[q];
            const float a = scale[s];
            v = make_float4(a * (float)c.x, a * (float)c.y, a * (float)c.z, a * (float)c.w);
        } else {
            v = reinterpret_cast<const float4 *>(block)[q];
        }
        stage[(int64_t)s * cap + tail + i] = v;
    }
}

struct Req {
    int64_t id = 0;
    int beam = 0;
    const void *block = nullptr;
    const float *scale = nullptr;
    int64_t index = 0;          // block number within the beam
    double t_submit = 0, t_start = 0, t_done = 0;
    int state = 0;              // 0 queued, 1 running, 2 done, 3 failed
    int slot = -1;
    int scratch = -1;           // 8-bit beams: slot holding the float32 filterbank until the block completes
    cudaEvent_t ev = nullptr;
    int64_t nseg = 0, seg0 = 0; // segments of this block's output and the global index of its first
};

struct Beam {
    cdmt_stream_desc d{};
    cdmt_plan_t plan = nullptr;
    int64_t N = 0, S = 0, nd = 0, M = 0, seglen = 0, max_seg = 0, cap = 0, rows = 0;
    int64_t stride = 0;         // floats between the rows of a block's float32 filterbank (a multiple of 4)
    float4 *stage[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t tail = 0, seg_total = 0, next_index = 0;
    // two block buffers: the copy of the next block (own stream) overlaps the compute of this one
    void *d_blk[2] = {nullptr, nullptr};
    float *d_scale[2] = {nullptr, nullptr};
    cudaStream_t cp = nullptr;
    cudaEvent_t blk_ready[2] = {nullptr, nullptr}, blk_free[2] = {nullptr, nullptr};
    // stage_free[x]: the last block that used staging buffer x has finished with it (complex64 blocks
    // from host memory are copied straight into the staging buffer behind the tail)
    cudaEvent_t stage_free[2] = {nullptr, nullptr};
    int cb = 0;                 // block buffer of the next block
    int64_t fb_bytes = 0;       // float32 filterbank of one block (8-bit beams: of one DM range of a block)
    int nq = 1, qdm = 0;        // 8-bit beams: DM ranges per block and DMs per range
    int64_t codes_bytes = 0;    // 8-bit beams: codes part of a slot (16-byte multiple); statistics follow,
    int64_t stats_bytes = 0;    // then one flag byte per row
    cudaStream_t st = nullptr;
    std::deque<int64_t> fifo;
    int64_t bytes = 0;
    int64_t out_bytes = 0;     // one block's output (max_seg segments)
    bool active = true;
};

struct Slot {
    uint8_t *p = nullptr;
    int64_t bytes = 0;
    int64_t owner = -1;   // request id, -1 when free
};

}  // namespace

struct cdmt_server_s {
    int device = 0;
    cdmt_server_opts o{};
    std::vector<Beam> beams;
    std::vector<Slot> slots;
    int64_t slot_total = 0;        // bytes held by output slots
    int64_t resident = 0;          // bytes held by beam state
    std::map<int64_t, Req> reqs;
    int64_t next_id = 1;
    std::vector<double> lat_ms;
    double t_first = 0, t_last = 0;
    double data_s = 0, units = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread sched;
    std::atomic<bool> stop{false};
    std::string last_error;
    std::string fatal;
};

namespace {

int sfail(cdmt_server_s *v, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (v) v->last_error = buf;
    else set_thread_error(buf);
    return code;
}

// Free slot i (unused) and re-point the requests that own later slots (lock held).
void erase_slot(cdmt_server_s *v, size_t i)
{
    cudaFree(v->slots[i].p);
    v->slot_total -= v->slots[i].bytes;
    v->slots.erase(v->slots.begin() + (std::ptrdiff_t)i);
    for (size_t j = i; j < v->slots.size(); j++) {   // the slot at j was at j + 1
        auto it = v->reqs.find(v->slots[j].owner);
        if (it == v->reqs.end()) continue;
        if (it->second.slot == (int)j + 1) it->second.slot = (int)j;
        else if (it->second.scratch == (int)j + 1) it->second.scratch = (int)j;
    }
}

// A free slot of at least `bytes` (lock held).  Takes the smallest free one
// that fits if it is at most twice the size asked for; otherwise allocates one
// of the size asked for while the budget and the slot limit allow, else takes
// the larger free slot, else frees unused slots that are too small and stand in
// the way (cudaFree waits for the device, so that is the last resort).  -1: the
// block has to wait for a release.
int take_slot(cdmt_server_s *v, int64_t bytes)
{
    int best = -1;
    for (size_t i = 0; i < v->slots.size(); i++) {
        const Slot &sl = v->slots[i];
        if (sl.owner < 0 && sl.bytes >= bytes && (best < 0 || sl.bytes < v->slots[best].bytes)) best = (int)i;
    }
    if (best >= 0 && v->slots[best].bytes <= 2 * bytes) return best;
    const int64_t max_slots = v->o.max_slots > 0 ? v->o.max_slots : 64;
    auto full = [&] {
        return (int64_t)v->slots.size() >= max_slots || v->resident + v->slot_total + bytes > v->o.hbm_budget;
    };
    if (best >= 0 && full()) return best;
    while (full()) {
        int small = -1;
        for (size_t i = 0; i < v->slots.size(); i++)
            if (v->slots[i].owner < 0 && (small < 0 || v->slots[i].bytes < v->slots[small].bytes)) small = (int)i;
        if (small < 0) return -1;
        erase_slot(v, (size_t)small);
    }
    Slot sl;
    sl.bytes = bytes;
    if (cudaMalloc((void **)&sl.p, (size_t)bytes) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    v->slots.push_back(sl);
    v->slot_total += bytes;
    return (int)v->slots.size() - 1;
}

// Free every unused slot (lock held), so that admission can reuse the memory.
void drop_free_slots(cdmt_server_s *v)
{
    for (size_t i = v->slots.size(); i-- > 0;)
        if (v->slots[i].owner < 0) erase_slot(v, i);
}

// Enqueue the GPU work of request r of beam b on the beam's stream (scheduler thread, lock held).
bool dispatch(cdmt_server_s *v, Beam &b, Req &r)
{
    const size_t es = b.d.in_dtype == CDMT_IN_I8 ? 4 : 16;
    const size_t bytes = es * (size_t)b.d.nsub * (size_t)b.d.block_len;
    const void *src = r.block;
    cudaPointerAttributes pa{};
    const bool on_device = cudaPointerGetAttributes(&pa, r.block) == cudaSuccess && pa.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    // Complex64 blocks from host memory go straight into the staging buffer; int8 blocks (and their
    // scales) into block buffer i on the copy stream, once the block that used the buffer before has
    // been appended, and k_append dequantises them behind the tail (it also appends blocks that are
    // already in device memory); the beam's stream waits for the copy
    const int i = b.cb;
    b.cb ^= 1;
    const bool i8 = b.d.in_dtype == CDMT_IN_I8;
    float4 *stage = b.stage[b.cur];
    if (!on_device && !i8) {
        // complex64 from host memory: one 2-D copy (rows of block_len samples) straight behind the tail
        // of this block's staging buffer, once the block before last has finished with that buffer
        if (cudaStreamWaitEvent(b.cp, b.stage_free[b.cur], 0) != cudaSuccess) return false;
        if (cudaMemcpy2DAsync(stage + b.tail, (size_t)b.cap * 16, r.block, (size_t)b.d.block_len * 16,
                              (size_t)b.d.block_len * 16, b.d.nsub, cudaMemcpyHostToDevice, b.cp) != cudaSuccess)
            return false;
        if (cudaEventRecord(b.blk_ready[i], b.cp) != cudaSuccess) return false;
        if (cudaStreamWaitEvent(b.st, b.blk_ready[i], 0) != cudaSuccess) return false;
    } else if (i8) {
        if (cudaStreamWaitEvent(b.cp, b.blk_free[i], 0) != cudaSuccess) return false;
        if (!on_device) {
            if (cudaMemcpyAsync(b.d_blk[i], r.block, bytes, cudaMemcpyHostToDevice, b.cp) != cudaSuccess) return false;
            src = b.d_blk[i];
        }
        if (i8 && cudaMemcpyAsync(b.d_scale[i], r.scale, sizeof(float) * b.d.nsub, cudaMemcpyDefault, b.cp) !=
                      cudaSuccess)
            return false;
        if (cudaEventRecord(b.blk_ready[i], b.cp) != cudaSuccess) return false;
        if (cudaStreamWaitEvent(b.st, b.blk_ready[i], 0) != cudaSuccess) return false;
    }
    if (on_device || i8) {
        k_append<<<512, 256, 0, b.st>>>(stage, b.cap, b.tail, src, b.d_scale[i], b.d.block_len, b.d.nsub, i8);
        if (cudaGetLastError() != cudaSuccess) return false;
        if (cudaEventRecord(b.blk_free[i], b.st) != cudaSuccess) return false;
    }
    const int64_t avail = b.tail + b.d.block_len;
    int64_t nseg = avail >= b.N ? (avail - b.N) / b.S + 1 : 0;
    nseg = std::min(nseg, b.max_seg);
    if (nseg > 0) {
        uint8_t *slot = v->slots[r.slot].p;
        if (b.d.out_dtype != CDMT_OUT_U8) {
            if (enqueue_chunk(b.plan, stage, b.cap, 0, reinterpret_cast<float *>(slot), b.stride, 0, (int)nseg, b.st) !=
                CDMT_OK)
                return false;
        } else {
            // 8-bit: the DM stage range by range into the scratch slot, each range redigitised into its
            // part of the output slot (codes [ndm][samples][rows], then (mu, sigma), then flags)
            if (enqueue_forward(b.plan, stage, b.cap, 0, (int)nseg, b.st) != CDMT_OK) return false;
            float *fb = reinterpret_cast<float *>(v->slots[r.scratch].p);
            const int64_t samples = nseg * b.seglen;
            for (int q = 0; q < b.nq; q++) {
                const int lo = q * b.qdm, cnt = std::min(b.qdm, b.d.ndm - lo);
                if (enqueue_dm(b.plan, fb, b.stride, 0, (int)nseg, b.nq > 1 ? lo : 0, b.nq > 1 ? cnt : 0, b.st) !=
                    CDMT_OK)
                    return false;
                if (redig_enqueue(b.plan, fb, samples, b.stride, slot + (int64_t)lo * samples * b.rows,
                                  reinterpret_cast<float *>(slot + b.codes_bytes) + (int64_t)lo * b.rows * 2, b.st,
                                  b.d.sk_nsigma, slot + b.codes_bytes + b.stats_bytes + (int64_t)lo * b.rows, cnt) !=
                    CDMT_OK)
                    return false;
            }
        }
    }
    const int64_t used = nseg * b.S;
    const int64_t tail = avail - used;
    if (tail > 0 &&
        cudaMemcpy2DAsync(b.stage[b.cur ^ 1], (size_t)b.cap * 16, stage + used, (size_t)b.cap * 16, (size_t)tail * 16,
                          b.d.nsub, cudaMemcpyDeviceToDevice, b.st) != cudaSuccess)
        return false;
    if (cudaEventRecord(b.stage_free[b.cur], b.st) != cudaSuccess) return false;
    b.cur ^= 1;
    b.tail = tail;
    r.nseg = nseg;
    r.seg0 = b.seg_total;
    b.seg_total += nseg;
    return cudaEventRecord(r.ev, b.st) == cudaSuccess;
}

void scheduler(cdmt_server_s *v)
{
    cudaSetDevice(v->device);
    std::unique_lock<std::mutex> lk(v->mu);
    while (!v->stop) {
        bool progress = false;
        // completions
        for (auto &kv : v->reqs) {
            Req &r = kv.second;
            if (r.state != 1) continue;
            const cudaError_t q = cudaEventQuery(r.ev);
            if (q == cudaSuccess) {
                r.state = 2;
                r.t_done = now_s();
                v->lat_ms.push_back((r.t_done - r.t_submit) * 1e3);
                v->t_last = r.t_done;
                const Beam &b = v->beams[r.beam];
                v->data_s += (double)b.d.block_len / (b.d.bw_sub_mhz * 1e6);
                v->units += (double)b.d.ndm * b.d.nsub * r.nseg * b.S;
                if (r.scratch >= 0) {   // the float32 filterbank of an 8-bit block is no longer needed
                    v->slots[r.scratch].owner = -1;
                    r.scratch = -1;
                }
                progress = true;
            } else if (q != cudaErrorNotReady) {
                r.state = 3;
                v->fatal = cudaGetErrorString(q);
                progress = true;
            }
        }
        // dispatch: oldest queued block first, across beams, while it gets a slot
        for (;;) {
            Req *best = nullptr;
            for (Beam &b : v->beams) {
                if (b.fifo.empty()) continue;
                Req &r = v->reqs[b.fifo.front()];
                if (!best || r.id < best->id) best = &r;
            }
            if (!best) break;
            Beam &b = v->beams[best->beam];
            // 8-bit beams: the float32 scratch slot first (the larger one), then the output slot
            // (taking the second may move the first: erase_slot re-points the request)
            if (b.d.out_dtype == CDMT_OUT_U8) {
                const int scratch = take_slot(v, b.fb_bytes);
                if (scratch < 0) break;
                best->scratch = scratch;
                v->slots[scratch].owner = best->id;
            }
            const int slot = take_slot(v, b.out_bytes);
            if (slot < 0) {
                if (best->scratch >= 0) v->slots[best->scratch].owner = -1;
                best->scratch = -1;
                break;
            }
            best->slot = slot;
            v->slots[slot].owner = best->id;
            b.fifo.pop_front();
            best->t_start = now_s();
            if (dispatch(v, b, *best)) best->state = 1;
            else {
                best->state = 3;
                v->fatal = "dispatch failed";
            }
            progress = true;
        }
        if (progress) v->cv_done.notify_all();
        v->cv_work.wait_for(lk, std::chrono::microseconds(progress ? 0 : 50));
    }
}

void free_beam(Beam &b)
{
    if (b.st) cudaStreamSynchronize(b.st);
    if (b.cp) cudaStreamSynchronize(b.cp);
    if (b.plan) cdmt_destroy(b.plan);
    for (float4 *p : b.stage)
        if (p) cudaFree(p);
    for (int i = 0; i < 2; i++) {
        if (b.d_blk[i]) cudaFree(b.d_blk[i]);
        if (b.d_scale[i]) cudaFree(b.d_scale[i]);
        if (b.blk_ready[i]) cudaEventDestroy(b.blk_ready[i]);
        if (b.blk_free[i]) cudaEventDestroy(b.blk_free[i]);
        if (b.stage_free[i]) cudaEventDestroy(b.stage_free[i]);
    }
    if (b.cp) cudaStreamDestroy(b.cp);
    if (b.st) cudaStreamDestroy(b.st);
    b = Beam{};
    b.active = false;
    cudaGetLastError();
}

}  // namespace

extern "C" {

int cdmt_server_create(cdmt_server_t *out, const cdmt_server_opts *opts)
{
    if (!out) return sfail(nullptr, CDMT_EINVAL, "server pointer is NULL");
    auto *v = new cdmt_server_s();
    if (opts) v->o = *opts;
    if (v->o.hbm_budget <= 0) v->o.hbm_budget = (int64_t)120 << 30;
    cudaGetDevice(&v->device);
    v->sched = std::thread(scheduler, v);
    *out = v;
    return CDMT_OK;
}

int cdmt_server_add_beam(cdmt_server_t v, const cdmt_stream_desc *d, int *beam_id)
{
    if (!v || !d || !beam_id) return sfail(v, CDMT_EINVAL, "NULL server, descriptor or id");
    if (d->block_len < 1 || d->nsub < 1 || d->ndm < 1) return sfail(v, CDMT_EINVAL, "bad stream descriptor");
    if (d->in_dtype != CDMT_IN_C64 && d->in_dtype != CDMT_IN_I8) return sfail(v, CDMT_ENOTSUP, "input dtype");
    if (d->out_dtype != CDMT_OUT_F32 && d->out_dtype != CDMT_OUT_U8) return sfail(v, CDMT_ENOTSUP, "output dtype");
    if (!(d->sk_nsigma >= 0.0)) return sfail(v, CDMT_EINVAL, "sk_nsigma must be >= 0");
    Beam b;
    b.d = *d;
    const int64_t nbin = d->nbin > 0 ? d->nbin : 4096LL * d->nchan;
    const double dmax = std::max(std::fabs(d->dm_first), std::fabs(d->dm_first + (d->ndm - 1) * d->dm_step));
    const int64_t nd = overlap_for(d->nsub, d->f_centre_mhz, d->bw_sub_mhz, dmax, d->nchan, d->nint, nbin);
    if (nd < 0) return sfail(v, CDMT_EINVAL, "the overlap does not fit N_bin = %lld", (long long)nbin);
    b.N = nbin;
    b.nd = nd;
    b.M = nbin / d->nchan;
    b.S = nbin - nd * d->nchan;
    b.seglen = (b.M - nd) / d->nint;
    b.cap = nbin + d->block_len;                  // tail (< N) + one block
    b.max_seg = (b.cap - nbin) / b.S + 1;
    b.rows = (int64_t)d->nsub * d->nchan;
    std::vector<double> dms(d->ndm);
    for (int i = 0; i < d->ndm; i++) dms[i] = d->dm_first + i * d->dm_step;
    cdmt_opts po{};
    po.nbin = nbin;
    po.nd = nd;
    po.precision = d->precision;
    po.seg_chunk = b.max_seg;
    po.dm_tile = d->dm_tile;
    std::lock_guard<std::mutex> lk(v->mu);
    int rc = cdmt_plan_ex(&b.plan, d->nsub, b.cap, d->f_centre_mhz, d->bw_sub_mhz, dms.data(), d->ndm, d->nchan,
                          d->nint, &po);
    if (rc != CDMT_OK) return sfail(v, rc, "beam plan: %s", cdmt_last_error(nullptr));
    cdmt_info inf;
    cdmt_plan_info(b.plan, &inf);
    const size_t es = d->in_dtype == CDMT_IN_I8 ? 4 : 16;
    const bool u8 = d->out_dtype == CDMT_OUT_U8;
    b.stride = (b.max_seg * b.seglen + 3) / 4 * 4;   // rows 16-byte aligned
    // 8-bit beams of a plan with one DM tile: when a block's float32 filterbank would take more than a
    // sixth of the HBM budget as scratch, the block's DM stage runs in 2 or 4 ranges (of at least 32
    // DMs) through a scratch of one range (one launch is faster when memory allows: 436.6 against
    // 426.7 DM-trial Gsamples/s on 8 beams of 288 subbands)
    b.nq = 1;
    if (u8 && inf.dm_tile >= d->ndm) {
        const int64_t full = (int64_t)sizeof(float) * d->ndm * b.rows * b.stride;
        while (b.nq < 4 && full / b.nq > v->o.hbm_budget / 6 && d->ndm / (2 * b.nq) >= 32) b.nq *= 2;
    }
    b.qdm = (d->ndm + b.nq - 1) / b.nq;
    b.fb_bytes = (int64_t)sizeof(float) * (u8 ? b.qdm : d->ndm) * b.rows * b.stride;
    b.codes_bytes = ((int64_t)d->ndm * b.rows * b.max_seg * b.seglen + 15) / 16 * 16;
    b.stats_bytes = (int64_t)sizeof(float) * 2 * d->ndm * b.rows;
    b.out_bytes = u8 ? b.codes_bytes + b.stats_bytes + (int64_t)d->ndm * b.rows : b.fb_bytes;
    // block buffers only for int8 blocks (complex64 blocks are copied straight into the staging buffer)
    const int64_t blk_bytes = d->in_dtype == CDMT_IN_I8 ? (int64_t)es * d->nsub * d->block_len : 0;
    b.bytes = inf.workspace_bytes + 2 * (int64_t)d->nsub * b.cap * 16 + 2 * blk_bytes +
              2 * (int64_t)sizeof(float) * d->nsub + (u8 ? (int64_t)sizeof(float) * 2 * d->ndm * b.rows : 0);
    // admission: resident state of every beam + the slots held + the slots one block of this beam
    // needs (an output slot; 8-bit beams also a float32 scratch slot) unless the pool has them
    auto need = [&] {
        int64_t big = 0, fit = 0;
        for (const Slot &sl : v->slots) {
            big += sl.bytes >= b.fb_bytes;
            fit += sl.bytes >= b.out_bytes;
        }
        int64_t extra = 0;
        if (u8) {
            if (big < 1) extra += b.fb_bytes;
            if (fit < 2) extra += b.out_bytes;
        } else if (fit < 1) {
            extra += b.out_bytes;
        }
        return v->resident + b.bytes + v->slot_total + extra;
    };
    if (need() > v->o.hbm_budget) drop_free_slots(v);
    if (need() > v->o.hbm_budget) {
        cdmt_destroy(b.plan);
        return sfail(v, CDMT_EBUDGET, "beam needs %lld resident bytes and a %lld-byte output slot; %lld of the "
                     "%lld-byte budget are in use", (long long)b.bytes, (long long)b.out_bytes,
                     (long long)(v->resident + v->slot_total), (long long)v->o.hbm_budget);
    }
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; i++) e = cudaMalloc((void **)&b.stage[i], (size_t)d->nsub * b.cap * 16);
    for (int i = 0; i < 2 && e == cudaSuccess; i++) {
        if (blk_bytes > 0) e = cudaMalloc(&b.d_blk[i], (size_t)blk_bytes);
        if (e == cudaSuccess) e = cudaMalloc((void **)&b.d_scale[i], sizeof(float) * d->nsub);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.blk_ready[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.blk_free[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.stage_free[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b.cp, cudaStreamNonBlocking);
    if (e == cudaSuccess && u8 && redig_reserve(b.plan) != CDMT_OK) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_beam(b);
        return sfail(v, CDMT_ENOMEM, "beam buffers: %s", cudaGetErrorString(e));
    }
    // the first block's tail is empty: the stream starts with the first sample received
    v->resident += b.bytes;
    // further slots are allocated by the scheduler as blocks need them
    *beam_id = (int)v->beams.size();
    v->beams.push_back(b);
    return CDMT_OK;
}

int cdmt_server_submit(cdmt_server_t v, int beam, const void *block, const float *scale, int64_t *request_id)
{
    if (!v || !block || !request_id) return sfail(v, CDMT_EINVAL, "NULL server, block or id");
    std::lock_guard<std::mutex> lk(v->mu);
    if (beam < 0 || beam >= (int)v->beams.size() || !v->beams[beam].active)
        return sfail(v, CDMT_EINVAL, "no beam %d", beam);
    Beam &b = v->beams[beam];
    if (b.d.in_dtype == CDMT_IN_I8 && !scale) return sfail(v, CDMT_EINVAL, "int8 blocks need a scale array");
    Req r;
    r.id = v->next_id++;
    r.beam = beam;
    r.block = block;
    r.scale = scale;
    r.index = b.next_index++;
    r.t_submit = now_s();
    if (!v->t_first) v->t_first = r.t_submit;
    if (cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess)
        return sfail(v, CDMT_ECUDA, "event creation failed");
    v->reqs[r.id] = r;
    b.fifo.push_back(r.id);
    *request_id = r.id;
    v->cv_work.notify_all();
    return CDMT_OK;
}

int cdmt_server_wait(cdmt_server_t v, int64_t id, double timeout_s, cdmt_block_result *res)
{
    if (!v) return sfail(nullptr, CDMT_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(v->mu);
    auto it = v->reqs.find(id);
    if (it == v->reqs.end()) return sfail(v, CDMT_EINVAL, "no request %lld", (long long)id);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (it->second.state < 2) {
        if (v->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second.state < 2)
            return sfail(v, CDMT_ETIMEOUT, "request %lld not done after %.3f s", (long long)id, timeout_s);
    }
    Req &r = it->second;
    if (r.state == 3) return sfail(v, CDMT_ECUDA, "request %lld failed: %s", (long long)id, v->fatal.c_str());
    if (res) {
        const Beam &b = v->beams[r.beam];
        std::memset(res, 0, sizeof *res);
        res->beam = r.beam;
        res->index = r.index;
        uint8_t *slot = v->slots[r.slot].p;
        if (b.d.out_dtype == CDMT_OUT_U8) {
            res->d_u8 = slot;
            res->d_stats = reinterpret_cast<float *>(slot + b.codes_bytes);
            res->d_flags = slot + b.codes_bytes + b.stats_bytes;
        } else {
            res->d_out = reinterpret_cast<float *>(slot);
        }
        res->nseg = r.nseg;
        res->first_sample = r.seg0 * b.seglen;
        res->samples = r.nseg * b.seglen;
        res->row_stride = b.stride;
        res->latency_ms = (r.t_done - r.t_submit) * 1e3;
    }
    return CDMT_OK;
}

int cdmt_server_release(cdmt_server_t v, int64_t id)
{
    if (!v) return sfail(nullptr, CDMT_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(v->mu);
    auto it = v->reqs.find(id);
    if (it == v->reqs.end() || it->second.state < 2) return sfail(v, CDMT_EINVAL, "request %lld is not done", (long long)id);
    if (it->second.slot >= 0) v->slots[it->second.slot].owner = -1;
    if (it->second.scratch >= 0) v->slots[it->second.scratch].owner = -1;
    cudaEventDestroy(it->second.ev);
    v->reqs.erase(it);
    v->cv_work.notify_all();
    return CDMT_OK;
}

int cdmt_server_get_stats(cdmt_server_t v, cdmt_server_stats *st)
{
    if (!v || !st) return sfail(v, CDMT_EINVAL, "NULL server or stats");
    std::lock_guard<std::mutex> lk(v->mu);
    std::memset(st, 0, sizeof *st);
    std::vector<double> l = v->lat_ms;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
    st->blocks_done = (int64_t)l.size();
    for (auto &kv : v->reqs) {
        if (kv.second.state == 0) st->blocks_queued++;
        if (kv.second.state == 1) st->blocks_running++;
    }
    st->latency_p50_ms = pct(0.50);
    st->latency_p99_ms = pct(0.99);
    st->latency_max_ms = l.empty() ? 0.0 : l.back();
    st->wall_s = v->t_last > v->t_first ? v->t_last - v->t_first : 0.0;
    st->data_s = v->data_s;
    st->realtime_factor = st->wall_s > 0 ? v->data_s / st->wall_s : 0.0;
    st->units_per_s = st->wall_s > 0 ? v->units / st->wall_s : 0.0;
    st->hbm_bytes = v->resident + v->slot_total;
    st->slots = (int32_t)v->slots.size();
    return CDMT_OK;
}

namespace {

// Checkpoint of a beam's stream: the shape it was made with, the counters, then
// the overlap tail, nsub rows of `tail` float4 samples.
struct BeamCheckpoint {
    uint64_t magic;
    int32_t version, nsub;
    int64_t block_len, nbin, nd, tail, seg_total, next_index;
    double f_centre, bw, dm_first, dm_step;
    int32_t ndm, nchan, nint, reserved;
};
constexpr uint64_t kCheckpointMagic = 0x636d646d74626d31ull;   // marks a beam checkpoint

// The beam's blocks are all done (none queued or running); called with the lock held.
bool beam_idle(const cdmt_server_s *v, int beam)
{
    for (const auto &kv : v->reqs)
        if (kv.second.beam == beam && kv.second.state < 2) return false;
    return true;
}

}  // namespace

int cdmt_server_save_beam(cdmt_server_t v, int beam, void *host, int64_t *bytes)
{
    if (!v || !bytes) return sfail(v, CDMT_EINVAL, "NULL server or size");
    std::lock_guard<std::mutex> lk(v->mu);
    if (beam < 0 || beam >= (int)v->beams.size() || !v->beams[beam].active)
        return sfail(v, CDMT_EINVAL, "no beam %d", beam);
    if (!beam_idle(v, beam)) return sfail(v, CDMT_EINVAL, "beam %d has blocks queued or running", beam);
    const Beam &b = v->beams[beam];
    const int64_t need = (int64_t)sizeof(BeamCheckpoint) + (int64_t)b.d.nsub * b.tail * 16;
    if (!host) {
        *bytes = need;
        return CDMT_OK;
    }
    if (*bytes < need) return sfail(v, CDMT_EINVAL, "checkpoint needs %lld bytes", (long long)need);
    BeamCheckpoint h{};
    h.magic = kCheckpointMagic;
    h.version = 1;
    h.nsub = b.d.nsub;
    h.block_len = b.d.block_len;
    h.nbin = b.N;
    h.nd = b.nd;
    h.tail = b.tail;
    h.seg_total = b.seg_total;
    h.next_index = b.next_index;
    h.f_centre = b.d.f_centre_mhz;
    h.bw = b.d.bw_sub_mhz;
    h.dm_first = b.d.dm_first;
    h.dm_step = b.d.dm_step;
    h.ndm = b.d.ndm;
    h.nchan = b.d.nchan;
    h.nint = b.d.nint;
    std::memcpy(host, &h, sizeof h);
    cudaSetDevice(v->device);
    if (b.tail > 0 && cudaMemcpy2D(static_cast<uint8_t *>(host) + sizeof h, (size_t)b.tail * 16, b.stage[b.cur],
                                   (size_t)b.cap * 16, (size_t)b.tail * 16, b.d.nsub, cudaMemcpyDeviceToHost) !=
                          cudaSuccess)
        return sfail(v, CDMT_ECUDA, "copy of the overlap tail failed");
    *bytes = need;
    return CDMT_OK;
}

int cdmt_server_restore_beam(cdmt_server_t v, int beam, const void *host, int64_t bytes)
{
    if (!v || !host) return sfail(v, CDMT_EINVAL, "NULL server or checkpoint");
    std::lock_guard<std::mutex> lk(v->mu);
    if (beam < 0 || beam >= (int)v->beams.size() || !v->beams[beam].active)
        return sfail(v, CDMT_EINVAL, "no beam %d", beam);
    if (!beam_idle(v, beam)) return sfail(v, CDMT_EINVAL, "beam %d has blocks queued or running", beam);
    Beam &b = v->beams[beam];
    BeamCheckpoint h;
    if (bytes < (int64_t)sizeof h) return sfail(v, CDMT_EINVAL, "checkpoint too short");
    std::memcpy(&h, host, sizeof h);
    if (h.magic != kCheckpointMagic || h.version != 1) return sfail(v, CDMT_EINVAL, "not a beam checkpoint");
    if (h.nsub != b.d.nsub || h.block_len != b.d.block_len || h.nbin != b.N || h.nd != b.nd || h.ndm != b.d.ndm ||
        h.nchan != b.d.nchan || h.nint != b.d.nint || h.f_centre != b.d.f_centre_mhz || h.bw != b.d.bw_sub_mhz ||
        h.dm_first != b.d.dm_first || h.dm_step != b.d.dm_step)
        return sfail(v, CDMT_EINVAL, "checkpoint of a stream of another shape");
    if (h.tail < 0 || h.tail >= b.N || bytes < (int64_t)sizeof h + (int64_t)h.nsub * h.tail * 16 ||
        h.seg_total < 0 || h.next_index < 0)
        return sfail(v, CDMT_EINVAL, "checkpoint corrupt or truncated");
    cudaSetDevice(v->device);
    if (cudaStreamSynchronize(b.st) != cudaSuccess) return sfail(v, CDMT_ECUDA, "beam stream failed");
    if (h.tail > 0 && cudaMemcpy2D(b.stage[b.cur], (size_t)b.cap * 16, static_cast<const uint8_t *>(host) + sizeof h,
                                   (size_t)h.tail * 16, (size_t)h.tail * 16, h.nsub, cudaMemcpyHostToDevice) !=
                          cudaSuccess)
        return sfail(v, CDMT_ECUDA, "copy of the overlap tail failed");
    b.tail = h.tail;
    b.seg_total = h.seg_total;
    b.next_index = h.next_index;
    return CDMT_OK;
}

int cdmt_server_reset_stats(cdmt_server_t v)
{
    if (!v) return sfail(nullptr, CDMT_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(v->mu);
    v->lat_ms.clear();
    v->t_first = v->t_last = 0;
    v->data_s = v->units = 0;
    return CDMT_OK;
}

const char *cdmt_server_last_error(cdmt_server_t v) { return v ? v->last_error.c_str() : cdmt_last_error(nullptr); }

int cdmt_server_destroy(cdmt_server_t v)
{
    if (!v) return CDMT_OK;
    v->stop = true;
    v->cv_work.notify_all();
    if (v->sched.joinable()) v->sched.join();
    cudaSetDevice(v->device);
    for (Beam &b : v->beams)
        if (b.active) free_beam(b);
    for (auto &kv : v->reqs)
        if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    for (Slot &sl : v->slots) cudaFree(sl.p);
    cudaGetLastError();
    delete v;
    return CDMT_OK;
}

}  // extern "C"
