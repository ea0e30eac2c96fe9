// FP32 kernels of the coherent-dedispersion hot path (sm_103a).
//
// Forward stage (Sec. 3: "unpack, segment and pad", "forward FFT", "swap halves
// per subband").  The N-point forward DFT of a segment is split as
// N = nchan * M with input n = n1 + nchan * n2 and output F = j + M c':
//   X[j + M c'] = sum_n1 W_nchan^{n1 c'} W_N^{n1 j} sum_n2 x[n1 + nchan n2] W_M^{n2 j}.
//   k_forward_decimated: one CTA per (subband, segment, n1) gathers the
//     decimated series x[k S + n1 + nchan n2], runs the M-point FFT and applies
//     W_N^{n1 j}.
//   k_forward_columns: the nchan-point DFT over n1 for every bin j, written in
//     place with the halves of the spectrum swapped: unshifted channel c' lands
//     in channel slot c = (c' + nchan/2) mod nchan, so that slot c holds bins of
//     increasing frequency of channel c.
//   k_forward_fused: both steps in one persistent launch (M = 4096, nchan <= 16),
//     the column DFTs of a chunk of segments run soon after its transforms, so
//     their intermediate spectra stay in L2; the two launches above serve the
//     other sizes, the batch rounds and the allocation-free entry point.
//
// DM stage (Sec. 3: "complex multiplication with transfer function", "swap
// halves per channel", "backward FFT", "transpose, unpad and detect"), fused in
// k_dedisperse (M = 512, 1024; M = 2048 .. 8192 run k_dedisperse_pair of
// kernels_fp32_pair.cu, the same steps with both polarisations per thread): one
// CTA per (DM tile, subband, segment, channel) keeps the channel's M spectral
// bins of both polarisations in registers (one polarisation per half of the CTA)
// and, for each DM of its tile, multiplies them by the chirp, runs the M-point
// backward FFT, forms |X|^2 + |Y|^2, drops nd/2 samples at each edge, sums nint
// samples and stores the filterbank row segment.  The per-channel swap of halves
// is a factor (-1)^m on the time series, which the detection removes, so it is
// not performed.  Spectra never leave the chip between chirp and detection.
//
// Chirp (Eq. 1, conjugated for dedispersion): bin j of channel c has
// exp(-2 pi i DM K), K = 1e6 D nu^2 / (nu_c^2 (nu_c + nu)).  The planner stores,
// per bin and DM tile, the 32-bit fixed-point phase a = -DM_0 K and step
// b = -dDM K (in cycles, computed in FP64); DM number d of the tile then has
// phase a + d b exactly modulo 2^32.  Lists that are not evenly spaced use the
// FP64 product DM K per bin and DM instead.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "cdmt_internal.h"
#include "fft_core.cuh"
#include "tc_ptx.cuh"

namespace cdmt {

constexpr float kTwoPiOver2p32 = 1.46291807926715968e-9f;  // 2 pi / 2^32

constexpr uint64_t kTmaWaitNs = 50ull * 1000 * 1000;   // a CTA's input copy takes microseconds
constexpr uint32_t kTmaWaitPolls = 1u << 26;

// ---------------------------------------------------------------------------
// I8: char4 samples (X re, X im, Y re, Y im) times the subband's scale, in FP32.
// TMA: the decimated series x[n1 + nchan n2], n2 < M, comes into the exchange
// buffer by TMA instead of per-thread loads: the input is a 3-D tensor map of
// rows of nchan samples ([subband][row][nchan samples]), and each of M / 256
// boxes takes 16 bytes of 256 rows, so one thread issues the whole gather and the
// threads read their points from shared memory.  Float samples: the box is the
// sample of column n1.  int8 samples (4 bytes, nchan >= 4): the box is the four
// samples of columns 4 (n1 / 4) .. + 3, of which the CTA keeps column n1.  A wait that gives up (never expected) sets *status.  With no loads in
// flight in registers the M = 4096 form fits three CTAs per SM (80 registers,
// a few bytes of spill): 3.12 against 3.48 ms per 64-subband step at two.
// This thread's 16 points of each polarisation of the decimated series staged in ex by TMA.
template <int R, bool I8>
__device__ __forceinline__ void fwd_read_staged(const float4 *ex, int n1, float sc, float2 *x, float2 *y, int t)
{
    constexpr int T = Fft3<R>::T;
    if constexpr (I8) {
        const char4 *q = reinterpret_cast<const char4 *>(ex) + (n1 & 3);
        #pragma unroll
        for (int j2 = 0; j2 < 16; j2++) {
            // products rounded on their own, as in the per-thread loads
            const char4 v = q[4 * (j2 * T + t)];
            x[j2] = make_float2(__fmul_rn((float)v.x, sc), __fmul_rn((float)v.y, sc));
            y[j2] = make_float2(__fmul_rn((float)v.z, sc), __fmul_rn((float)v.w, sc));
        }
    } else {
        #pragma unroll
        for (int j2 = 0; j2 < 16; j2++) {
            const float4 v = ex[j2 * T + t];
            x[j2] = make_float2(v.x, v.y);
            y[j2] = make_float2(v.z, v.w);
        }
    }
}

// One thread issues the TMA gather of the decimated series of phase n1 (rows row0 .. row0 + M - 1
// of subband s) into ex, completing on bar.
template <int R, bool I8>
__device__ __forceinline__ void fwd_issue_gather(float4 *ex, uint64_t *bar, const CUtensorMap *tmap, int n1, int row0,
                                                 int s)
{
    constexpr int M = Fft3<R>::M;
    tc::mbar_arrive_expect_tx(bar, (uint32_t)(sizeof(float4) * M));
    const int c0 = I8 ? 16 * (n1 / 4) : 4 * n1;   // bytes of int8, floats of float4
    for (int b = 0; b < M / 256; b++) tc::tma_load_3d(ex + 256 * b, tmap, c0, row0 + 256 * b, s, bar);
}

// The M-point transform of a decimated series (x, y: this thread's points), times W_N^{n1 j},
// stored at dst.  ex is free on entry.
template <int R>
__device__ __forceinline__ void fwd_transform_store(float2 *x, float2 *y, float4 *ex, const float2 *__restrict__ tw_a,
                                                    const float2 *__restrict__ tw_b, const float2 *__restrict__ tw_n,
                                                    int n1, float4 *__restrict__ dst, int t)
{
    using F = Fft3<R>;
    F::template pass_a<-1>(x, y, ex, tw_a, t);
    __syncthreads();
    F::template pass_b<-1>(x, y, ex, tw_b, t);
    __syncthreads();
    // W_N^{n1 j} for j = beta + 256 m2 as W_N^{n1 beta} W_N^{256 n1 m2}: one scattered table read per
    // beta (16 / R per thread) and warp-uniform ones for the second factor, instead of 16 scattered
    // reads that each use 8 bytes of a 32-byte sector
    F::template pass_c<-1>(ex, t, [&](int beta, int m2, float2 a, float2 b) {
        const float2 w = cmul(__ldg(tw_n + n1 * beta), __ldg(tw_n + 256 * n1 * m2));
        dst[beta + 256 * m2] = pack(cmul(a, w), cmul(b, w));
    });
}

template <int R, bool I8, bool TMA = false>
__global__ void __launch_bounds__(16 * R, (R == 16 && TMA) ? 3 : 1)   // TMA, M = 4096: 3 CTAs per SM
k_forward_decimated(const __grid_constant__ CUtensorMap tmap, const void *__restrict__ in,
                    const float *__restrict__ scale, float4 *__restrict__ spec, const float2 *__restrict__ tw_a,
                    const float2 *__restrict__ tw_b, const float2 *__restrict__ tw_n, int64_t nsamp, int64_t nvalid,
                    int nchan, int64_t k0, int kc, const int *__restrict__ round_dev, int64_t nseg,
                    int *__restrict__ status)
{
    // batches: the chunk's first segment is round * kc, read from device memory;
    // segments past the end of the input are skipped
    if (round_dev) k0 = (int64_t)(*round_dev) * kc;
    if (k0 + (int64_t)blockIdx.y >= nseg) return;
    using F = Fft3<R>;
    constexpr int M = F::M, T = F::T;
    extern __shared__ __align__(128) float4 smem[];
    float4 *ex = smem;   // the exchange buffer; the pass twiddles are read through the cache

    const int t = threadIdx.x;
    const int n1 = blockIdx.x;
    const int kk = blockIdx.y;
    const int s = blockIdx.z;

    const int64_t s0 = (int64_t)s * nsamp + (k0 + kk) * nvalid + n1;
    float2 x[16], y[16];
    if constexpr (TMA) {
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem + M);
        if (t == 0) {
            tc::mbar_init(bar, 1);
            tc::fence_mbar_init();
        }
        __syncthreads();
        // segments start on whole rows
        if (t == 0) fwd_issue_gather<R, I8>(ex, bar, &tmap, n1, (int)(((k0 + kk) * nvalid) / nchan), s);
        if (!tc::mbar_wait(bar, 0, kTmaWaitNs, kTmaWaitPolls)) {
            if (status) atomicExch(status, 1);
            (void)tc::mbar_wait(bar, 0, kTmaWaitNs, kTmaWaitPolls);   // a late copy lands before the CTA leaves
        }
        fwd_read_staged<R, I8>(ex, n1, I8 ? __ldg(scale + s) : 1.f, x, y, t);
        __syncthreads();   // every thread holds its points before pass A writes the buffer
    } else if constexpr (I8) {
        const char4 *src = static_cast<const char4 *>(in) + s0;
        const float sc = __ldg(scale + s);
        #pragma unroll
        for (int j2 = 0; j2 < 16; j2++) {
            // products rounded on their own (never contracted into the FFT's additions), so the
            // result equals that of the dequantised float32 voltages
            const char4 v = __ldg(src + (int64_t)nchan * (j2 * T + t));
            x[j2] = make_float2(__fmul_rn((float)v.x, sc), __fmul_rn((float)v.y, sc));
            y[j2] = make_float2(__fmul_rn((float)v.z, sc), __fmul_rn((float)v.w, sc));
        }
    } else {
        const float4 *src = static_cast<const float4 *>(in) + s0;
        #pragma unroll
        for (int j2 = 0; j2 < 16; j2++) {
            const float4 v = __ldg(src + (int64_t)nchan * (j2 * T + t));
            x[j2] = make_float2(v.x, v.y);
            y[j2] = make_float2(v.z, v.w);
        }
    }
    fwd_transform_store<R>(x, y, ex, tw_a, tw_b, tw_n, n1, spec + (((int64_t)s * kc + kk) * nchan + n1) * M, t);
}

// The nchan-point DFT over n1 (stride m) of one bin j, col = &spec[segment][n1 = 0][j], in place,
// with the halves swapped: unshifted channel c' goes to slot (c' + NC / 2) mod NC.  CG: the loads
// go through L2 only (spectra that other CTAs of the same launch have just stored).
template <int NC, bool CG = false>
__device__ __forceinline__ void column_dft(float4 *col, const float2 *__restrict__ tw_n, int m, int64_t nbin)
{
    float2 x[NC], y[NC];
    #pragma unroll
    for (int n1 = 0; n1 < NC; n1++) {
        const float4 v = CG ? __ldcg(col + (int64_t)n1 * m) : col[(int64_t)n1 * m];
        x[n1] = make_float2(v.x, v.y);
        y[n1] = make_float2(v.z, v.w);
    }
    if constexpr (NC <= 16) {
        dft_r<NC, -1>(x);
        dft_r<NC, -1>(y);
    } else {
        // NC = 32: two 16-point DFTs (even / odd n1) and one radix-2 step with
        // twiddles W_32^k = W_N^{k N / 32}
        float2 ex_[16], ox[16], ey[16], oy[16];
        #pragma unroll
        for (int i = 0; i < 16; i++) {
            ex_[i] = x[2 * i]; ox[i] = x[2 * i + 1];
            ey[i] = y[2 * i]; oy[i] = y[2 * i + 1];
        }
        dft16<-1>(ex_); dft16<-1>(ox); dft16<-1>(ey); dft16<-1>(oy);
        #pragma unroll
        for (int k = 0; k < 16; k++) {
            float2 w = __ldg(tw_n + (int64_t)k * (nbin / 32));
            float2 a = cmul(ox[k], w), b = cmul(oy[k], w);
            x[k] = cadd(ex_[k], a); x[k + 16] = csub(ex_[k], a);
            y[k] = cadd(ey[k], b); y[k + 16] = csub(ey[k], b);
        }
    }
    #pragma unroll
    for (int cp = 0; cp < NC; cp++) {
        const int c = (cp + NC / 2) % NC;
        col[(int64_t)c * m] = pack(x[cp], y[cp]);
    }
}

// nchan-point DFT over n1 (stride M) for every bin j; in place.
template <int NC>
__global__ void __launch_bounds__(256) k_forward_columns(float4 *__restrict__ spec, const float2 *__restrict__ tw_n,
                                                         int m, int64_t nbin)
{
    const int j = blockIdx.x * 256 + threadIdx.x;
    if (j >= m) return;
    column_dft<NC>(spec + ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * nbin + j, tw_n, m, nbin);
}

// ---------------------------------------------------------------------------
// The forward stage in one persistent launch (TMA gather, M = 4096, nchan <= 16).  CTAs take
// work items from a queue whose tickets sync[0] hands out in order: D items are the decimated
// transforms of k_forward_decimated (segment, n1), C items the column DFTs of k_forward_columns
// (segment, block of 256 bins).  The segments, subband by subband, form chunks of kFwdChunk; the
// queue puts the D items of chunk i + kFwdLag before the C items of chunk i, and a C item first
// waits until all D items of its chunk have stored their spectra (sync[1 + i] counts them).  So
// the transforms' output is read back from L2 shortly after it was written, and the stage moves
// its input once from HBM and its output once to HBM, where the two launches move the spectra
// through HBM three times.
// Each CTA holds two tickets, the item it works on and the next one (fetched while it works), and
// runs its items in ticket order.  A C item waits only on D items with smaller tickets, and D items
// wait on nothing but their own copy, so every wait ends: of the waiting items take the one with
// the smallest ticket.  Each D item it waits on has a smaller ticket, so it has been handed out
// (tickets go out in order), and it is not the next item of a CTA whose current item waits (that
// item's ticket would be smaller still): it is done, running, or next after an item that runs.
// This holds however many of the grid's CTAs are resident at a time, since only running CTAs take
// tickets.  The waits are bounded all the same: one that gives up (never expected) sets *status
// and skips its item.
constexpr int kFwdChunk = 2;   // segments per chunk
constexpr int kFwdLag = 16;    // chunks between a chunk's D items and its C items in the queue

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// bounded wait until *p >= need (one thread)
__device__ __forceinline__ int wait_count(const int *p, int need)
{
    const uint64_t t0 = tc::globaltimer_ns();
    for (uint32_t it = 0; it < kTmaWaitPolls; it++) {
        if (ld_acquire_gpu(p) >= need) return 1;
        if ((it & 15) == 15 && tc::globaltimer_ns() - t0 > kTmaWaitNs) return 0;
        __nanosleep(64);
    }
    return 0;
}

template <int R, bool I8>
__global__ void __launch_bounds__(16 * R, 3)
k_forward_fused(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ scale, float4 *__restrict__ spec,
                const float2 *__restrict__ tw_a, const float2 *__restrict__ tw_b, const float2 *__restrict__ tw_n,
                int64_t nvalid, int nchan, int64_t k0, int kc, int nsub, int *__restrict__ sync,
                int *__restrict__ status)
{
    constexpr int M = Fft3<R>::M;
    extern __shared__ __align__(128) float4 smem[];
    float4 *ex = smem;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + M);
    int *shared_word = reinterpret_cast<int *>(bar + 1);   // [0] the CTA's ticket, [1] a C item's wait result
    const int t = threadIdx.x;
    const int nsegs = nsub * kc;
    const int nchunk = (nsegs + kFwdChunk - 1) / kFwdChunk;
    const int nd_items = kFwdChunk * nchan, nc_items = kFwdChunk * (M / 256);   // per chunk
    const int lag = min(kFwdLag, nchunk);
    const int64_t head = (int64_t)lag * nd_items;                              // D items of chunks 0 .. lag - 1
    const int64_t mid = (int64_t)(nchunk - lag) * (nd_items + nc_items);     // D(k), then C(k - lag)
    const int64_t total = (int64_t)nchunk * (nd_items + nc_items);
    if (t == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    uint32_t nd_run = 0;   // D items this CTA has run: the parity of the mbarrier's phase
    int next = t == 0 ? atomicAdd(sync, 1) : 0;   // thread 0 holds the ticket after the current one
    for (;;) {
        __syncthreads();   // the previous item is done with ex and the shared words
        if (t == 0) {
            shared_word[0] = next;
            next = atomicAdd(sync, 1);   // in flight while the CTA works on this item
        }
        __syncthreads();
        const int64_t tk = shared_word[0];
        if (tk >= total) break;
        bool is_d;
        int chunk, idx;
        if (tk < head) {
            is_d = true;
            chunk = (int)(tk / nd_items);
            idx = (int)(tk % nd_items);
        } else if (tk - head < mid) {
            const int64_t u = tk - head;
            const int k = lag + (int)(u / (nd_items + nc_items)), r = (int)(u % (nd_items + nc_items));
            is_d = r < nd_items;
            chunk = is_d ? k : k - lag;
            idx = is_d ? r : r - nd_items;
        } else {
            const int64_t u = tk - head - mid;
            is_d = false;
            chunk = nchunk - lag + (int)(u / nc_items);
            idx = (int)(u % nc_items);
        }
        if (is_d) {
            const int g = chunk * kFwdChunk + idx / nchan, n1 = idx % nchan;
            if (g < nsegs) {   // the last chunk's missing segment counts as done
                const int s = g / kc, kk = g % kc;
                if (t == 0) {
                    tc::fence_async_smem();   // the previous item's accesses to ex before the copy into it
                    fwd_issue_gather<R, I8>(ex, bar, &tmap, n1, (int)(((k0 + kk) * nvalid) / nchan), s);
                }
                if (!tc::mbar_wait(bar, nd_run & 1, kTmaWaitNs, kTmaWaitPolls)) {
                    if (status) atomicExch(status, 1);
                    (void)tc::mbar_wait(bar, nd_run & 1, kTmaWaitNs, kTmaWaitPolls);
                }
                nd_run++;
                float2 x[16], y[16];
                fwd_read_staged<R, I8>(ex, n1, I8 ? __ldg(scale + s) : 1.f, x, y, t);
                __syncthreads();   // every thread holds its points before pass A writes the buffer
                fwd_transform_store<R>(x, y, ex, tw_a, tw_b, tw_n, n1, spec + ((int64_t)g * nchan + n1) * M, t);
            }
            __syncthreads();   // all of the item's stores precede its count
            if (t == 0) {
                __threadfence();
                atomicAdd(sync + 1 + chunk, 1);
            }
        } else {
            const int g = chunk * kFwdChunk + idx / (M / 256), jb = idx % (M / 256);
            if (g >= nsegs) continue;
            if (t == 0) shared_word[1] = wait_count(sync + 1 + chunk, nd_items);
            __syncthreads();
            if (!shared_word[1]) {
                if (t == 0 && status) atomicExch(status, 1);
                continue;
            }
            float4 *col = spec + (int64_t)g * nchan * M + 256 * jb + t;
            const int64_t nbin = (int64_t)nchan * M;
            switch (nchan) {
            case 2: column_dft<2, true>(col, tw_n, M, nbin); break;
            case 4: column_dft<4, true>(col, tw_n, M, nbin); break;
            case 8: column_dft<8, true>(col, tw_n, M, nbin); break;
            default: column_dft<16, true>(col, tw_n, M, nbin); break;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// One CTA of 2T threads per (DM tile, subband, segment, channel): threads
// [0, T) carry polarisation X, [T, 2T) polarisation Y.  Each thread keeps its
// 16 spectral bins of its polarisation in registers for the whole DM tile.
// Shared memory holds the phase words of the channel's M bins, the twiddles,
// one exchange buffer per polarisation and one detected-power row per
// polarisation.
// UNIFORM: the phase table holds (a, b) per bin for the tile; otherwise it
// holds K per bin as double and the DM values come from dm_list.
template <int R, bool UNIFORM>
__global__ void __launch_bounds__(32 * R, 16 / R)
k_dedisperse(const float4 *__restrict__ spec, const uint2 *__restrict__ nco, const double *__restrict__ ktab,
             const double *__restrict__ dm_list, const float2 *__restrict__ tw_a, const float2 *__restrict__ tw_b,
             float *__restrict__ out, int nsub, int kc, int64_t k0, int nchan, int ndm, int dm_tile, int nd,
             int nint, int64_t nout, float scale, const int *__restrict__ round_dev, int64_t nseg, int dm_off,
             int dm_cnt, int64_t tlim)
{
    using F = Fft3<R>;
    constexpr int M = F::M, T = F::T, NT = 2 * T;
    extern __shared__ float4 smem[];
    float2 *ex = reinterpret_cast<float2 *>(smem);        // [2][M] exchange buffers
    uint2 *ph = reinterpret_cast<uint2 *>(ex + 2 * M);   // M phase words (a, b) or K as double
    float2 *ta = reinterpret_cast<float2 *>(ph + M);
    float2 *tb = ta + F::NTA;
    float *ib = reinterpret_cast<float *>(tb + F::NTB);  // [2][M] detected powers

    const int tid = threadIdx.x;
    const int pol = tid / T, t = tid % T;
    int64_t item = blockIdx.x;
    const int c = (int)(item % nchan); item /= nchan;
    const int kk = (int)(item % kc); item /= kc;
    const int s = (int)(item % nsub); item /= nsub;
    const int tile = (int)item;
    const int dm0 = tile * dm_tile + dm_off;          // first DM of this tile's range
    const int ndt = min(dm_cnt, ndm - dm0);
    if (ndt <= 0) return;
    // batches: this chunk's segments start at round * kc; none past the end of the input
    if (round_dev && (int64_t)(*round_dev) * kc + kk >= nseg) return;
    // output samples of this segment before the filterbank's end (position tlim on)
    const int64_t room = tlim - (k0 + kk) * (int64_t)((M - nd) / nint);
    const int ulim = room <= 0 ? 0 : (int)(room < (M - nd) / nint ? room : (M - nd) / nint);
    if (ulim == 0) return;

    const float4 *src = spec + (((int64_t)s * kc + kk) * nchan + c) * M;
    float2 xr[16];
    #pragma unroll
    for (int j2 = 0; j2 < 16; j2++) {
        float4 v = __ldg(src + j2 * T + t);
        xr[j2] = pol ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
    }
    if constexpr (UNIFORM) {
        const uint2 *p = nco + ((int64_t)tile * nsub + s) * (int64_t)nchan * M + (int64_t)c * M;
        for (int i = tid; i < M; i += NT) ph[i] = p[i];
    } else {
        const uint2 *p = reinterpret_cast<const uint2 *>(ktab + ((int64_t)s * nchan + c) * M);
        for (int i = tid; i < M; i += NT) ph[i] = p[i];
    }
    for (int i = tid; i < F::NTA; i += NT) ta[i] = tw_a[i];
    for (int i = tid; i < F::NTB; i += NT) tb[i] = tw_b[i];
    __syncthreads();

    float2 *exp_ = ex + pol * M;
    float *ibp = ib + pol * M;
    const int half = nd / 2;
    const int seglen = (M - nd) / nint;
    const int64_t rows = (int64_t)nsub * nchan;
    const int64_t obase = (int64_t)(s * nchan + c) * nout + (k0 + kk) * seglen;
    // conflict-free integration: lane l starts its nint-sample sum at a rotated offset
    const bool pow2 = (nint & (nint - 1)) == 0 && nint <= 32;
    const int rot = pow2 ? (((tid & 31) * nint) >> 5) : 0;

    for (int d = 0; d < ndt; d++) {
        float2 x[16];
        double dmv = 0.0;
        if constexpr (!UNIFORM) dmv = dm_list[dm0 + d];
        #pragma unroll
        for (int j2 = 0; j2 < 16; j2++) {
            const int j = j2 * T + t;
            float sn, cs;
            if constexpr (UNIFORM) {
                uint2 ab = ph[j];
                int32_t p = (int32_t)(ab.x + (uint32_t)(dm_off + d) * ab.y);
                __sincosf((float)p * kTwoPiOver2p32, &sn, &cs);
            } else {
                double kj = __hiloint2double((int)ph[j].y, (int)ph[j].x);
                double cyc = dmv * kj;
                cyc -= rint(cyc);
                __sincosf(-6.283185307179586f * (float)cyc, &sn, &cs);
            }
            x[j2] = make_float2(xr[j2].x * cs - xr[j2].y * sn, xr[j2].x * sn + xr[j2].y * cs);
        }
        F::template pass_a1<+1>(x, exp_, ta, t);
        __syncthreads();
        F::template pass_b1<+1>(x, exp_, tb, t);
        __syncthreads();
        F::template pass_c1<+1>(exp_, t, [&](int m, float2 a) { ibp[m] = fmaf(a.x, a.x, a.y * a.y); });
        __syncthreads();
        float *orow = out + ((int64_t)tile * dm_cnt + d) * rows * nout + obase;
        for (int u = tid; u < ulim; u += NT) {
            const float *px = ib + half + u * nint;
            const float *py = px + M;
            float acc = 0.f;
            if (pow2) {
                for (int q = 0; q < nint; q++) {
                    const int qq = (q + rot) & (nint - 1);
                    acc += px[qq] + py[qq];
                }
            } else {
                for (int q = 0; q < nint; q++) acc += px[q] + py[q];
            }
            orow[u] = acc * scale;
        }
    }
}

// M = 8192: R = 32 (k_forward_decimated; the DM stage is k_dedisperse_pair)
constexpr int kR8k = 32;

// ---------------------------------------------------------------------------
// launchers

template <int R> static size_t smem_forward() { return sizeof(float4) * Fft3<R>::M; }
template <int R> static size_t smem_forward_tma() { return sizeof(float4) * Fft3<R>::M + 16; }   // + mbarrier
template <int R> static size_t smem_forward_fused() { return sizeof(float4) * Fft3<R>::M + 16; }   // + mbarrier, 2 words
template <int R> static size_t smem_dedisp()
{
    using F = Fft3<R>;
    return sizeof(float2) * 2 * F::M + sizeof(uint2) * F::M + sizeof(float2) * (F::NTA + F::NTB) + sizeof(float) * 2 * F::M;
}


template <int R> static cudaError_t set_attrs()
{
    cudaError_t e = cudaFuncSetAttribute(k_forward_decimated<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_forward<R>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_forward_decimated<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_forward<R>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_forward_decimated<R, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_forward_tma<R>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_forward_decimated<R, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_forward_tma<R>());
    if (e != cudaSuccess) return e;
    if constexpr (R == 16) {
        e = cudaFuncSetAttribute(k_forward_fused<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_forward_fused<R>());
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_forward_fused<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_forward_fused<R>());
        if (e != cudaSuccess) return e;
    }
    if constexpr (R == 8 || R == 16) {
        return fp32_pair_prepare(R);   // the DM stage at M = 2048 and 4096 is k_dedisperse_pair
    } else {
        e = cudaFuncSetAttribute(k_dedisperse<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_dedisp<R>());
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_dedisperse<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_dedisp<R>());
    }
}

static cudaError_t set_attrs_8k()
{
    cudaError_t e = cudaFuncSetAttribute(k_forward_decimated<kR8k, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_forward<kR8k>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_forward_decimated<kR8k, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_forward<kR8k>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_forward_decimated<kR8k, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_forward_tma<kR8k>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_forward_decimated<kR8k, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_forward_tma<kR8k>());
    if (e == cudaSuccess) e = fp32_pair_prepare(kR8k);
    return e;
}

cudaError_t fp32_prepare(int r)
{
    switch (r) {
    case 2: return set_attrs<2>();
    case 4: return set_attrs<4>();
    case 8: return set_attrs<8>();
    case 16: return set_attrs<16>();
    case kR8k: return set_attrs_8k();
    default: return cudaErrorInvalidValue;
    }
}

size_t fp32_dedisp_smem(int r)
{
    switch (r) {
    case 2: return smem_dedisp<2>();
    case 4: return smem_dedisp<4>();
    case 8: return fp32_pair_smem(8);
    case 16: return fp32_pair_smem(16);
    case kR8k: return fp32_pair_smem(kR8k);
    default: return 0;
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (looked up once per process)
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// The input as the forward kernel's TMA sees it: [nsub][nsamp / nchan rows][nchan samples], row
// pitch nchan samples, subband pitch nsamp samples; boxes of 16 bytes of 256 rows (one float4
// sample, or four int8 samples).  Rows past nsamp / nchan are never read: a segment ends at or
// before sample nsamp of its subband.  int8 rows need nchan >= 4 (16-byte row pitch).
static bool input_tmap(CUtensorMap &tm, const ForwardArgs &a)
{
    const PFN_cuTensorMapEncodeTiled_v12000 fn = tmap_encoder();
    const uint64_t es_bytes = a.i8 ? 4 : 16;
    if (!fn || reinterpret_cast<uintptr_t>(a.in) % 16 || a.nsamp / a.nchan < 1) return false;
    if (a.i8 && (a.nchan < 4 || (a.nsamp * 4) % 16)) return false;
    cuuint64_t dims[3] = {a.i8 ? 4ull * (cuuint64_t)a.nchan : 4ull * (cuuint64_t)a.nchan,
                          (cuuint64_t)(a.nsamp / a.nchan), (cuuint64_t)a.nsub};
    cuuint64_t strides[2] = {es_bytes * (cuuint64_t)a.nchan, es_bytes * (cuuint64_t)a.nsamp};
    cuuint32_t box[3] = {a.i8 ? 16u : 4u, 256, 1}, es[3] = {1, 1, 1};
    return fn(&tm, a.i8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(a.in),
              dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int R> static void launch_forward(const ForwardArgs &a, cudaStream_t st)
{
    dim3 g(a.nchan, a.kc, a.nsub);
    const int64_t nseg = a.round_dev ? a.nseg : INT64_MAX;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    const bool tma = input_tmap(tm, a);
    if (a.i8 && tma)
        k_forward_decimated<R, true, true><<<g, Fft3<R>::T, smem_forward_tma<R>(), st>>>(
            tm, a.in, a.scale, a.spec, a.tw_a, a.tw_b, a.tw_n, a.nsamp, a.nvalid, a.nchan, a.k0, a.kc, a.round_dev,
            nseg, a.status);
    else if (a.i8)
        k_forward_decimated<R, true><<<g, Fft3<R>::T, smem_forward<R>(), st>>>(
            tm, a.in, a.scale, a.spec, a.tw_a, a.tw_b, a.tw_n, a.nsamp, a.nvalid, a.nchan, a.k0, a.kc, a.round_dev,
            nseg, a.status);
    else if (tma)
        k_forward_decimated<R, false, true><<<g, Fft3<R>::T, smem_forward_tma<R>(), st>>>(
            tm, a.in, a.scale, a.spec, a.tw_a, a.tw_b, a.tw_n, a.nsamp, a.nvalid, a.nchan, a.k0, a.kc, a.round_dev,
            nseg, a.status);
    else
        k_forward_decimated<R, false><<<g, Fft3<R>::T, smem_forward<R>(), st>>>(
            tm, a.in, a.scale, a.spec, a.tw_a, a.tw_b, a.tw_n, a.nsamp, a.nvalid, a.nchan, a.k0, a.kc, a.round_dev,
            nseg, a.status);
}

template <int NC> static void launch_columns(const ForwardArgs &a, cudaStream_t st)
{
    const int m = (int)(a.nbin / NC);
    dim3 g((m + 255) / 256, a.kc, a.nsub);
    k_forward_columns<NC><<<g, 256, 0, st>>>(a.spec, a.tw_n, m, a.nbin);
}

// The one-launch forward stage where it applies (M = 4096, nchan 2..16, the TMA gather, a queue
// buffer of 1 + chunks words, no batch rounds, a stream that is not being captured into a graph);
// cudaErrorNotSupported where it does not.  A grid of at most the CTAs that fit on the device at
// once, launched as an ordinary kernel: its waits end whichever of its CTAs are resident (see
// k_forward_fused), and a cooperative launch, which needs the whole grid resident, would hold the
// stage back until other streams' kernels (a server's other beams) have left the GPU.
static cudaError_t launch_forward_fused(const ForwardArgs &a, cudaStream_t st)
{
    if (!a.sync || a.r != 16 || a.round_dev || a.nchan < 2 || a.nchan > 16 || a.nsm < 1) return cudaErrorNotSupported;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return cudaErrorNotSupported;
    }
    const int64_t nsegs = (int64_t)a.nsub * a.kc;
    const int64_t nchunk = (nsegs + kFwdChunk - 1) / kFwdChunk;
    if (nsegs < 1 || 1 + nchunk > a.sync_n || nsegs * (a.nchan + 16) > INT32_MAX) return cudaErrorNotSupported;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    if (!input_tmap(tm, a)) return cudaErrorNotSupported;
    const void *fn = a.i8 ? reinterpret_cast<const void *>(k_forward_fused<16, true>)
                          : reinterpret_cast<const void *>(k_forward_fused<16, false>);
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, Fft3<16>::T, smem_forward_fused<16>());
    if (e != cudaSuccess || occ < 1) return e != cudaSuccess ? e : cudaErrorNotSupported;
    const int64_t total = nchunk * (int64_t)kFwdChunk * (a.nchan + 16);
    const unsigned grid = (unsigned)std::min<int64_t>(total, (int64_t)occ * a.nsm);
    if ((e = cudaMemsetAsync(a.sync, 0, sizeof(int) * (size_t)(1 + nchunk), st)) != cudaSuccess) return e;
    if (a.i8)
        k_forward_fused<16, true><<<grid, Fft3<16>::T, smem_forward_fused<16>(), st>>>(
            tm, a.scale, a.spec, a.tw_a, a.tw_b, a.tw_n, a.nvalid, a.nchan, a.k0, a.kc, a.nsub, a.sync, a.status);
    else
        k_forward_fused<16, false><<<grid, Fft3<16>::T, smem_forward_fused<16>(), st>>>(
            tm, a.scale, a.spec, a.tw_a, a.tw_b, a.tw_n, a.nvalid, a.nchan, a.k0, a.kc, a.nsub, a.sync, a.status);
    return cudaGetLastError();
}

cudaError_t fp32_forward(const ForwardArgs &a, cudaStream_t st)
{
    const cudaError_t ef = launch_forward_fused(a, st);
    if (ef != cudaErrorNotSupported) return ef;
    switch (a.r) {
    case 2: launch_forward<2>(a, st); break;
    case 4: launch_forward<4>(a, st); break;
    case 8: launch_forward<8>(a, st); break;
    case 16: launch_forward<16>(a, st); break;
    case kR8k: launch_forward<kR8k>(a, st); break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (a.nchan) {
    case 2: launch_columns<2>(a, st); break;
    case 4: launch_columns<4>(a, st); break;
    case 8: launch_columns<8>(a, st); break;
    case 16: launch_columns<16>(a, st); break;
    case 32: launch_columns<32>(a, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int R, bool U> static void launch_dedisp(const DedispArgs &a, cudaStream_t st)
{
    const int64_t ntile = (a.ndm + a.dm_tile - 1) / a.dm_tile;
    const int64_t nblk = ntile * a.nsub * a.kc * a.nchan;
    k_dedisperse<R, U><<<(unsigned)nblk, 2 * Fft3<R>::T, smem_dedisp<R>(), st>>>(
        a.spec, a.nco, a.ktab, a.dm_list, a.tw_a, a.tw_b, a.out, a.nsub, a.kc, a.k0, a.nchan, a.ndm, a.dm_tile,
        a.nd, a.nint, a.nout, a.scale, a.round_dev, a.nseg, a.dm_off, a.dm_cnt > 0 ? a.dm_cnt : a.dm_tile, a.tlim);
}

cudaError_t fp32_dedisperse(const DedispArgs &a, cudaStream_t st)
{
    if (a.r == kR8k) return fp32_dedisperse_pair(a, st);
    switch (a.r * 2 + (a.uniform ? 1 : 0)) {
    case 4 + 1: launch_dedisp<2, true>(a, st); break;
    case 4: launch_dedisp<2, false>(a, st); break;
    case 8 + 1: launch_dedisp<4, true>(a, st); break;
    case 8: launch_dedisp<4, false>(a, st); break;
    case 16 + 1:
    case 16:
    case 32 + 1:
    case 32: return fp32_dedisperse_pair(a, st);   // M = 2048, 4096: both polarisations per thread
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cdmt
