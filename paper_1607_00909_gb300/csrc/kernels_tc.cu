// Tensor-core form of the DM stage (sm_103a tcgen05), for channels of
// M = 64 P bins, P = 64 (M = 4096) or P = 32 (M = 2048).
//
// The backward M-point DFT of each channel is split as M = P x 64 (input
// j = 64 j_hi + j_lo, output m = m0 + P m1):
//   pass A  for every j_lo:  y[m0] = sum_j_hi x[64 j_hi + j_lo] W_P^{j_hi m0},  y *= W_M^{j_lo m0}
//   pass B  for every m0:    z[m1] = sum_j_lo y_j_lo[m0] W_64^{j_lo m1}
// Each pass is one real GEMM on the tensor cores with the real form of a DFT
// matrix (real and imaginary parts interleaved on its input side) as one
// operand, half-precision operands and an FP32 accumulator in tensor memory:
//   pass A  D[(j_lo, pol)][(re/im, m0)]  = X[(j_lo, pol)][(j_hi, re/im)] . F_P     128 x 2P x 2P
//   pass B  D[(m1, re/im)][(pol, m0)]    = F_64^T . Y[(j_lo, re/im)][(pol, m0)]     128 x 2P x 128
// F_P sits in shared memory (output parts split: real parts of m = 0..P-1,
// then imaginary parts) as pass A's B operand, and F_64 in tensor memory
// (output parts interleaved) as pass B's A operand.  Between the passes each thread reads
// its own pass-A row from tensor memory, applies the W_4096 twiddles with
// packed FP32 pairs (two consecutive m0 per instruction) and writes the row as
// a K-row of pass B's data operand (MN-major), so the transposition costs only
// 16-byte shared-memory stores.  Pass-A rows pair the polarisations of one
// j_lo in neighbouring lanes, which share their twiddle loads.  Pass B's
// orientation puts the real and imaginary parts of one time
// sample in neighbouring TMEM lanes and both polarisations and consecutive
// time samples in one thread's columns, so detection and integration run in
// registers: one fused multiply-add per value, one shuffle per output.  The
// time shift by n_d / 2 that drops the wrapped overlap (Sec. 2) is folded into
// the chirp phase (a circular shift of the output is a phase ramp on the
// bins, exact in the 32-bit fixed-point phase), so integration windows start
// on multiples of nint; nint must divide 32.  The two sizes differ in their
// pipes: M = 4096 runs three pipes of 256 threads (128-column accumulators),
// M = 2048 six pipes of 128 threads (64-column accumulators).
//
// The chirp (Eq. 1, conjugated) and the data scaling run in FP32 before the
// rounding to half precision; the chirp phase comes from the same FP64-derived
// fixed-point (phase, step) words as in the FP32 form.  Each CTA scales its
// spectrum by a power of two so that every half-precision operand stays below
// 2^15 whatever the signal; the scale is undone exactly on the output.
//
// Work split: one CTA per (DM tile, subband, segment, channel).  FP16: three
// pipes of 256 threads take every third DM of the tile, each with its own
// operand buffer, tensor-memory columns and mbarrier, so the tensor core works
// on one pipe's GEMM while the others do their FP32 work.
//
// BF16 operands carry 8 mantissa bits, too few for the 2e-3 error target, so in
// BF16 mode both the data and the DFT matrix are split into hi + lo parts and
// each K-step issues three MMAs (hi*hi + lo*hi + hi*lo); the CTA then runs one
// DM at a time with all 512 threads (two operand sets do not fit).
#include <algorithm>

#include "cdmt_internal.h"
#include "fft_core.cuh"
#include "tc_ptx.cuh"

namespace cdmt {

namespace {

constexpr uint32_t kLboA = 128;                  // K-major operands: stride between 8-element K cores
constexpr uint32_t kSboB = 128;                  // pass-B data (MN-major): stride between 8-element N cores
constexpr uint32_t kF64Sbo = 2048;               // F_64 in global memory: K-major, 128 x 128 half
constexpr uint32_t kF64Bytes = 32768;
constexpr uint32_t kWaitPolls = 1u << 26;          // backstop on polls
constexpr uint64_t kWaitNs = 50ull * 1000 * 1000;  // a GEMM batch takes microseconds; give up after 50 ms
constexpr uint64_t kDrainNs = 20ull * 1000 * 1000; // after giving up: a late GEMM's last chance, per phase
constexpr float kTwoPiOver2p32 = 1.46291807926715968e-9f;

// Sizes, shared-memory map, tensor-memory map and thread organisation for
// M = 2^LM.  The per-bin chirp-phase words live in tensor memory after the
// accumulators: the chirp-stage thread q of every pipe reads TMEM lane q mod
// 128, and the bins a lane's threads handle are the same in every pipe, so one
// copy serves all pipes.
template <int AB, int LM> struct TcLayout {
    static constexpr int M = 1 << LM;
    static constexpr int P = M / 64;                    // pass-A DFT length
    static constexpr int npipe = LM == 12 ? (AB ? 1 : 3) : (AB ? 2 : 6);   // DMs in flight per CTA
    static constexpr int pt = LM == 12 ? (AB ? 512 : 256) : (AB ? 256 : 128);   // threads per pipe
    static constexpr int nt = npipe * pt;
    static constexpr int ncg = pt / 128;                // TMEM column groups of a pipe's read-outs
    static constexpr int jh = M / pt;                   // chirp bins (j_hi values) per thread
    static constexpr uint32_t nb = AB ? 2 : 1;          // F_P planes (hi, lo)
    static constexpr uint32_t na = AB ? 2 : 1;          // operand planes per pipe (hi, lo)
    static constexpr uint32_t sbo_f = 32 * P;           // F_P, K-major: stride between 8-row cores
    static constexpr uint32_t fbytes = 8 * P * P;       // one 2P x 2P half-precision F_P
    static constexpr uint32_t sbo_x = 32 * P + 16;      // pass-A data, K-major: row-core stride padded by 16 B
    static constexpr uint32_t lbo_y = 32 * P + 16;      // pass-B data, MN-major: K-core stride padded by 16 B
    static constexpr uint32_t abuf = 16 * lbo_y;        // one operand: 16 K cores, or 16 row cores of pass A
    static constexpr uint32_t off_b = 0;
    static constexpr uint32_t off_x = off_b + nb * fbytes;
    static constexpr uint32_t off_tw = off_x + 16 * M;  // W_M twiddle pairs [m0 / 2][j_lo]
    static constexpr uint32_t off_a = off_tw + 8 * M;
    static constexpr uint32_t abytes = na * abuf;
    static constexpr uint32_t off_misc = off_a + npipe * abytes;
    // misc: mbarriers (one per pipe, <= 8) at +0, TMEM slot at +64, one float per
    // warp (<= 32) at +128, queue ticket at +256, the CTA's work split (6 words) at +264
    static constexpr uint32_t m_tslot = 64, m_red = 128, m_next = 256, m_book = 264;
    static constexpr uint32_t total = off_misc + 320;
    static_assert(npipe <= 8 && nt <= 1024, "misc area");
    static constexpr uint32_t tmem_cols = 512;
    static constexpr uint32_t acc_cols = 2 * P;         // one accumulator
    static constexpr uint32_t ph_col = npipe * acc_cols;   // first phase-word column
    static constexpr uint32_t f_col = ph_col + 2 * jh * ncg;   // F_64 as pass B's A operand (64 columns; BF16 lo: 64 more)
    static_assert(f_col + 64 * nb <= tmem_cols, "tensor memory");
    static_assert(total <= 232448, "shared memory");
};

__device__ __forceinline__ bool bar_and(int id, int count, bool v)
{
    uint32_t r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}"
                 : "=r"(r)
                 : "r"((uint32_t)v), "r"(id), "r"(count)
                 : "memory");
    return r != 0;
}

template <int AB> __device__ __forceinline__ uint32_t pk(float lo, float hi)
{
    return AB ? tc::pack_bf16(lo, hi) : tc::pack_f16(lo, hi);
}

// hi part of a bf16 split: round to bf16 and back
__device__ __forceinline__ float bf16_round(float x) { return __uint_as_float(__float_as_uint(__uint_as_float(tc::pack_bf16(x, 0.f) << 16))); }

// Detection and integration of one pass-B result, by the thread of TMEM lane
// 2 m1 + ro (ro: 0 real, 1 imaginary part) and detection group cg (m0 in
// [32 cg, 32 cg + 32)).  Columns pol * P + m0 hold polarisation pol at time
// m' = m0 + P m1, counted from the first valid sample.  Each thread sums the
// squares of its part over both polarisations and N consecutive m0, then the
// lane pair (re, im) adds its partial sums: ro = 0 keeps the first half of the
// windows of a chunk and ro = 1 the second half, one shuffle per output.
template <int N, int P>
__device__ __forceinline__ void tc_detect(uint32_t taddr, int cg, int m1, int ro, float *__restrict__ orow, int seglen,
                                          float oscale)
{
    constexpr int WC = N >= 16 ? 1 : 16 / N;   // windows (or window halves, N = 32) per chunk of 16 m0
    float carry = 0.f;
    #pragma unroll
    for (int h = 0; h < 2; h++) {
        float acc[WC];
        uint64_t acc2[WC];
        #pragma unroll
        for (int c = 0; c < 2; c++) {   // 8 columns of each polarisation at a time
            uint32_t bx[8], by[8];
            tc::tmem_ld8_async(taddr + 32 * cg + 16 * h + 8 * c, bx);
            tc::tmem_ld8_async(taddr + P + 32 * cg + 16 * h + 8 * c, by);
            tc::tmem_wait();
            if constexpr (N == 1) {
                #pragma unroll
                for (int i8 = 0; i8 < 8; i8++) {
                    const float x = __uint_as_float(bx[i8]), y = __uint_as_float(by[i8]);
                    acc[8 * c + i8] = fmaf(y, y, x * x);
                }
            } else {
                // neighbouring columns (one window, N even) as packed FP32 pairs
                #pragma unroll
                for (int i8 = 0; i8 < 8; i8 += 2) {
                    const int i = 8 * c + i8;
                    const uint64_t X = tc::f2_pack(__uint_as_float(bx[i8]), __uint_as_float(bx[i8 + 1]));
                    const uint64_t Y = tc::f2_pack(__uint_as_float(by[i8]), __uint_as_float(by[i8 + 1]));
                    const int w = N >= 16 ? 0 : i / N;
                    acc2[w] = (i % N == 0) ? tc::f2_mul(X, X) : tc::f2_fma(X, X, acc2[w]);
                    acc2[w] = tc::f2_fma(Y, Y, acc2[w]);
                }
            }
        }
        if constexpr (N > 1) {
            #pragma unroll
            for (int w = 0; w < WC; w++) {
                float lo, hi;
                tc::f2_unpack(acc2[w], lo, hi);
                acc[w] = lo + hi;
            }
        }
        if constexpr (N == 32) {
            if (h == 0) {
                carry = acc[0];
                continue;
            }
            acc[0] += carry;
        }
        const int ubase = (P * m1 + 32 * cg + (N == 32 ? 0 : 16 * h)) / N;
        if constexpr (WC == 1) {
            const float tot = acc[0] + __shfl_xor_sync(0xffffffffu, acc[0], 1);
            if (ro == 0 && ubase < seglen) orow[ubase] = tot * oscale;
        } else {
            #pragma unroll
            for (int k = 0; k < WC / 2; k++) {
                const float send = ro ? acc[k] : acc[k + WC / 2];
                const float keep = ro ? acc[k + WC / 2] : acc[k];
                const float tot = keep + __shfl_xor_sync(0xffffffffu, send, 1);
                const int u = ubase + ro * (WC / 2) + k;
                if (u < seglen) orow[u] = tot * oscale;
            }
        }
    }
}

}  // namespace

// One work item: the M spectral bins of one channel of one overlap-save
// segment of one subband, and a tile of consecutive DM trials.
struct TcItem {
    const float4 *src;     // M bins, (X re, X im, Y re, Y im)
    const uint2 *ph;       // per-bin words: uniform DM list (a, b) of this tile, otherwise K as double
    const double *dms;     // DM values from the item's first DM (uneven lists)
    int ndt;               // DMs of the item
    int dbase;             // index of the item's first DM within its tile (the phase step count)
    float *out;            // output of the tile's first DM at this channel row and segment offset
    int64_t dm_stride;     // floats between the rows of consecutive DMs
    int nd, nint;
    int ulim;              // output samples of this segment that are stored: (M - nd) / nint, less where
                           // the segment reaches past the filterbank's last sample
    float scale_out;
};

// Per-CTA set-up: F_P and twiddles to shared memory, F_64 to tensor memory,
// mbarriers.  Returns the TMEM base address.
template <int AB, int LM>
__device__ __forceinline__ uint32_t tc_cta_setup(uint8_t *smem, const uint4 *__restrict__ bmat,
                                                 const uint4 *__restrict__ bmat64, const float2 *__restrict__ twq)
{
    using L = TcLayout<AB, LM>;
    constexpr int NT = L::nt;
    const int tid = threadIdx.x, warp = tid >> 5;
    uint8_t *bm = smem + L::off_b;
    float2 *tws = reinterpret_cast<float2 *>(smem + L::off_tw);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L::off_misc);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + L::off_misc + L::m_tslot);
    for (int i = tid; i < (int)(L::nb * L::fbytes / 16); i += NT) reinterpret_cast<uint4 *>(bm)[i] = bmat[i];
    for (int i = tid; i < L::M; i += NT) tws[i] = __ldg(twq + i);
    if (warp == 0) tc::tmem_alloc(tslot, L::tmem_cols);
    if (tid < L::npipe) {
        tc::mbar_init(&mbar[tid], 1);
        tc::fence_mbar_init();
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    // F_64 (and its BF16 lo part) into tensor memory as pass B's A operand: warp
    // w < 4 writes TMEM rows 32 w .. 32 w + 31; row 2 m1 + ro is row 64 ro + m1 of
    // the K-major copy in global memory, column c holds its K elements 2c, 2c + 1
    const uint8_t *f64 = reinterpret_cast<const uint8_t *>(bmat64);
    if (warp < 4) {
        const int r = 32 * warp + (tid & 31);
        const int n = (r & 1) * 64 + (r >> 1);
        #pragma unroll 1
        for (uint32_t part = 0; part < L::nb; part++) {
            #pragma unroll 1
            for (int h = 0; h < 2; h++) {
                uint32_t w[32];
                #pragma unroll
                for (int c = 0; c < 32; c++) {
                    const int k = 2 * (32 * h + c);
                    w[c] = __ldg(reinterpret_cast<const uint32_t *>(f64 + part * kF64Bytes + (n / 8) * kF64Sbo +
                                                                    (k / 8) * kLboA + (n % 8) * 16 + (k % 8) * 2));
                }
                tc::tmem_st32(tmem + ((uint32_t)(32 * warp) << 16) + L::f_col + 64 * part + 32 * h, w);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    return tmem;
}

// After an item's wait gave up (CTA-uniform): one more bounded wait for each
// phase of every pipe's mbarrier, by one thread, so that a GEMM that is merely
// late completes before the tensor memory it writes is freed.  A phase that is
// not pending completed earlier or costs one bounded wait.
template <int AB, int LM> __device__ __forceinline__ void tc_cta_drain(uint8_t *smem)
{
    if (threadIdx.x != 0) return;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + TcLayout<AB, LM>::off_misc);
    for (int p = 0; p < TcLayout<AB, LM>::npipe; p++) {
        (void)tc::mbar_wait(&mbar[p], 0, kDrainNs, kWaitPolls);
        (void)tc::mbar_wait(&mbar[p], 1, kDrainNs, kWaitPolls);
    }
}

template <int AB, int LM> __device__ __forceinline__ void tc_cta_teardown(uint32_t tmem)
{
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if ((threadIdx.x >> 5) == 0) tc::tmem_free(tmem, TcLayout<AB, LM>::tmem_cols);
}

// The DM stage of one item.  Must be called by every thread of the CTA;
// returns false (for every thread) if a tensor-core wait gave up.  NI > 0: the
// item's nint, fixed at compile time (one detection variant in the per-DM loop);
// NI = 0: nint chosen per DM among the six variants.
template <bool UNIFORM, int AB, int LM, int NI>
__device__ __forceinline__ bool tc_run_item(const TcItem &it, uint8_t *smem, uint32_t tmem)
{
    using L = TcLayout<AB, LM>;
    constexpr int kM = L::M;
    constexpr int P = L::P;
    constexpr int NT = L::nt;
    constexpr int NPIPE = L::npipe;
    constexpr int PT = L::pt;                // threads per pipe
    constexpr int NCG = L::ncg;             // TMEM column groups per pipe
    constexpr int JH = L::jh;               // j_hi values per thread in the chirp stage
    constexpr uint32_t kSboA = L::sbo_f, kSboX = L::sbo_x, kLboB = L::lbo_y, kAbuf = L::abuf, kBmat = L::fbytes;
    uint8_t *bm = smem + L::off_b;
    float4 *xs = reinterpret_cast<float4 *>(smem + L::off_x);
    float2 *tws = reinterpret_cast<float2 *>(smem + L::off_tw);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L::off_misc);
    float *red = reinterpret_cast<float *>(smem + L::off_misc + L::m_red);   // one float per warp

    const int tid = threadIdx.x, warp = tid >> 5;
    const int pipe = tid / PT;
    const int q = tid % PT;                  // index within the pipe
    const int t = q & 127;                   // TMEM lane = GEMM row = 32 (warp % 4) + lane
    const int cg = q >> 7;                   // column group of this thread's read-outs / phase words
    const int jlo = q & 63;                  // chirp stage: bins j_hi * 64 + jlo, j_hi in [jbase, jbase + JH)
    const int jbase = JH * (q >> 6);
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    tc::fence_after();   // order this item's tensor-memory writes after the previous item's reads

    // ---- the channel's spectrum, scaled by a power of two so that |x| 2^e <= 512
    //      (a 64-point pass then stays below 2^15); the scale is undone on the output
    //      Staged as bin pairs (j_hi = 2 h, 2 h + 1 at one j_lo), one plane per polarisation:
    //      xs[pol * M / 2 + 64 h + j_lo] = (re even, re odd, im even, im odd), so that the chirp
    //      stage multiplies two bins per packed FP32-pair instruction.
    float vmax = 0.f;
    for (int i = tid; i < kM / 2; i += NT) {
        const int jl = i & 63, h2 = i >> 6;
        const float4 a = __ldg(it.src + 128 * h2 + jl), b = __ldg(it.src + 128 * h2 + 64 + jl);
        xs[i] = make_float4(a.x, b.x, a.y, b.y);
        xs[kM / 2 + i] = make_float4(a.z, b.z, a.w, b.w);
        vmax = fmaxf(vmax, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
        vmax = fmaxf(vmax, fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fmaxf(fabsf(b.z), fabsf(b.w))));
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if ((tid & 31) == 0) red[warp] = vmax;
    __syncthreads();
    float bmax = 0.f;
    for (int w = 0; w < NT / 32; w++) bmax = fmaxf(bmax, red[w]);
    int e = bmax > 0.f ? (int)floorf(log2f(512.f / bmax)) : 0;
    e = max(-100, min(100, e));
    const float xscale = ldexpf(1.f, e);
    const float oscale = it.scale_out * ldexpf(1.f, -2 * e);
    for (int i = tid; i < kM; i += NT) {
        float4 v = xs[i];
        xs[i] = make_float4(v.x * xscale, v.y * xscale, v.z * xscale, v.w * xscale);
    }
    // phase words of this thread's chirp bins -> TMEM (pipe 0 writes; every pipe reads the same lanes)
    const uint32_t ph_taddr = tmem + lane_off + L::ph_col + 2 * JH * cg;
    if (pipe == 0) {
        uint32_t w[2 * JH];
        #pragma unroll
        for (int i = 0; i < JH; i++) {
            const uint2 v = __ldg(it.ph + (jbase + i) * 64 + jlo);
            w[2 * i] = v.x;
            w[2 * i + 1] = v.y;
        }
        if constexpr (JH == 16) tc::tmem_st32(ph_taddr, w);
        else tc::tmem_st16(ph_taddr, w);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();

    const uint32_t dcol = tmem + L::acc_cols * pipe;
    uint8_t *ab = smem + L::off_a + pipe * L::abytes;
    uint64_t *mb = &mbar[pipe];
    const int bar_id = 1 + pipe;
    const int ndt = it.ndt;
    const int nd = it.nd, nint = it.nint;
    const int half = nd / 2;
    const int ulim = it.ulim;
    const uint32_t id_a = tc::idesc(128, 2 * P, AB, 0, 0);   // pass A: data (K-major) x F_P (K-major)
    const uint32_t id_b = tc::idesc(128, 2 * P, AB, 0, 1);   // pass B: F_64^T (K-major) x data (MN-major)
    const uint32_t bm_addr = tc::smem_addr(bm), ab_addr = tc::smem_addr(ab);
    // The issuing thread builds each operand's descriptor of K step 0 once per GEMM;
    // step ks adds ks * (byte step >> 4) to the address field (bits 0-13, no carry:
    // every operand lies below 256 KB), so a GEMM costs it a few instructions per MMA.
    constexpr uint64_t kStepK = 256 >> 4, kStepY = (2 * kLboB) >> 4;
    uint32_t ok = 1;

    for (int d = pipe; d < ndt; d += NPIPE) {
        // ---- chirp, round: pass-A operand, K-major, row = 2 j_lo + pol, k = 2 j_hi + (re, im);
        //      two bins per packed FP32-pair multiply
        {
            double dmv = 0.0;
            if constexpr (!UNIFORM) dmv = it.dms[d];
            // phase words (a, b) of the thread's bins, 8 bins (16 words) per tensor-memory load:
            // half the registers of loading all 16 bins at once, for one more wait
            constexpr int CH = JH / 4 < 2 ? JH / 4 : 2;   // 4-bin groups per load
            uint32_t wl[8 * CH];
            #pragma unroll
            for (int c4 = 0; c4 < JH / 4; c4++) {
                if (c4 % CH == 0) {
                    if constexpr (CH == 2) tc::tmem_ld16_async(ph_taddr + 8 * c4, wl);
                    else tc::tmem_ld8_async(ph_taddr + 8 * c4, wl);
                    tc::tmem_wait();
                }
                uint32_t hx[4], hy[4], lx[4], ly[4];
                #pragma unroll
                for (int i2 = 0; i2 < 2; i2++) {
                    // bins j_hi = jbase + b and jbase + b + 1 (jbase and b even) of column j_lo
                    const int b = 4 * c4 + 2 * i2;
                    float sn[2], cs[2];
                    #pragma unroll
                    for (int e2 = 0; e2 < 2; e2++) {
                        if constexpr (UNIFORM) {
                            const int q = 8 * (c4 % CH) + 2 * (2 * i2 + e2);   // bin b + e2 in wl
                            const int32_t p = (int32_t)(wl[q] + (uint32_t)(d + it.dbase) * wl[q + 1]);
                            __sincosf((float)p * kTwoPiOver2p32, &sn[e2], &cs[e2]);
                        } else {
                            const int j = (jbase + b + e2) * 64 + jlo;
                            const int q = 8 * (c4 % CH) + 2 * (2 * i2 + e2);
                            const double kj = __hiloint2double((int)wl[q + 1], (int)wl[q]);
                            double cyc = dmv * kj;
                            cyc -= rint(cyc);
                            const uint32_t pf = (uint32_t)(long long)llrint(-cyc * 4294967296.0) + ((uint32_t)(j * half) << (32 - LM));
                            __sincosf((float)(int32_t)pf * kTwoPiOver2p32, &sn[e2], &cs[e2]);
                        }
                    }
                    const int pidx = ((jbase + b) >> 1) * 64 + jlo;
                    const float4 vx = xs[pidx], vy = xs[kM / 2 + pidx];
                    const uint64_t CS = tc::f2_pack(cs[0], cs[1]), SN = tc::f2_pack(sn[0], sn[1]);
                    float xr[2], xi[2], yr[2], yi[2];
                    {
                        const uint64_t R = tc::f2_pack(vx.x, vx.y), I = tc::f2_pack(vx.z, vx.w);
                        tc::f2_unpack(tc::f2_sub(tc::f2_mul(R, CS), tc::f2_mul(I, SN)), xr[0], xr[1]);
                        tc::f2_unpack(tc::f2_fma(R, SN, tc::f2_mul(I, CS)), xi[0], xi[1]);
                    }
                    {
                        const uint64_t R = tc::f2_pack(vy.x, vy.y), I = tc::f2_pack(vy.z, vy.w);
                        tc::f2_unpack(tc::f2_sub(tc::f2_mul(R, CS), tc::f2_mul(I, SN)), yr[0], yr[1]);
                        tc::f2_unpack(tc::f2_fma(R, SN, tc::f2_mul(I, CS)), yi[0], yi[1]);
                    }
                    #pragma unroll
                    for (int e2 = 0; e2 < 2; e2++) {
                        const int i = 2 * i2 + e2;
                        hx[i] = pk<AB>(xr[e2], xi[e2]);
                        hy[i] = pk<AB>(yr[e2], yi[e2]);
                        if constexpr (AB) {
                            lx[i] = tc::pack_bf16(xr[e2] - bf16_round(xr[e2]), xi[e2] - bf16_round(xi[e2]));
                            ly[i] = tc::pack_bf16(yr[e2] - bf16_round(yr[e2]), yi[e2] - bf16_round(yi[e2]));
                        }
                    }
                }
                const int kcore = (jbase + 4 * c4) / 4;
                const uint32_t ox = (uint32_t)((2 * jlo) / 8) * kSboX + kcore * kLboA + ((2 * jlo) % 8) * 16;
                const uint32_t oy = (uint32_t)((2 * jlo + 1) / 8) * kSboX + kcore * kLboA + ((2 * jlo + 1) % 8) * 16;
                *reinterpret_cast<uint4 *>(ab + ox) = make_uint4(hx[0], hx[1], hx[2], hx[3]);
                *reinterpret_cast<uint4 *>(ab + oy) = make_uint4(hy[0], hy[1], hy[2], hy[3]);
                if constexpr (AB) {
                    *reinterpret_cast<uint4 *>(ab + kAbuf + ox) = make_uint4(lx[0], lx[1], lx[2], lx[3]);
                    *reinterpret_cast<uint4 *>(ab + kAbuf + oy) = make_uint4(ly[0], ly[1], ly[2], ly[3]);
                }
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        tc::bar(bar_id, PT);
        tc::fence_after();
        if (q == 0) {
            const uint32_t xa = tc::opaque(ab_addr), fa = tc::opaque(bm_addr);
            const uint64_t dX = tc::sdesc(xa, kLboA, kSboX), dF = tc::sdesc(fa, kLboA, kSboA);
            uint64_t dXl = 0, dFl = 0;
            if constexpr (AB) {
                dXl = tc::sdesc(xa + kAbuf, kLboA, kSboX);
                dFl = tc::sdesc(fa + kBmat, kLboA, kSboA);
            }
            #pragma unroll
            for (int ks = 0; ks < P / 8; ks++) {   // K = 2P
                tc::mma(dcol, dX + kStepK * ks, dF + kStepK * ks, id_a, ks > 0);
                if constexpr (AB) {
                    tc::mma(dcol, dXl + kStepK * ks, dF + kStepK * ks, id_a, 1);
                    tc::mma(dcol, dX + kStepK * ks, dFl + kStepK * ks, id_a, 1);
                }
            }
            tc::commit(mb);
        }
        // warp 0 of the pipe polls the mbarrier (bounded); the other warps wait at the pipe's named
        // barrier, which takes no issue slots, and the vote makes a timeout pipe-uniform
        ok = bar_and(bar_id, PT, q >= 32 || tc::mbar_wait(mb, 0, kWaitNs, kWaitPolls));
        if (!ok) break;
        tc::fence_after();

        // ---- pass-A row (j_lo, pol) -> twiddle -> pass-B operand (MN-major): column pol * P + m0,
        //      k = 2 j_lo + (re, im).  Eight m0 at a time: their real parts (TMEM columns m0)
        //      and imaginary parts (P + m0) are loaded together and waited for once.
        {
            const int pol = t & 1, rjlo = t >> 1;
            constexpr int MPT = P / NCG;              // m0 per thread
            const float4 *tw4 = reinterpret_cast<const float4 *>(tws);
            #pragma unroll
            for (int st = 0; st < MPT / 8; st++) {
                const int m0b = cg * MPT + 8 * st;
                uint32_t vr[8], vi[8];
                tc::tmem_ld8_async(dcol + lane_off + m0b, vr);
                tc::tmem_ld8_async(dcol + lane_off + P + m0b, vi);
                tc::tmem_wait();
                float re[8], im[8];
                #pragma unroll
                for (int i = 0; i < 4; i++) {
                    // (wr, wr', wi, wi') of m0 = m0b + 2i, m0b + 2i + 1
                    const float4 w = tw4[((m0b >> 1) + i) * 64 + rjlo];
                    const uint64_t P = tc::f2_pack(__uint_as_float(vr[2 * i]), __uint_as_float(vr[2 * i + 1]));
                    const uint64_t Q = tc::f2_pack(__uint_as_float(vi[2 * i]), __uint_as_float(vi[2 * i + 1]));
                    const uint64_t WR = tc::f2_pack(w.x, w.y), WI = tc::f2_pack(w.z, w.w);
                    const uint64_t R = tc::f2_sub(tc::f2_mul(P, WR), tc::f2_mul(Q, WI));
                    const uint64_t I = tc::f2_fma(P, WI, tc::f2_mul(Q, WR));
                    tc::f2_unpack(R, re[2 * i], re[2 * i + 1]);
                    tc::f2_unpack(I, im[2 * i], im[2 * i + 1]);
                }
                // Polarisation 0 stores its real parts in K row 2 j_lo and its imaginary parts in row
                // 2 j_lo + 1.  Polarisation 1 stores i y instead: its real parts in row 2 j_lo + 1 and
                // its negated imaginary parts (sign bits flipped) in row 2 j_lo.  Pass B is linear, so
                // that polarisation's output is i times the true one, which detection does not see;
                // the neighbouring lanes of the two polarisations then write different banks.
                const uint32_t o = (uint32_t)((pol * P + m0b) / 8) * kSboB + (uint32_t)(2 * rjlo / 8) * kLboB +
                                   (uint32_t)((2 * rjlo) % 8) * 16;
                const uint32_t flip = pol ? 0x80008000u : 0u, o_re = o + 16 * pol, o_im = o + 16 * (1 - pol);
                *reinterpret_cast<uint4 *>(ab + o_re) =
                    make_uint4(pk<AB>(re[0], re[1]), pk<AB>(re[2], re[3]), pk<AB>(re[4], re[5]), pk<AB>(re[6], re[7]));
                *reinterpret_cast<uint4 *>(ab + o_im) =
                    make_uint4(pk<AB>(im[0], im[1]) ^ flip, pk<AB>(im[2], im[3]) ^ flip, pk<AB>(im[4], im[5]) ^ flip,
                               pk<AB>(im[6], im[7]) ^ flip);
                if constexpr (AB) {
                    float lr[8], li[8];
                    #pragma unroll
                    for (int z = 0; z < 8; z++) {
                        lr[z] = re[z] - bf16_round(re[z]);
                        li[z] = im[z] - bf16_round(im[z]);
                    }
                    *reinterpret_cast<uint4 *>(ab + kAbuf + o_re) = make_uint4(
                        pk<1>(lr[0], lr[1]), pk<1>(lr[2], lr[3]), pk<1>(lr[4], lr[5]), pk<1>(lr[6], lr[7]));
                    *reinterpret_cast<uint4 *>(ab + kAbuf + o_im) = make_uint4(
                        pk<1>(li[0], li[1]) ^ flip, pk<1>(li[2], li[3]) ^ flip, pk<1>(li[4], li[5]) ^ flip,
                        pk<1>(li[6], li[7]) ^ flip);
                }
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        tc::bar(bar_id, PT);
        tc::fence_after();
        if (q == 0) {
            const uint32_t ya = tc::opaque(ab_addr), f_taddr = tc::opaque(tmem) + L::f_col;
            const uint64_t dY = tc::sdesc(ya, kLboB, kSboB);
            uint64_t dYl = 0;
            if constexpr (AB) dYl = tc::sdesc(ya + kAbuf, kLboB, kSboB);
            #pragma unroll
            for (int ks = 0; ks < 8; ks++) {
                tc::mma_ta(dcol, f_taddr + 8 * ks, dY + kStepY * ks, id_b, ks > 0);
                if constexpr (AB) {
                    tc::mma_ta(dcol, f_taddr + 8 * ks, dYl + kStepY * ks, id_b, 1);
                    tc::mma_ta(dcol, f_taddr + 64 + 8 * ks, dY + kStepY * ks, id_b, 1);
                }
            }
            tc::commit(mb);
        }
        ok = bar_and(bar_id, PT, q >= 32 || tc::mbar_wait(mb, 1, kWaitNs, kWaitPolls));
        if (!ok) break;
        tc::fence_after();

        // ---- detect + integrate in registers (see the head of this file), by P / 32
        //      groups of 32 m0 (the pipe's other warpgroups, if any, skip)
        if (cg < P / 32) {
            float *orow = it.out + (int64_t)d * it.dm_stride;
            const uint32_t taddr = dcol + lane_off;
            const int m1 = t >> 1, ro = t & 1;
            if constexpr (NI > 0) {
                tc_detect<NI, P>(taddr, cg, m1, ro, orow, ulim, oscale);
            } else switch (nint) {
            case 1: tc_detect<1, P>(taddr, cg, m1, ro, orow, ulim, oscale); break;
            case 2: tc_detect<2, P>(taddr, cg, m1, ro, orow, ulim, oscale); break;
            case 4: tc_detect<4, P>(taddr, cg, m1, ro, orow, ulim, oscale); break;
            case 8: tc_detect<8, P>(taddr, cg, m1, ro, orow, ulim, oscale); break;
            case 16: tc_detect<16, P>(taddr, cg, m1, ro, orow, ulim, oscale); break;
            default: tc_detect<32, P>(taddr, cg, m1, ro, orow, ulim, oscale); break;
            }
        }
    }
    tc::fence_before();
    return __syncthreads_and(ok) != 0;
}

// AB: 0 = FP16 operands, 1 = BF16 hi/lo operands.
// FP16: three pipes of 256 threads (M = 4096) or six of 128 (M = 2048), each
// carrying one DM at a time through its own operand buffer, TMEM columns and
// mbarrier.  BF16: one pipe of 512 threads (M = 4096; one hi/lo operand set
// fits) or two of 256 (M = 2048).  Within a pipe the chirp stage is split
// over all its threads, and each tensor-memory read-out is split by column
// groups over its warpgroups (warp w reads TMEM lanes 32 (w % 4) .. + 31).
// Persistent: one CTA per SM sets up once (DFT matrix and twiddles in shared
// memory, F in tensor memory) and takes items (DM tile, subband, segment,
// channel) blockIdx.x, + gridDim.x, ...; while it works on one item, the next
// item's spectrum and phase words are prefetched into L2.  NI: nint fixed at
// compile time (8), or 0 for any nint dividing 32.
template <bool UNIFORM, int AB, int LM, int NI>
__global__ void __launch_bounds__(TcLayout<AB, LM>::nt, 1)
k_dedisperse_tc(const float4 *__restrict__ spec, const uint2 *__restrict__ nco, const double *__restrict__ ktab,
                const double *__restrict__ dm_list, const uint4 *__restrict__ bmat, const uint4 *__restrict__ bmat64,
                const float2 *__restrict__ twq, float *__restrict__ out, int *__restrict__ status, int nsub, int kc,
                int64_t k0, int nchan, int ndm, int dm_tile, int nd, int nint, int64_t nout, float scale_out,
                int64_t nitems, int dm_off, int dm_cnt, int64_t tlim)
{
    constexpr int kM = 1 << LM;
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x;
    // once any CTA has given up on a tensor-core wait, the rest of the launch
    // returns at once (one read, block-uniform decision)
    if (__syncthreads_or(tid == 0 ? *reinterpret_cast<volatile int *>(status) : 0)) return;
    const int seglen = (kM - nd) / nint;
    const int64_t rows = (int64_t)nsub * nchan;
    auto make = [&](int64_t item) {
        const int c = (int)(item % nchan); item /= nchan;
        const int kk = (int)(item % kc); item /= kc;
        const int s = (int)(item % nsub); item /= nsub;
        const int tile = (int)item;
        const int dm0 = tile * dm_tile + dm_off;   // the item's DMs: dm_off .. dm_off + dm_cnt - 1 of the tile
        TcItem it;
        it.src = spec + (((int64_t)s * kc + kk) * nchan + c) * kM;
        if constexpr (UNIFORM) it.ph = nco + ((int64_t)tile * nsub + s) * (int64_t)nchan * kM + (int64_t)c * kM;
        else it.ph = reinterpret_cast<const uint2 *>(ktab + ((int64_t)s * nchan + c) * kM);
        it.dms = dm_list + dm0;
        it.ndt = min(dm_cnt, ndm - dm0);
        it.dbase = dm_off;
        it.out = out + (int64_t)tile * dm_cnt * rows * nout + (int64_t)(s * nchan + c) * nout + (k0 + kk) * seglen;
        it.dm_stride = rows * nout;
        it.nd = nd;
        it.nint = nint;
        const int64_t room = tlim - (k0 + kk) * seglen;
        it.ulim = room <= 0 ? 0 : (int)(room < seglen ? room : seglen);
        it.scale_out = scale_out;
        return it;
    };
    // Work split: whole items round-robin (item blockIdx.x + k gridDim.x) for every full round of
    // the grid, which keeps the items running at once neighbours (one subband's phase words and
    // segments); then the (item, DM) pairs of the last, partial round split into equal shares, so
    // that no CTA is left a whole item behind the others (a served block of 4608 items on 152 SMs
    // had 48 CTAs working a 31st item while 104 idled).  A part of an item is computed exactly as
    // the whole item would compute those DMs.  The split's bookkeeping is kept in shared memory, so
    // that it holds no registers through the per-DM loop.
    int64_t *book = reinterpret_cast<int64_t *>(smem + TcLayout<AB, LM>::off_misc + TcLayout<AB, LM>::m_book);
    if (tid == 0) {
        const int64_t tile_items = (int64_t)nsub * kc * nchan;
        const int64_t ntile = nitems / tile_items;
        const int64_t ndt_last = max(0, min(dm_cnt, ndm - ((int)(ntile - 1) * dm_tile + dm_off)));
        const int64_t f_full = (ntile - 1) * tile_items * dm_cnt;   // pairs of the full tiles
        const int64_t last0 = (ntile - 1) * tile_items;              // first item of the last tile
        const int64_t total = f_full + tile_items * ndt_last;
        const int64_t rounds = nitems / gridDim.x;                   // whole-item rounds
        const int64_t i0 = rounds * gridDim.x;                       // first item of the partial round
        const int64_t f0 = i0 <= last0 ? i0 * dm_cnt : f_full + (i0 - last0) * ndt_last;
        const int64_t share = (total - f0 + gridDim.x - 1) / gridDim.x;
        book[0] = f_full;
        book[1] = ndt_last;
        book[2] = last0;
        book[3] = min(total, f0 + (int64_t)blockIdx.x * share);
        book[4] = min(total, book[3] + share);
        book[5] = rounds;
    }
    auto locate = [&](int64_t f, int64_t &item, int &off, int &ndt) {
        const int64_t f_full = book[0];
        if (f < f_full) {
            item = f / dm_cnt;
            off = (int)(f % dm_cnt);
            ndt = dm_cnt;
        } else {
            const int64_t last = book[1];
            item = book[2] + (f - f_full) / last;
            off = (int)((f - f_full) % last);
            ndt = (int)last;
        }
    };
    const uint32_t tmem = tc_cta_setup<AB, LM>(smem, bmat, bmat64, twq);   // ends with a CTA barrier
    constexpr int kSrcChunks = kM / 256, kPhChunks = kM / 512;   // 4 KB chunks of 16 M and 8 M bytes
    // step k < rounds: whole item blockIdx.x + k gridDim.x; then parts of the partial round's items
    int64_t k = 0, f = book[3];
    for (;;) {
        int64_t item;
        int off = 0, n;
        if (k < book[5]) {
            item = blockIdx.x + k * gridDim.x;
            n = -1;   // the whole item
        } else {
            if (f >= book[4]) break;
            int ndt;
            locate(f, item, off, ndt);
            n = (int)min((int64_t)(ndt - off), book[4] - f);
        }
        TcItem it = make(item);
        if (n >= 0) {
            it.ndt = n;
            it.dbase += off;
            it.dms += off;
            it.out += (int64_t)off * it.dm_stride;
        }
        if (tid < kSrcChunks + kPhChunks) {   // the next step's spectrum and phase words into L2
            int64_t nitem = -1;
            if (k + 1 < book[5]) {
                nitem = blockIdx.x + (k + 1) * gridDim.x;
            } else {
                const int64_t fn = n >= 0 ? f + n : book[3];
                if (fn < book[4]) {
                    int noff, nndt;
                    locate(fn, nitem, noff, nndt);
                }
            }
            if (nitem >= 0) {
                const TcItem nx = make(nitem);
                if (tid < kSrcChunks) tc::prefetch_l2(reinterpret_cast<const uint8_t *>(nx.src) + 4096 * tid, 4096);
                else tc::prefetch_l2(reinterpret_cast<const uint8_t *>(nx.ph) + 4096 * (tid - kSrcChunks), 4096);
            }
        }
        if (!tc_run_item<UNIFORM, AB, LM, NI>(it, smem, tmem)) {
            if (tid == 0) atomicExch(status, 1);
            tc_cta_drain<AB, LM>(smem);
            break;
        }
        if (n >= 0) f += n;
        else k++;
    }
    tc_cta_teardown<AB, LM>(tmem);
}

// Persistent form for batches of beams of uneven shapes (FP16, evenly spaced
// DM lists): one CTA per SM takes items from a device queue until the round's
// items are exhausted.  The round number is read from device memory, so one
// captured graph serves every round.
template <int AB>
__global__ void __launch_bounds__(TcLayout<AB, 12>::nt, 1)
k_dedisperse_tc_batch(const TcBeam *__restrict__ beams, int nbeam, const int *__restrict__ round_dev,
                      int *__restrict__ queue, const uint4 *__restrict__ bmat, const float2 *__restrict__ twq,
                      int *__restrict__ status)
{
    constexpr int kM = 4096;   // batched beams use channels of 4096 bins (F_P = F_64)
    extern __shared__ __align__(1024) uint8_t smem[];
    int *next = reinterpret_cast<int *>(smem + TcLayout<AB, 12>::off_misc + TcLayout<AB, 12>::m_next);
    const int tid = threadIdx.x;
    if (__syncthreads_or(tid == 0 ? *reinterpret_cast<volatile int *>(status) : 0)) return;
    const int round = *round_dev;
    const uint32_t tmem = tc_cta_setup<AB, 12>(smem, bmat, bmat, twq);
    for (;;) {
        if (tid == 0) *next = atomicAdd(queue, 1);
        __syncthreads();
        int64_t item = *next;
        __syncthreads();
        // find the beam of this item (items of this round, beam after beam)
        int b = 0;
        int64_t kc_b = 0;
        for (; b < nbeam; b++) {
            const TcBeam &B = beams[b];
            const int64_t k0 = (int64_t)round * B.kc;
            kc_b = k0 < B.nseg ? min((int64_t)B.kc, B.nseg - k0) : 0;
            const int64_t n = (int64_t)B.ntile * B.nsub * kc_b * B.nchan;
            if (item < n) break;
            item -= n;
        }
        if (b >= nbeam) break;
        const TcBeam &B = beams[b];
        const int c = (int)(item % B.nchan); item /= B.nchan;
        const int kk = (int)(item % kc_b); item /= kc_b;
        const int s = (int)(item % B.nsub); item /= B.nsub;
        const int tile = (int)item;
        const int dm0 = tile * B.dm_tile;
        TcItem it;
        it.src = B.spec + (((int64_t)s * B.kc + kk) * B.nchan + c) * kM;
        it.ph = B.nco + ((int64_t)tile * B.nsub + s) * (int64_t)B.nchan * kM + (int64_t)c * kM;
        it.dms = nullptr;
        it.ndt = min(B.dm_tile, B.ndm - dm0);
        it.dbase = 0;
        const int seglen = (kM - B.nd) / B.nint;
        const int64_t rows = (int64_t)B.nsub * B.nchan;
        it.out = B.out + (int64_t)dm0 * rows * B.out_stride + (int64_t)(s * B.nchan + c) * B.out_stride + kk * seglen;
        it.dm_stride = rows * B.out_stride;
        it.nd = B.nd;
        it.nint = B.nint;
        it.ulim = seglen;
        it.scale_out = B.scale;
        if (!tc_run_item<true, AB, 12, 0>(it, smem, tmem)) {
            if (tid == 0) atomicExch(status, 1);
            tc_cta_drain<AB, 12>(smem);
            break;
        }
    }
    tc_cta_teardown<AB, 12>(tmem);
}

// ---------------------------------------------------------------------------

size_t tc_smem(int ab, int lm)
{
    if (lm == 11) return ab ? TcLayout<1, 11>::total : TcLayout<0, 11>::total;
    return ab ? TcLayout<1, 12>::total : TcLayout<0, 12>::total;
}

template <bool U, int AB, int LM, int NI = 0> static cudaError_t set_attr()
{
    return cudaFuncSetAttribute(k_dedisperse_tc<U, AB, LM, NI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TcLayout<AB, LM>::total);
}

template <int AB> static cudaError_t prepare_ab()
{
    cudaError_t e = set_attr<true, AB, 12>();
    if (e == cudaSuccess) e = set_attr<false, AB, 12>();
    if (e == cudaSuccess) e = set_attr<true, AB, 11>();
    if (e == cudaSuccess) e = set_attr<false, AB, 11>();
    if constexpr (AB == 0) {   // the FP16 form with nint = 8 fixed at compile time
        if (e == cudaSuccess) e = set_attr<true, 0, 12, 8>();
        if (e == cudaSuccess) e = set_attr<false, 0, 12, 8>();
        if (e == cudaSuccess) e = set_attr<true, 0, 11, 8>();
        if (e == cudaSuccess) e = set_attr<false, 0, 11, 8>();
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dedisperse_tc_batch<AB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TcLayout<AB, 12>::total);
    return e;
}

cudaError_t tc_prepare(int ab) { return ab ? prepare_ab<1>() : prepare_ab<0>(); }

cudaError_t tc_batch_launch(const TcBeam *beams, int nbeam, const int *round_dev, int *queue, const uint4 *bmat,
                            const float2 *twq, int *status, int ab, int nctas, cudaStream_t st)
{
    if (ab)
        k_dedisperse_tc_batch<1><<<nctas, TcLayout<1, 12>::nt, TcLayout<1, 12>::total, st>>>(
            beams, nbeam, round_dev, queue, bmat, twq, status);
    else
        k_dedisperse_tc_batch<0><<<nctas, TcLayout<0, 12>::nt, TcLayout<0, 12>::total, st>>>(
            beams, nbeam, round_dev, queue, bmat, twq, status);
    return cudaGetLastError();
}

template <bool U, int AB, int LM, int NI = 0> static void launch(const TcArgs &a, cudaStream_t st)
{
    const int64_t ntile = (a.ndm + a.dm_tile - 1) / a.dm_tile;
    const int64_t nitems = ntile * a.nsub * a.kc * a.nchan;
    // one CTA per SM, none without a share of the (item, DM) pairs
    const int cnt = a.dm_cnt > 0 ? a.dm_cnt : a.dm_tile;
    const int64_t last = std::max(0, std::min(cnt, a.ndm - ((int)(ntile - 1) * a.dm_tile + a.dm_off)));
    const int64_t pairs = (int64_t)a.nsub * a.kc * a.nchan * ((ntile - 1) * cnt + last);
    const int64_t nblk = std::max<int64_t>(1, std::min<int64_t>(pairs, std::max(1, a.nsm)));
    k_dedisperse_tc<U, AB, LM, NI><<<(unsigned)nblk, TcLayout<AB, LM>::nt, TcLayout<AB, LM>::total, st>>>(
        a.spec, a.nco, a.ktab, a.dm_list, a.bmat, a.bmat64, a.twq, a.out, a.status, a.nsub, a.kc, a.k0, a.nchan,
        a.ndm, a.dm_tile, a.nd, a.nint, a.nout, a.scale, nitems, a.dm_off, a.dm_cnt > 0 ? a.dm_cnt : a.dm_tile,
        a.tlim);
}

template <int LM> static void launch_lm(const TcArgs &a, cudaStream_t st)
{
    const bool n8 = a.nint == 8;
    if (a.uniform) {
        if (a.ab) launch<true, 1, LM>(a, st);
        else if (n8) launch<true, 0, LM, 8>(a, st);
        else launch<true, 0, LM>(a, st);
    } else {
        if (a.ab) launch<false, 1, LM>(a, st);
        else if (n8) launch<false, 0, LM, 8>(a, st);
        else launch<false, 0, LM>(a, st);
    }
}

cudaError_t tc_dedisperse(const TcArgs &a, cudaStream_t st)
{
    if (a.lm == 11) launch_lm<11>(a, st);
    else launch_lm<12>(a, st);
    return cudaGetLastError();
}

}  // namespace cdmt
