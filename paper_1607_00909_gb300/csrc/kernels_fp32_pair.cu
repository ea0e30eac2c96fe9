// FP32 form of the DM stage for channels of M = 2048, 4096 and 8192 bins, with both
// polarisations in every thread and their arithmetic paired in packed f32x2
// instructions.
//
// The steps are those of k_dedisperse (Sec. 3: "complex multiplication with
// transfer function", "backward FFT", "transpose, unpad and detect"; Eq. 1 for the
// chirp): per (DM tile, subband, segment, channel) item, for every DM of the tile,
// chirp the channel's M bins, run the M-point backward FFT in three passes (radix 16,
// 16 and R, M = 256 R), form |X|^2 + |Y|^2, drop nd/2 samples at each edge, integrate
// nint samples and store.  What differs is the mapping onto the machine:
// - Each of the CTA's T = M / 16 threads (128, 256 or 512) carries 16 bins of BOTH
//   polarisations.  The two polarisations go through exactly the same operations with
//   the same twiddles, so the butterflies run on pairs (X re, Y re) and (X im, Y im) in
//   packed add/sub/mul/fma.rn.f32x2 instructions: one instruction does the work of two.
//   The f32x2 instructions round each lane as the scalar ones do, and the butterflies
//   and twiddle products take fft_core.cuh's operations in its order, so each lane's FFT
//   rounds as the one-polarisation kernel's does.
// - The channel's spectrum (16 M bytes) and its chirp-phase words (8 M bytes) live in
//   tensor memory: thread t holds its bins j = j2 T + t in TMEM lane t mod 128, columns
//   64 (t / 128) + 4 j2 + (X re, Y re, X im, Y im) and 64 T / 128 + 32 (t / 128) + 2 j2 +
//   (phase word pair); 96 of 128 columns at M = 2048, 192 of 256 at 4096, 384 of 512 at
//   8192.  Shared memory keeps the exchange buffer, the pass twiddles and one
//   detected-power row: 56 KB at M = 2048 (four CTAs per SM), 112 KB at 4096 (two),
//   224 KB at 8192 (one).
// - M = 8192 (R = 32): the radix-32 butterflies of the last pass are shared by lane
//   pairs as in fft_core.cuh (a 16-point DFT each, then one radix-2 step through lane
//   shuffles), so one CTA carries both polarisations of a channel: no cluster and no
//   exchange of sums between CTAs.
// - The detected powers of both polarisations are summed per bin before they are
//   stored, so integration reads one row.
#include "cdmt_internal.h"
#include "fft_core.cuh"
#include "tc_ptx.cuh"

namespace cdmt {

namespace {

constexpr float kPhaseScale = 1.46291807926715968e-9f;   // 2 pi / 2^32

// M = 256 R bins per channel, T = 16 R threads; tensor memory: T / 128 column groups of 64
// spectrum words, then as many groups of 32 phase words (96 columns of 128 at R = 8, 192 of 256
// at R = 16, 384 of 512 at R = 32)
template <int R> struct PairLayout {
    static constexpr int M = 256 * R, T = 16 * R, NG = T / 128;
    static constexpr uint32_t tmem_cols = R == 8 ? 128 : R == 16 ? 256 : 512;
    static constexpr int ctas_per_sm = R == 8 ? 4 : R == 16 ? 2 : 1;
};

using u64 = uint64_t;

__device__ __forceinline__ u64 pk2(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up2(u64 v, float &lo, float &hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ __forceinline__ u64 add2(u64 a, u64 b)
{
    u64 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b)
{
    u64 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b)
{
    u64 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c)
{
    u64 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// One complex value of each polarisation: re = (X re, Y re), im = (X im, Y im).
struct P2 {
    u64 re, im;
};
__device__ __forceinline__ P2 padd(P2 a, P2 b) { return {add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ P2 psub(P2 a, P2 b) { return {sub2(a.re, b.re), sub2(a.im, b.im)}; }

// a * (c + S i s) for constants, rounded as mul_cs rounds: (re c - im s', re s' + im c), s' = S s.
// Scalar multiplies take the constants as immediates; packed ones would need them as register pairs.
template <int S> __device__ __forceinline__ P2 pmul_cs(P2 a, float c, float s)
{
    const float ss = S > 0 ? s : -s;
    float xr, yr, xi, yi;
    up2(a.re, xr, yr);
    up2(a.im, xi, yi);
    return {pk2(fmaf(xr, c, -xi * ss), fmaf(yr, c, -yi * ss)), pk2(fmaf(xr, ss, xi * c), fmaf(yr, ss, yi * c))};
}
// a * (S i), exact
template <int S> __device__ __forceinline__ P2 pmul_i(P2 a)
{
    const u64 neg = pk2(-1.f, -1.f);
    return S > 0 ? P2{mul2(a.im, neg), a.re} : P2{a.im, mul2(a.re, neg)};
}

// dft4 of fft_core.cuh on pairs; the multiplication by S i of (a1 - a3) is folded into the
// last additions (t + (-d) and t - d round alike)
template <int S> __device__ __forceinline__ void pdft4(P2 &a0, P2 &a1, P2 &a2, P2 &a3)
{
    const P2 t0 = padd(a0, a2), t1 = psub(a0, a2), t2 = padd(a1, a3), d = psub(a1, a3);
    a0 = padd(t0, t2);
    a2 = psub(t0, t2);
    if (S > 0) {
        a1 = {sub2(t1.re, d.im), add2(t1.im, d.re)};
        a3 = {add2(t1.re, d.im), sub2(t1.im, d.re)};
    } else {
        a1 = {add2(t1.re, d.im), sub2(t1.im, d.re)};
        a3 = {sub2(t1.re, d.im), add2(t1.im, d.re)};
    }
}

// dft16 of fft_core.cuh (4 x 4, natural order in and out) on pairs
template <int S> __device__ __forceinline__ void pdft16(P2 *v)
{
    #pragma unroll
    for (int n2 = 0; n2 < 4; n2++) pdft4<S>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    v[5] = pmul_cs<S>(v[5], kC16, kS16);
    v[6] = pmul_cs<S>(v[6], kC8, kC8);
    v[7] = pmul_cs<S>(v[7], kS16, kC16);
    v[9] = pmul_cs<S>(v[9], kC8, kC8);
    v[10] = pmul_i<S>(v[10]);
    v[11] = pmul_cs<S>(v[11], -kC8, kC8);
    v[13] = pmul_cs<S>(v[13], kS16, kC16);
    v[14] = pmul_cs<S>(v[14], -kC8, kC8);
    v[15] = pmul_cs<S>(v[15], -kC16, -kS16);
    #pragma unroll
    for (int k1 = 0; k1 < 4; k1++) pdft4<S>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    P2 t;
    t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[2]; v[2] = v[8]; v[8] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[6]; v[6] = v[9]; v[9] = t;
    t = v[7]; v[7] = v[13]; v[13] = t;
    t = v[11]; v[11] = v[14]; v[14] = t;
}

// dft8 of fft_core.cuh on pairs (radix-2 decimation in time over two dft4)
template <int S> __device__ __forceinline__ void pdft8(P2 *v)
{
    P2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    P2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    pdft4<S>(e0, e1, e2, e3);
    pdft4<S>(o0, o1, o2, o3);
    o1 = pmul_cs<S>(o1, kC8, kC8);    // W8^1
    o2 = pmul_i<S>(o2);               // W8^2
    o3 = pmul_cs<S>(o3, -kC8, kC8);   // W8^3
    v[0] = padd(e0, o0); v[4] = psub(e0, o0);
    v[1] = padd(e1, o1); v[5] = psub(e1, o1);
    v[2] = padd(e2, o2); v[6] = psub(e2, o2);
    v[3] = padd(e3, o3); v[7] = psub(e3, o3);
}

// The radix-2 step of a radix-32 butterfly shared by lanes (2 beta, 2 beta + 1), as join32 of
// fft_core.cuh does it, on pairs: v holds this lane's 16-point half (inputs j0 = 2a + e) and
// leaves its outputs m2 = k + 16 e in v[k]
template <int S> __device__ __forceinline__ void pjoin32(P2 *v, int e)
{
    #pragma unroll
    for (int k = 0; k < 16; k++) {
        const P2 other = {__shfl_xor_sync(0xffffffffu, v[k].re, 1), __shfl_xor_sync(0xffffffffu, v[k].im, 1)};
        const P2 ev = e ? other : v[k], od = e ? v[k] : other;
        const P2 w = pmul_cs<S>(od, kW32[k][0], kW32[k][1]);   // W_32^k
        v[k] = e ? psub(ev, w) : padd(ev, w);
    }
}

// a * w for one twiddle w shared by both polarisations, rounded as cmul rounds:
// (re wx + im (-wy), re wy + im wx) with the products of im rounded first
__device__ __forceinline__ P2 ptwiddle(P2 a, float2 w)
{
    const u64 WX = pk2(w.x, w.x), WY = pk2(w.y, w.y), NWY = pk2(-w.y, -w.y);
    return {fma2(a.re, WX, mul2(a.im, NWY)), fma2(a.re, WY, mul2(a.im, WX))};
}

__device__ __forceinline__ void st_pair(float4 *p, P2 a)
{
    *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(a.re, a.im);
}
__device__ __forceinline__ P2 ld_pair(const float4 *p)
{
    const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p);
    return {v.x, v.y};
}

// Exchange-buffer swizzle of the second re-ordering (row j0, column beta ^ sw(j0)).  R = 32: the
// low three bits of j0 rotated (bit 0 to bit 2), so that the lane pairs of pass C, which read rows
// 2a and 2a + 1 at four neighbouring beta, meet eight different bank groups; the rows of one
// quarter-warp's pass-B stores stay distinct.
template <int R> __device__ __forceinline__ int sw_col(int j0)
{
    return R == 32 ? (j0 & 24) | ((j0 & 1) << 2) | ((j0 >> 1) & 3) : j0;
}
// Index of output m in the detected-power row.  R = 32: the upper half (m >= 4096) shifted by 16
// words, so that the two lanes of a pass-C pair, whose outputs are 4096 apart, store to different banks.
template <int R> __device__ __forceinline__ int pw_idx(int m) { return R == 32 ? m + ((m >> 12) << 4) : m; }

}  // namespace

// Shared memory: exchange buffer [M] float4 (X re, Y re, X im, Y im), pass-A twiddles
// W_M^{t m0} [15][T], pass-B twiddles W_M^{16 j0 m1} [15][R], detected powers [M], and the
// TMEM base address.
template <int R> static size_t smem_pair()
{
    using L = PairLayout<R>;
    return 16u * L::M + 8u * 15u * (L::T + R) + 4u * (L::M + (R == 32 ? 16 : 0)) + 16u;
}

template <int R, bool UNIFORM>
__global__ void __launch_bounds__(PairLayout<R>::T, PairLayout<R>::ctas_per_sm)
k_dedisperse_pair(const float4 *__restrict__ spec, const uint2 *__restrict__ nco, const double *__restrict__ ktab,
                  const double *__restrict__ dm_list, const float2 *__restrict__ tw_a, const float2 *__restrict__ tw_b,
                  float *__restrict__ out, int nsub, int kc, int64_t k0, int nchan, int ndm, int dm_tile, int nd,
                  int nint, int64_t nout, float scale, const int *__restrict__ round_dev, int64_t nseg, int dm_off,
                  int dm_cnt, int64_t tlim)
{
    using L = PairLayout<R>;
    constexpr int kM = L::M, kT = L::T, kR = R;
    constexpr uint32_t kTmemCols = L::tmem_cols;
    extern __shared__ __align__(16) float4 smem[];
    float4 *ex = smem;
    float2 *ta = reinterpret_cast<float2 *>(ex + kM);
    float2 *tb = ta + 15 * kT;
    float *pw = reinterpret_cast<float *>(tb + 15 * kR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(pw + kM + (R == 32 ? 16 : 0));

    const int t = threadIdx.x, warp = t >> 5;
    int64_t item = blockIdx.x;
    const int c = (int)(item % nchan); item /= nchan;
    const int kk = (int)(item % kc); item /= kc;
    const int s = (int)(item % nsub); item /= nsub;
    const int tile = (int)item;
    const int dm0 = tile * dm_tile + dm_off;
    const int ndt = min(dm_cnt, ndm - dm0);
    // every early return depends on the item only (before tensor memory is allocated)
    if (ndt <= 0) return;
    if (round_dev && (int64_t)(*round_dev) * kc + kk >= nseg) return;
    const int64_t room = tlim - (k0 + kk) * (int64_t)((kM - nd) / nint);
    const int ulim = room <= 0 ? 0 : (int)(room < (kM - nd) / nint ? room : (kM - nd) / nint);
    if (ulim == 0) return;

    if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
    for (int i = t; i < 15 * kT; i += kT) ta[i] = tw_a[i];
    for (int i = t; i < 15 * kR; i += kT) tb[i] = tw_b[i];
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t lane = *tslot + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t col_s = lane + 64u * (uint32_t)(t >> 7);                   // spectrum words of this thread's bins
    const uint32_t col_p = lane + 64u * L::NG + 32u * (uint32_t)(t >> 7);     // phase words

    // the thread's 16 bins j2 * T + t of both polarisations, and their phase words, into tensor memory
    {
        const float4 *src = spec + (((int64_t)s * kc + kk) * nchan + c) * kM;
        #pragma unroll
        for (int h = 0; h < 2; h++) {
            uint32_t w[32];
            #pragma unroll
            for (int b = 0; b < 8; b++) {
                const float4 v = __ldg(src + (8 * h + b) * kT + t);   // (X re, X im, Y re, Y im)
                w[4 * b] = __float_as_uint(v.x);
                w[4 * b + 1] = __float_as_uint(v.z);
                w[4 * b + 2] = __float_as_uint(v.y);
                w[4 * b + 3] = __float_as_uint(v.w);
            }
            tc::tmem_st32(col_s + 32 * h, w);
        }
        const uint2 *p = UNIFORM ? nco + ((int64_t)tile * nsub + s) * (int64_t)nchan * kM + (int64_t)c * kM
                                 : reinterpret_cast<const uint2 *>(ktab + ((int64_t)s * nchan + c) * kM);
        uint32_t w[32];
        #pragma unroll
        for (int j2 = 0; j2 < 16; j2++) {
            const uint2 v = __ldg(p + j2 * kT + t);
            w[2 * j2] = v.x;
            w[2 * j2 + 1] = v.y;
        }
        tc::tmem_st32(col_p, w);
    }

    const int half = nd / 2;
    const int seglen = (kM - nd) / nint;
    const int64_t rows = (int64_t)nsub * nchan;
    const int64_t obase = (int64_t)(s * nchan + c) * nout + (k0 + kk) * seglen;
    const bool pow2 = (nint & (nint - 1)) == 0 && nint <= 32;
    const int rot = pow2 ? (((t & 31) * nint) >> 5) : 0;   // conflict-free integration: rotated start

    for (int d = 0; d < ndt; d++) {
        P2 x[16];
        double dmv = 0.0;
        if constexpr (!UNIFORM) dmv = dm_list[dm0 + d];
        // ---- chirp, four bins per tensor-memory load
        #pragma unroll
        for (int g = 0; g < 4; g++) {
            uint32_t sw[16], pwd[8];
            tc::tmem_ld16_async(col_s + 16 * g, sw);
            tc::tmem_ld8_async(col_p + 8 * g, pwd);
            tc::tmem_wait();
            #pragma unroll
            for (int b = 0; b < 4; b++) {
                float sn, cs;
                if constexpr (UNIFORM) {
                    const int32_t ph = (int32_t)(pwd[2 * b] + (uint32_t)(dm_off + d) * pwd[2 * b + 1]);
                    __sincosf((float)ph * kPhaseScale, &sn, &cs);
                } else {
                    const double kj = __hiloint2double((int)pwd[2 * b + 1], (int)pwd[2 * b]);
                    double cyc = dmv * kj;
                    cyc -= rint(cyc);
                    __sincosf(-6.283185307179586f * (float)cyc, &sn, &cs);
                }
                const float xr = __uint_as_float(sw[4 * b]), yr = __uint_as_float(sw[4 * b + 1]);
                const float xi = __uint_as_float(sw[4 * b + 2]), yi = __uint_as_float(sw[4 * b + 3]);
                x[4 * g + b] = {pk2(fmaf(xr, cs, -xi * sn), fmaf(yr, cs, -yi * sn)),
                                pk2(fmaf(xr, sn, xi * cs), fmaf(yr, sn, yi * cs))};
            }
        }
        // ---- pass A: 16-point DFTs over j2, twiddles W_M^{t m0}
        pdft16<+1>(x);
        #pragma unroll
        for (int m0 = 1; m0 < 16; m0++) x[m0] = ptwiddle(x[m0], ta[(m0 - 1) * kT + t]);
        #pragma unroll
        for (int m0 = 0; m0 < 16; m0++) st_pair(ex + m0 * kT + (t ^ ((m0 * kR) & 15)), x[m0]);
        __syncthreads();
        // ---- pass B: thread (m0, j0), 16-point DFTs over j1, twiddles W_M^{16 j0 m1}
        {
            const int m0 = t / kR, j0 = t % kR;
            #pragma unroll
            for (int j1 = 0; j1 < 16; j1++) x[j1] = ld_pair(ex + m0 * kT + ((j1 * kR + j0) ^ ((m0 * kR) & 15)));
            __syncthreads();
            pdft16<+1>(x);
            #pragma unroll
            for (int m1 = 1; m1 < 16; m1++) x[m1] = ptwiddle(x[m1], tb[(m1 - 1) * kR + j0]);
            #pragma unroll
            for (int m1 = 0; m1 < 16; m1++) st_pair(ex + j0 * 256 + ((m0 + 16 * m1) ^ sw_col<R>(j0)), x[m1]);
        }
        __syncthreads();
        // ---- pass C: radix-R butterflies over j0, output m = beta + 256 m2; detection
        if constexpr (R == 8) {   // beta = t, t + T; inputs j0 < 8
            #pragma unroll
            for (int i = 0; i < 2; i++) {
                const int beta = t + kT * i;
                P2 y[8];
                #pragma unroll
                for (int j0 = 0; j0 < 8; j0++) y[j0] = ld_pair(ex + j0 * 256 + (beta ^ j0));
                pdft8<+1>(y);
                #pragma unroll
                for (int m2 = 0; m2 < 8; m2++) {
                    float px, py;
                    up2(fma2(y[m2].re, y[m2].re, mul2(y[m2].im, y[m2].im)), px, py);
                    pw[beta + 256 * m2] = px + py;
                }
            }
        } else if constexpr (R == 16) {   // beta = t
            #pragma unroll
            for (int j0 = 0; j0 < 16; j0++) x[j0] = ld_pair(ex + j0 * 256 + (t ^ j0));
            pdft16<+1>(x);
            #pragma unroll
            for (int m2 = 0; m2 < 16; m2++) {
                float px, py;
                up2(fma2(x[m2].re, x[m2].re, mul2(x[m2].im, x[m2].im)), px, py);
                pw[t + 256 * m2] = px + py;
            }
        } else {   // R = 32: lanes 2 beta + e share beta's butterfly, inputs j0 = 2a + e
            const int beta = t >> 1, e = t & 1;
            #pragma unroll
            for (int a = 0; a < 16; a++) x[a] = ld_pair(ex + (2 * a + e) * 256 + (beta ^ sw_col<R>(2 * a + e)));
            pdft16<+1>(x);
            pjoin32<+1>(x, e);
            #pragma unroll
            for (int k = 0; k < 16; k++) {
                float px, py;
                up2(fma2(x[k].re, x[k].re, mul2(x[k].im, x[k].im)), px, py);
                pw[pw_idx<R>(beta + 256 * (k + 16 * e))] = px + py;
            }
        }
        __syncthreads();
        float *orow = out + ((int64_t)tile * dm_cnt + d) * rows * nout + obase;
        for (int u = t; u < ulim; u += kT) {
            const int m = half + u * nint;
            float acc = 0.f;
            if (pow2) {
                for (int q = 0; q < nint; q++) acc += pw[pw_idx<R>(m + ((q + rot) & (nint - 1)))];
            } else {
                for (int q = 0; q < nint; q++) acc += pw[pw_idx<R>(m + q)];
            }
            orow[u] = acc * scale;
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_free(*tslot, kTmemCols);
}

template <int R> static cudaError_t prepare_pair()
{
    cudaError_t e = cudaFuncSetAttribute(k_dedisperse_pair<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_pair<R>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_dedisperse_pair<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_pair<R>());
}

cudaError_t fp32_pair_prepare(int r)
{
    return r == 8 ? prepare_pair<8>() : r == 16 ? prepare_pair<16>() : r == 32 ? prepare_pair<32>()
                                                                          : cudaErrorInvalidValue;
}

size_t fp32_pair_smem(int r)
{
    return r == 8 ? smem_pair<8>() : r == 16 ? smem_pair<16>() : r == 32 ? smem_pair<32>() : 0;
}

template <int R> static void launch_pair(const DedispArgs &a, cudaStream_t st)
{
    const int64_t ntile = (a.ndm + a.dm_tile - 1) / a.dm_tile;
    const int64_t nblk = ntile * a.nsub * a.kc * a.nchan;
    const int cnt = a.dm_cnt > 0 ? a.dm_cnt : a.dm_tile;
    if (a.uniform)
        k_dedisperse_pair<R, true><<<(unsigned)nblk, PairLayout<R>::T, smem_pair<R>(), st>>>(
            a.spec, a.nco, a.ktab, a.dm_list, a.tw_a, a.tw_b, a.out, a.nsub, a.kc, a.k0, a.nchan, a.ndm, a.dm_tile,
            a.nd, a.nint, a.nout, a.scale, a.round_dev, a.nseg, a.dm_off, cnt, a.tlim);
    else
        k_dedisperse_pair<R, false><<<(unsigned)nblk, PairLayout<R>::T, smem_pair<R>(), st>>>(
            a.spec, a.nco, a.ktab, a.dm_list, a.tw_a, a.tw_b, a.out, a.nsub, a.kc, a.k0, a.nchan, a.ndm, a.dm_tile,
            a.nd, a.nint, a.nout, a.scale, a.round_dev, a.nseg, a.dm_off, cnt, a.tlim);
}

cudaError_t fp32_dedisperse_pair(const DedispArgs &a, cudaStream_t st)
{
    if (a.r == 8) launch_pair<8>(a, st);
    else if (a.r == 16) launch_pair<16>(a, st);
    else if (a.r == 32) launch_pair<32>(a, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace cdmt
