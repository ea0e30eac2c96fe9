// Device FFT machinery for the coherent-dedispersion kernels.
//
// An M-point DFT (M = 256 R, R in {2, 4, 8, 16, 32}) is computed by T = M/16
// threads in three radix passes, P = 16, Q = 16 and R (a three-factor
// Cooley-Tukey decomposition).  With input index j = j2 (16R) + j1 R + j0 and output index
// m = m0 + 16 m1 + 256 m2:
//   pass A  thread t = j1 R + j0:   a[m0]  = sum_j2 x[j2 T + t] W_16^{j2 m0},  a *= W_M^{t m0}
//   pass B  thread u = m0 R + j0:   b[m1]  = sum_j1 a[m0; j1, j0] W_16^{j1 m1}, b *= W_M^{16 j0 m1}
//   pass C  butterfly (m0, m1):     y[m2]  = sum_j0 b[m0, m1; j0] W_R^{j0 m2}
// W_n = exp(S 2 pi i / n), S = -1 forward, +1 backward.  Each thread keeps 16
// points in registers, of both polarisations (float4 exchange elements:
// X re, X im, Y re, Y im) or of one (float2 elements); the two re-orderings
// between passes go through one shared-memory buffer of M elements.  The buffer
// indices carry an XOR swizzle on their low four bits that makes every access
// pattern of the passes free of bank conflicts (16-byte elements per
// quarter-warp, 8-byte elements per half-warp) for R <= 16.  With R = 32 each
// radix-32 butterfly of pass C is shared by two neighbouring lanes: lane e of
// the pair takes the 16 inputs j0 = 2a + e, runs their 16-point DFT, and one
// radix-2 step with W_32^k, its operands swapped through lane shuffles, gives
// outputs m2 = k + 16 e (decimation in time).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cdmt {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * (S i)
template <int S> __device__ __forceinline__ float2 mul_i(float2 a)
{
    return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// a * (c + S i s) for compile-time constants
template <int S> __device__ __forceinline__ float2 mul_cs(float2 a, float c, float s)
{
    const float ss = S > 0 ? s : -s;
    return make_float2(fmaf(a.x, c, -a.y * ss), fmaf(a.x, ss, a.y * c));
}

// (cos, sin) of pi k / 16, k = 0..15: the radix-2 twiddles W_32^k of the R = 32 pass C
static __device__ __constant__ float kW32[16][2] = {
    {1.00000000000000000000f, 0.00000000000000000000f},
    {0.98078528040323043058f, 0.19509032201612824808f},
    {0.92387953251128673848f, 0.38268343236508978178f},
    {0.83146961230254523567f, 0.55557023301960217765f},
    {0.70710678118654757274f, 0.70710678118654746172f},
    {0.55557023301960228867f, 0.83146961230254523567f},
    {0.38268343236508983729f, 0.92387953251128673848f},
    {0.19509032201612833135f, 0.98078528040323043058f},
    {0.00000000000000000000f, 1.00000000000000000000f},
    {-0.19509032201612819257f, 0.98078528040323043058f},
    {-0.38268343236508972627f, 0.92387953251128673848f},
    {-0.55557023301960195560f, 0.83146961230254545772f},
    {-0.70710678118654746172f, 0.70710678118654757274f},
    {-0.83146961230254534669f, 0.55557023301960217765f},
    {-0.92387953251128673848f, 0.38268343236508989280f},
    {-0.98078528040323043058f, 0.19509032201612860891f}};

constexpr float kC8 = 0.70710678118654752440f;   // cos(pi/4)
constexpr float kC16 = 0.92387953251128675613f;  // cos(pi/8)
constexpr float kS16 = 0.38268343236508977173f;  // sin(pi/8)

// 2-, 4-, 8-, 16-point DFTs in registers, natural order in and out.
template <int S> __device__ __forceinline__ void dft2(float2 *v)
{
    float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
}

template <int S> __device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_i<S>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}
template <int S> __device__ __forceinline__ void dft4(float2 *v) { dft4<S>(v[0], v[1], v[2], v[3]); }

template <int S> __device__ __forceinline__ void dft8(float2 *v)
{
    // radix-2 decimation in time: X[k] = E[k] + W8^k O[k], X[k+4] = E[k] - W8^k O[k]
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<S>(e0, e1, e2, e3);
    dft4<S>(o0, o1, o2, o3);
    o1 = mul_cs<S>(o1, kC8, kC8);    // W8^1
    o2 = mul_i<S>(o2);               // W8^2
    o3 = mul_cs<S>(o3, -kC8, kC8);   // W8^3
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <int S> __device__ __forceinline__ void dft16(float2 *v)
{
    // 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2
    #pragma unroll
    for (int n2 = 0; n2 < 4; n2++) dft4<S>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    // v[4 k1 + n2] *= W16^{n2 k1}
    v[5] = mul_cs<S>(v[5], kC16, kS16);      // W^1
    v[6] = mul_cs<S>(v[6], kC8, kC8);        // W^2
    v[7] = mul_cs<S>(v[7], kS16, kC16);      // W^3
    v[9] = mul_cs<S>(v[9], kC8, kC8);        // W^2
    v[10] = mul_i<S>(v[10]);                 // W^4
    v[11] = mul_cs<S>(v[11], -kC8, kC8);     // W^6
    v[13] = mul_cs<S>(v[13], kS16, kC16);    // W^3
    v[14] = mul_cs<S>(v[14], -kC8, kC8);     // W^6
    v[15] = mul_cs<S>(v[15], -kC16, -kS16);  // W^9
    #pragma unroll
    for (int k1 = 0; k1 < 4; k1++) dft4<S>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // now v[4 k1 + k2] = X[k1 + 4 k2]: transpose the 4 x 4 register block
    float2 t;
    t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[2]; v[2] = v[8]; v[8] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[6]; v[6] = v[9]; v[9] = t;
    t = v[7]; v[7] = v[13]; v[13] = t;
    t = v[11]; v[11] = v[14]; v[14] = t;
}

template <int R, int S> __device__ __forceinline__ void dft_r(float2 *v)
{
    if constexpr (R == 2) dft2<S>(v);
    else if constexpr (R == 4) dft4<S>(v);
    else if constexpr (R == 8) dft8<S>(v);
    else dft16<S>(v);
}

__device__ __forceinline__ float4 pack(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// ---- three-pass M-point FFT, M = 256 R, T = 16 R threads ------------------------
template <int R> struct Fft3 {
    static constexpr int M = 256 * R;
    static constexpr int T = 16 * R;
    static constexpr int NTA = 15 * T;  // pass-A twiddles W_M^{t m0}, m0 = 1..15, layout [m0-1][t]
    static constexpr int NTB = 15 * R;  // pass-B twiddles W_M^{16 j0 m1}, m1 = 1..15, layout [m1-1][j0]
    static constexpr int GB = R >= 8 ? 1 : 8 / R;   // pass-B write swizzle step, 16-byte elements
    static constexpr int GB1 = R >= 16 ? 1 : 16 / R;   // the same for 8-byte elements

    __device__ __forceinline__ static int ex1(int m0, int t) { return m0 * T + (t ^ ((m0 * R) & 15)); }
    __device__ __forceinline__ static int ex2(int j0, int beta) { return j0 * 256 + (beta ^ (j0 * GB)); }
    __device__ __forceinline__ static int ex2s(int j0, int beta) { return j0 * 256 + (beta ^ (j0 * GB1)); }

    // ---- one polarisation per thread (float2 exchange) ----
    template <int S>
    __device__ __forceinline__ static void pass_a1(float2 *x, float2 *ex, const float2 *ta, int t)
    {
        dft16<S>(x);
        #pragma unroll
        for (int m0 = 1; m0 < 16; m0++) x[m0] = cmul(x[m0], ta[(m0 - 1) * T + t]);
        #pragma unroll
        for (int m0 = 0; m0 < 16; m0++) ex[ex1(m0, t)] = x[m0];
    }

    template <int S>
    __device__ __forceinline__ static void pass_b1(float2 *x, float2 *ex, const float2 *tb, int t)
    {
        const int m0 = t / R, j0 = t % R;
        #pragma unroll
        for (int j1 = 0; j1 < 16; j1++) x[j1] = ex[ex1(m0, j1 * R + j0)];
        __syncthreads();
        dft16<S>(x);
        #pragma unroll
        for (int m1 = 1; m1 < 16; m1++) x[m1] = cmul(x[m1], tb[(m1 - 1) * R + j0]);
        #pragma unroll
        for (int m1 = 0; m1 < 16; m1++) ex[ex2s(j0, m0 + 16 * m1)] = x[m1];
    }

    // R = 32: the radix-2 step joining the two 16-point halves of a butterfly held by lanes
    // (2 beta, 2 beta + 1); v holds this lane's half (inputs j0 = 2a + e), leaves its outputs
    // m2 = k + 16 e in v[k]
    template <int S> __device__ __forceinline__ static void join32(float2 *v, int e)
    {
        #pragma unroll
        for (int k = 0; k < 16; k++) {
            const float2 other = make_float2(__shfl_xor_sync(0xffffffffu, v[k].x, 1), __shfl_xor_sync(0xffffffffu, v[k].y, 1));
            const float2 ev = e ? other : v[k], od = e ? v[k] : other;
            // W_32^k = exp(S 2 pi i k / 32)
            const float2 w = cmul(od, make_float2(kW32[k][0], S > 0 ? kW32[k][1] : -kW32[k][1]));
            v[k] = e ? csub(ev, w) : cadd(ev, w);
        }
    }

    template <int S, class Emit>
    __device__ __forceinline__ static void pass_c1(const float2 *ex, int t, Emit &&emit)
    {
        if constexpr (R == 32) {
            const int beta = t >> 1, e = t & 1;
            float2 x[16];
            #pragma unroll
            for (int a = 0; a < 16; a++) x[a] = ex[ex2s(2 * a + e, beta)];
            dft16<S>(x);
            join32<S>(x, e);
            #pragma unroll
            for (int k = 0; k < 16; k++) emit(beta + 256 * (k + 16 * e), x[k]);
        } else {
            #pragma unroll
            for (int i = 0; i < 16 / R; i++) {
                const int beta = t + T * i;
                float2 x[R];
                #pragma unroll
                for (int j0 = 0; j0 < R; j0++) x[j0] = ex[ex2s(j0, beta)];
                dft_r<R, S>(x);
                #pragma unroll
                for (int m2 = 0; m2 < R; m2++) emit(beta + 256 * m2, x[m2]);
            }
        }
    }

    // x, y: the 16 points x[j2 T + t] (j2 = 0..15) of each polarisation.  Leaves
    // pass-A results in ex.  Caller synchronises before pass_b.
    template <int S>
    __device__ __forceinline__ static void pass_a(float2 *x, float2 *y, float4 *ex, const float2 *ta, int t)
    {
        dft16<S>(x);
        dft16<S>(y);
        #pragma unroll
        for (int m0 = 1; m0 < 16; m0++) {
            float2 w = ta[(m0 - 1) * T + t];
            x[m0] = cmul(x[m0], w);
            y[m0] = cmul(y[m0], w);
        }
        #pragma unroll
        for (int m0 = 0; m0 < 16; m0++) ex[ex1(m0, t)] = pack(x[m0], y[m0]);
    }

    // Reads pass-A results, synchronises (ex is reused), transforms, writes
    // pass-B results.  Caller synchronises before pass_c.
    template <int S>
    __device__ __forceinline__ static void pass_b(float2 *x, float2 *y, float4 *ex, const float2 *tb, int t)
    {
        const int m0 = t / R, j0 = t % R;
        #pragma unroll
        for (int j1 = 0; j1 < 16; j1++) {
            float4 v = ex[ex1(m0, j1 * R + j0)];
            x[j1] = make_float2(v.x, v.y);
            y[j1] = make_float2(v.z, v.w);
        }
        __syncthreads();
        dft16<S>(x);
        dft16<S>(y);
        #pragma unroll
        for (int m1 = 1; m1 < 16; m1++) {
            float2 w = tb[(m1 - 1) * R + j0];
            x[m1] = cmul(x[m1], w);
            y[m1] = cmul(y[m1], w);
        }
        #pragma unroll
        for (int m1 = 0; m1 < 16; m1++) ex[ex2(j0, m0 + 16 * m1)] = pack(x[m1], y[m1]);
    }

    // Final radix-R butterflies; emit(beta, m2, xm, ym) receives output
    // m = beta + 256 m2 (beta < 256) of both polarisations.
    template <int S, class Emit>
    __device__ __forceinline__ static void pass_c(const float4 *ex, int t, Emit &&emit)
    {
        if constexpr (R == 32) {
            const int beta = t >> 1, e = t & 1;
            float2 x[16], y[16];
            #pragma unroll
            for (int a = 0; a < 16; a++) {
                const float4 v = ex[ex2(2 * a + e, beta)];
                x[a] = make_float2(v.x, v.y);
                y[a] = make_float2(v.z, v.w);
            }
            dft16<S>(x);
            dft16<S>(y);
            join32<S>(x, e);
            join32<S>(y, e);
            #pragma unroll
            for (int k = 0; k < 16; k++) emit(beta, k + 16 * e, x[k], y[k]);
        } else {
            #pragma unroll
            for (int i = 0; i < 16 / R; i++) {
                const int beta = t + T * i;
                float2 x[R], y[R];
                #pragma unroll
                for (int j0 = 0; j0 < R; j0++) {
                    float4 v = ex[ex2(j0, beta)];
                    x[j0] = make_float2(v.x, v.y);
                    y[j0] = make_float2(v.z, v.w);
                }
                dft_r<R, S>(x);
                dft_r<R, S>(y);
                #pragma unroll
                for (int m2 = 0; m2 < R; m2++) emit(beta, m2, x[m2], y[m2]);
            }
        }
    }
};

}  // namespace cdmt
