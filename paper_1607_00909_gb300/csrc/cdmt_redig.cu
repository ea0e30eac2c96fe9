// Redigitisation of a plan's filterbank to 8 bits (Sec. 3: after the
// transpose, "compute block sums", "compute channel statistics" and
// "redigitize" of Algorithm 1).  The data offsets and scales of every channel
// follow from the mean and standard deviation of its samples in the block;
// one kernel forms the sums and the statistics of each (DM, channel) row, a
// second one converts the samples and writes them in the paper's filterbank
// order: per DM, time-major spectra in decreasing frequency.
//
// The mapping (left open by the paper): code = clamp(rint((I - mu) * g + 128),
// 0, 255) with g = 16 / sigma, evaluated in FP32 as one fused multiply-add.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/cdmt.h"
#include "cdmt_plan_impl.h"

namespace {

constexpr int kTile = 64;

// Spectral-kurtosis flag of a row of n samples, each a sum of k squared
// magnitudes, from its mean and (population) standard deviation: the
// generalised estimator SK = (n k + 1) / (n - 1) * sigma^2 / mu^2 (n S2 / S1^2
// - 1 = sigma^2 / mu^2), flagged when |SK - 1| > nsigma sqrt(2 (k + 1) / (k n)),
// its large-n deviation for Gaussian voltages; mu = 0 gives SK = 0 and fewer
// than two samples are never flagged.  nsigma <= 0: no flagging.
struct SkRule {
    float nsigma = 0.f;
    int k = 1;
    uint8_t *flags = nullptr;   // [rows of the launch] (may be NULL)
};

__device__ __forceinline__ bool sk_flag(double mu, double sigma, int64_t n, const SkRule &sk)
{
    if (!(sk.nsigma > 0.f) || n < 2) return false;
    const double nn = (double)n, k = (double)sk.k;
    const double v = mu > 0.0 ? (nn * k + 1.0) / (nn - 1.0) * (sigma * sigma) / (mu * mu) : 0.0;
    return fabs(v - 1.0) > (double)sk.nsigma * sqrt(2.0 * (k + 1.0) / (k * nn));
}

__device__ __forceinline__ bool sk_flag_f(float mu, float sigma, int64_t n, const SkRule &sk)
{
    if (!(sk.nsigma > 0.f) || n < 2) return false;
    const float nn = (float)n, k = (float)sk.k;
    const float v = mu > 0.f ? (nn * k + 1.f) / (nn - 1.f) * (sigma * sigma) / (mu * mu) : 0.f;
    return fabsf(v - 1.f) > sk.nsigma * sqrtf(2.f * (k + 1.f) / (k * nn));
}

// One CTA per (DM, channel) row of nt samples (rows of kShortRow samples or
// more; shorter rows use k_redig_stats_rows): sums of I and I^2 (FP32 within a
// thread, FP64 across threads), then mean mu, standard deviation sigma, and the
// row's (mu, g = levels / sigma) as FP32.  VEC: rows start 16-byte aligned
// (stride % 4 == 0) and are read as float4, four loads in flight per thread.
template <bool VEC>
__global__ void __launch_bounds__(256) k_redig_stats(const float *__restrict__ fb, int64_t nt, int64_t stride,
                                                     float2 *__restrict__ mg, float *__restrict__ stats, SkRule sk)
{
    const int64_t row = blockIdx.x;
    const float *p = fb + row * stride;
    float s1 = 0.f, s2 = 0.f;
    if constexpr (VEC) {
        const float4 *p4 = reinterpret_cast<const float4 *>(p);
        const int64_t n4 = nt / 4;
        #pragma unroll 4
        for (int64_t t = threadIdx.x; t < n4; t += blockDim.x) {
            const float4 v = __ldg(p4 + t);
            s1 += (v.x + v.y) + (v.z + v.w);
            s2 = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, s2))));
        }
        for (int64_t t = 4 * n4 + threadIdx.x; t < nt; t += blockDim.x) {   // the last nt % 4 samples
            const float v = __ldg(p + t);
            s1 += v;
            s2 = fmaf(v, v, s2);
        }
    } else {
        #pragma unroll 4
        for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) {
            const float v = __ldg(p + t);
            s1 += v;
            s2 = fmaf(v, v, s2);
        }
    }
    double d1 = s1, d2 = s2;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d1 += __shfl_xor_sync(0xffffffffu, d1, o);
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    }
    __shared__ double r1[8], r2[8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        r1[w] = d1;
        r2[w] = d2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
            a += r1[i];
            b += r2[i];
        }
        const double mu = nt > 0 ? a / (double)nt : 0.0;
        const double var = nt > 0 ? fmax(b / (double)nt - mu * mu, 0.0) : 0.0;
        const double sigma = sqrt(var);
        const bool flag = sk_flag(mu, sigma, nt, sk);
        // the gain from sigma rounded to FP32, divided in FP32: the codes then follow from the
        // reported (mu, sigma) alone
        mg[row] = make_float2((float)mu, sigma > 0.0 && !flag ? (float)CDMT_REDIG_LEVELS / (float)sigma : 0.f);
        if (sk.flags) sk.flags[row] = flag;
        if (stats) {
            stats[2 * row] = (float)mu;
            stats[2 * row + 1] = (float)sigma;
        }
    }
}

// Rows shorter than kShortRow samples (a served block holds one or two
// segments per row): one warp per row, eight rows per CTA, all in FP32 (the
// GPU's FP64 rate would make a per-row FP64 epilogue the bottleneck for
// millions of short rows).  Two passes over the row (the second one hits the
// cache): the mean, then the mean squared deviation from it, which has no
// cancellation even when sigma << mu.
constexpr int64_t kShortRow = 8192;

__device__ __forceinline__ float warp_sum(float v)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool VEC>
__global__ void __launch_bounds__(256) k_redig_stats_rows(const float *__restrict__ fb, int64_t nrow, int64_t nt,
                                                          int64_t stride, float2 *__restrict__ mg,
                                                          float *__restrict__ stats, SkRule sk)
{
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= nrow) return;
    const int lane = threadIdx.x & 31;
    const float *p = fb + row * stride;
    const float4 *p4 = reinterpret_cast<const float4 *>(p);
    const int64_t n4 = VEC ? nt / 4 : 0;   // float4 part; samples from 4 n4 on are read singly
    float s1 = 0.f;
    #pragma unroll 4
    for (int64_t t = lane; t < n4; t += 32) {
        const float4 v = __ldg(p4 + t);
        s1 += (v.x + v.y) + (v.z + v.w);
    }
    for (int64_t t = 4 * n4 + lane; t < nt; t += 32) s1 += __ldg(p + t);
    const float mu = warp_sum(s1) / (float)nt;
    float s2 = 0.f;
    #pragma unroll 4
    for (int64_t t = lane; t < n4; t += 32) {
        const float4 v = __ldg(p4 + t);
        const float a = v.x - mu, b = v.y - mu, c = v.z - mu, d = v.w - mu;
        s2 = fmaf(a, a, fmaf(b, b, fmaf(c, c, fmaf(d, d, s2))));
    }
    for (int64_t t = 4 * n4 + lane; t < nt; t += 32) {
        const float a = __ldg(p + t) - mu;
        s2 = fmaf(a, a, s2);
    }
    const float sigma = sqrtf(warp_sum(s2) / (float)nt);
    if (lane == 0) {
        const bool flag = sk_flag_f(mu, sigma, nt, sk);
        mg[row] = make_float2(mu, sigma > 0.f && !flag ? (float)CDMT_REDIG_LEVELS / sigma : 0.f);
        if (sk.flags) sk.flags[row] = flag;
        if (stats) {
            stats[2 * row] = mu;
            stats[2 * row + 1] = sigma;
        }
    }
}

__device__ __forceinline__ uint8_t code8(float v, float2 m)
{
    const float x = rintf(fmaf(v - m.x, m.y, 128.f));
    return (uint8_t)fminf(fmaxf(x, 0.f), 255.f);
}

// One CTA per (64-sample, 64-row) tile of one DM: codes into shared memory,
// then each output spectrum's 64 bytes (rows reversed) in 4-byte words.  VEC:
// full-width tiles of 16-byte aligned rows are read as float4 (4 per thread).
// Rows of the filterbank are `stride` floats apart; nt samples of each are coded.
// Short rows in one pass: one CTA per R rows of one DM stages them in shared
// memory by asynchronous copies (16-byte chunks where rows are 16-byte aligned),
// takes each row's statistics from there (as k_redig_stats_rows: FP32 mean,
// then mean squared deviation; spectral-kurtosis flag) and writes the R rows'
// codes of every sample, rows reversed, as 4-byte words: one read of the
// filterbank instead of two.  Row r starts at r * ldr + 4 ((r / 4) mod 8)
// floats (ldr a multiple of 32): the code pass reads 8 rows 4 apart at 4
// consecutive samples per instruction, which then meet 32 distinct banks.
__host__ __device__ constexpr int fused_ldr(int64_t nt) { return (int)((nt + 31) / 32 * 32) + 32; }

template <int R>
__global__ void __launch_bounds__(256) k_redig_fused(const float *__restrict__ fb, int rows, int64_t nt,
                                                     int64_t stride, uint8_t *__restrict__ out,
                                                     float *__restrict__ stats, SkRule sk, bool vec)
{
    extern __shared__ __align__(16) float sm[];
    const int ldr = fused_ldr(nt);
    float *tile = sm;               // [R][ldr]
    float *mus = sm + R * ldr;      // [R]
    float *gs = mus + R;            // [R]
    auto at = [&](int r, int t) { return r * ldr + 4 * ((r >> 2) & 7) + t; };
    const int dm = blockIdx.y;
    const int r0 = blockIdx.x * R;
    const int nr = min(R, rows - r0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float *src = fb + ((int64_t)dm * rows + r0) * stride;
    const uint32_t tile_s = (uint32_t)__cvta_generic_to_shared(tile);
    const int n4 = vec ? (int)(nt / 4) : 0;   // 16-byte chunks per row; samples from 4 n4 on singly
    for (int r = warp; r < nr; r += 8) {
        const float *row = src + (int64_t)r * stride;
        for (int c = lane; c < n4; c += 32)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tile_s + 4u * (uint32_t)at(r, 4 * c)),
                         "l"(row + 4 * c)
                         : "memory");
        for (int t = 4 * n4 + lane; t < nt; t += 32)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tile_s + 4u * (uint32_t)at(r, t)),
                         "l"(row + t)
                         : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (int r = warp; r < nr; r += 8) {
        const float *x = tile + at(r, 0);
        float s1 = 0.f;
        for (int t = lane; t < nt; t += 32) s1 += x[t];
        const float mu = warp_sum(s1) / (float)nt;
        float s2 = 0.f;
        for (int t = lane; t < nt; t += 32) {
            const float a = x[t] - mu;
            s2 = fmaf(a, a, s2);
        }
        const float sigma = sqrtf(warp_sum(s2) / (float)nt);
        if (lane == 0) {
            const bool flag = sk_flag_f(mu, sigma, nt, sk);
            mus[r] = mu;
            gs[r] = sigma > 0.f && !flag ? (float)CDMT_REDIG_LEVELS / sigma : 0.f;
            const int64_t g = (int64_t)dm * rows + r0 + r;
            if (sk.flags) sk.flags[g] = flag;
            if (stats) {
                stats[2 * g] = mu;
                stats[2 * g + 1] = sigma;
            }
        }
    }
    __syncthreads();
    // spectrum t of this DM: row r0 + rr at position rows - 1 - r0 - rr
    uint8_t *dst = out + (int64_t)dm * nt * rows + (rows - r0 - nr);
    if (nr == R && (rows & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 3) == 0) {
        constexpr int W = R / 4;    // 4-byte words of the R rows in one spectrum
        // a thread keeps one word position (the block's threads are a multiple of W): its four
        // rows' (mean, gain) stay in registers
        const int wd = (int)(threadIdx.x % W);
        const int rr = R - 1 - 4 * wd;   // rows rr, rr-1, rr-2, rr-3 at positions 4wd .. 4wd+3
        float2 mg[4];
        #pragma unroll
        for (int b = 0; b < 4; b++) mg[b] = make_float2(mus[rr - b], gs[rr - b]);
        for (int64_t t = threadIdx.x / W; t < nt; t += blockDim.x / W) {
            uint32_t v = 0;
            #pragma unroll
            for (int b = 0; b < 4; b++) v |= (uint32_t)code8(tile[at(rr - b, (int)t)], mg[b]) << (8 * b);
            *reinterpret_cast<uint32_t *>(dst + t * rows + 4 * wd) = v;
        }
    } else {
        for (int64_t i = threadIdx.x; i < nt * nr; i += blockDim.x) {
            const int t = (int)(i / nr), pos = (int)(i % nr);
            const int rr = nr - 1 - pos;
            dst[(int64_t)t * rows + pos] = code8(tile[at(rr, t)], make_float2(mus[rr], gs[rr]));
        }
    }
}

// Dynamic shared memory of k_redig_fused<R> for rows of nt samples.
constexpr size_t fused_smem(int r, int64_t nt) { return sizeof(float) * ((size_t)r * (size_t)fused_ldr(nt) + 2 * (size_t)r); }
// at most 110 KB, so that two CTAs share an SM (one CTA per SM leaves too few copies in flight)
constexpr size_t kFusedSmemMax = 110 * 1024;

template <bool VEC>
__global__ void __launch_bounds__(256) k_redig_codes(const float *__restrict__ fb, const float2 *__restrict__ mg,
                                                     uint8_t *__restrict__ out, int rows, int64_t nt, int64_t stride)
{
    __shared__ uint8_t tile[kTile][kTile + 4];   // [sample][row]
    const int dm = blockIdx.z;
    const int r0 = blockIdx.y * kTile;
    const int64_t t0 = (int64_t)blockIdx.x * kTile;
    const int nr = min(kTile, rows - r0);
    const int ntt = (int)(nt - t0 < kTile ? nt - t0 : kTile);
    const float *src = fb + ((int64_t)dm * rows + r0) * stride + t0;
    const float2 *g = mg + (int64_t)dm * rows + r0;
    if (VEC && ntt == kTile) {
        #pragma unroll
        for (int k = 0; k < kTile * kTile / 4 / 256; k++) {
            const int i = k * 256 + (int)threadIdx.x;
            const int rr = i / (kTile / 4), tt = 4 * (i % (kTile / 4));
            if (rr < nr) {
                const float2 m = g[rr];
                const float4 v = __ldg(reinterpret_cast<const float4 *>(src + (int64_t)rr * stride + tt));
                tile[tt][rr] = code8(v.x, m);
                tile[tt + 1][rr] = code8(v.y, m);
                tile[tt + 2][rr] = code8(v.z, m);
                tile[tt + 3][rr] = code8(v.w, m);
            }
        }
    } else {
        for (int i = threadIdx.x; i < kTile * kTile; i += blockDim.x) {
            const int rr = i / kTile, tt = i % kTile;
            if (rr < nr && tt < ntt) tile[tt][rr] = code8(__ldg(src + (int64_t)rr * stride + tt), g[rr]);
        }
    }
    __syncthreads();
    // output position of row r0 + rr within a spectrum: rows - 1 - r0 - rr
    uint8_t *dst = out + ((int64_t)dm * nt + t0) * rows + (rows - r0 - nr);
    if (nr == kTile && (rows & 3) == 0) {
        for (int i = threadIdx.x; i < ntt * (kTile / 4); i += blockDim.x) {
            const int tt = i / (kTile / 4), wd = i % (kTile / 4);
            const int rr = kTile - 1 - 4 * wd;   // rows rr, rr-1, rr-2, rr-3 at positions 4wd .. 4wd+3
            const uint32_t v = (uint32_t)tile[tt][rr] | ((uint32_t)tile[tt][rr - 1] << 8) |
                               ((uint32_t)tile[tt][rr - 2] << 16) | ((uint32_t)tile[tt][rr - 3] << 24);
            *reinterpret_cast<uint32_t *>(dst + (int64_t)tt * rows + 4 * wd) = v;
        }
    } else {
        for (int i = threadIdx.x; i < ntt * nr; i += blockDim.x) {
            const int tt = i / nr, pos = i % nr;
            dst[(int64_t)tt * rows + pos] = tile[tt][nr - 1 - pos];
        }
    }
}

int rfail(cdmt_plan_s *p, int code, const char *msg)
{
    p->last_error = msg;
    return code;
}

}  // namespace

namespace cdmt {

// Redigitisation of a filterbank [ndm][nsub*nchan][stride] whose first nt samples per row form
// one block, into d_u8 [ndm][nt][nsub*nchan] (decreasing frequency); plan-owned (mu, g) array.
int redig_reserve(cdmt_plan_s *p)
{
    const int rows = p->nsub * p->nchan;
    if (p->ndm > 65535 || (rows + kTile - 1) / kTile > 65535)
        return rfail(p, CDMT_ENOTSUP, "more than 65535 DM trials or 64-row tiles");
    if (!p->redig_mg) {
        if (cudaMalloc((void **)&p->redig_mg, sizeof(float2) * (size_t)p->ndm * rows) != cudaSuccess) {
            cudaGetLastError();
            return rfail(p, CDMT_ENOMEM, "redigitisation statistics buffer");
        }
        p->bytes += (int64_t)sizeof(float2) * p->ndm * rows;
    }
    return CDMT_OK;
}

int redig_enqueue(cdmt_plan_s *p, const float *d_fb, int64_t nt, int64_t stride, uint8_t *d_u8, float *d_stats,
                  cudaStream_t st, double sk_nsigma, uint8_t *d_flags, int ndm_r)
{
    const cdmt::Range range("cdmt redigitisation");
    const int rows = p->nsub * p->nchan;
    const int ndm = ndm_r > 0 ? ndm_r : p->ndm;   // DMs in d_fb (a range of the plan's)
    if (nt < 1) return rfail(p, CDMT_EINVAL, "no samples to redigitise");
    const int rc = redig_reserve(p);
    if (rc != CDMT_OK) return rc;
    // float4 reads need every row to start 16-byte aligned (rows' last nt % 4 samples are read singly)
    const bool vec = stride % 4 == 0 && (reinterpret_cast<uintptr_t>(d_fb) & 15) == 0;
    const unsigned nrow = (unsigned)((int64_t)ndm * rows);
    const dim3 grid((unsigned)((nt + kTile - 1) / kTile), (unsigned)((rows + kTile - 1) / kTile), (unsigned)ndm);
    const unsigned nrow8 = (nrow + 7) / 8;
    SkRule sk;
    sk.nsigma = sk_nsigma > 0.0 ? (float)sk_nsigma : 0.f;
    sk.k = 2 * p->nint;
    sk.flags = d_flags;
    // short rows: one pass, 32 (or 16) rows of a DM staged in shared memory
    const int fr = fused_smem(32, nt) <= kFusedSmemMax ? 32 : fused_smem(16, nt) <= kFusedSmemMax ? 16 : 0;
    if (fr) {
        const size_t smem = fused_smem(fr, nt);
        // set on every call: the attribute is per device, and plans on several devices or
        // threads may launch this kernel (the call costs microseconds)
        const cudaError_t ea = fr == 32 ? cudaFuncSetAttribute(k_redig_fused<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               (int)kFusedSmemMax)
                                        : cudaFuncSetAttribute(k_redig_fused<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               (int)kFusedSmemMax);
        if (ea != cudaSuccess) return rfail(p, CDMT_ECUDA, cudaGetErrorString(ea));
        const dim3 fg((unsigned)((rows + fr - 1) / fr), (unsigned)ndm);
        if (fr == 32) k_redig_fused<32><<<fg, 256, smem, st>>>(d_fb, rows, nt, stride, d_u8, d_stats, sk, vec);
        else k_redig_fused<16><<<fg, 256, smem, st>>>(d_fb, rows, nt, stride, d_u8, d_stats, sk, vec);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return rfail(p, CDMT_ECUDA, cudaGetErrorString(e));
        return CDMT_OK;
    }
    if (vec) {
        if (nt < kShortRow) k_redig_stats_rows<true><<<nrow8, 256, 0, st>>>(d_fb, nrow, nt, stride, p->redig_mg, d_stats, sk);
        else k_redig_stats<true><<<nrow, 256, 0, st>>>(d_fb, nt, stride, p->redig_mg, d_stats, sk);
        k_redig_codes<true><<<grid, 256, 0, st>>>(d_fb, p->redig_mg, d_u8, rows, nt, stride);
    } else {
        if (nt < kShortRow) k_redig_stats_rows<false><<<nrow8, 256, 0, st>>>(d_fb, nrow, nt, stride, p->redig_mg, d_stats, sk);
        else k_redig_stats<false><<<nrow, 256, 0, st>>>(d_fb, nt, stride, p->redig_mg, d_stats, sk);
        k_redig_codes<false><<<grid, 256, 0, st>>>(d_fb, p->redig_mg, d_u8, rows, nt, stride);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rfail(p, CDMT_ECUDA, cudaGetErrorString(e));
    return CDMT_OK;
}

}  // namespace cdmt

extern "C" int cdmt_redigitise_sk(cdmt_plan_t p, const float *d_fb, uint8_t *d_u8, float *d_stats, double sk_nsigma,
                                  uint8_t *d_flags, void *cuda_stream)
{
    if (!p) return CDMT_EINVAL;
    if (!d_fb || !d_u8) return rfail(p, CDMT_EINVAL, "NULL filterbank or output pointer");
    if (!(sk_nsigma >= 0.0)) return rfail(p, CDMT_EINVAL, "sk_nsigma must be >= 0");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device && cudaSetDevice(p->device) != cudaSuccess) return rfail(p, CDMT_ECUDA, "cudaSetDevice failed");
    const int rc = cdmt::redig_enqueue(p, d_fb, p->nout, p->nout, d_u8, d_stats, static_cast<cudaStream_t>(cuda_stream),
                                       sk_nsigma, d_flags);
    if (cur != p->device) cudaSetDevice(cur);
    return rc;
}

extern "C" int cdmt_redigitise(cdmt_plan_t p, const float *d_fb, uint8_t *d_u8, float *d_stats, void *cuda_stream)
{
    return cdmt_redigitise_sk(p, d_fb, d_u8, d_stats, 0.0, nullptr, cuda_stream);
}
