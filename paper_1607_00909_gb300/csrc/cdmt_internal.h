// Internal interfaces between the host planner and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cdmt {

struct ForwardArgs {
    const void *in;    // first sample of the block's subband 0 (segment 0 of the chunk at in + k0 * nvalid):
                       // float4 samples, or char4 samples when i8 (times scale[subband])
    float4 *spec;      // [nsub][kc][nchan][M] float4 workspace
    const float2 *tw_a, *tw_b, *tw_n;
    int64_t nsamp;     // samples between consecutive subbands in `in`
    int64_t nvalid;    // S
    int64_t nbin;
    int64_t k0;        // first segment of the chunk, counted from `in`
    int nchan, kc, nsub, r;
    const int *round_dev = nullptr;  // batches: first segment = *round_dev * kc (k0 ignored)
    int64_t nseg = 0;                // batches: segments of the whole input
    bool i8 = false;                 // int8 samples (X re, X im, Y re, Y im) ...
    const float *scale = nullptr;    // ... times a DEVICE per-subband scale
    int *status = nullptr;           // set to 1 by a CTA whose input copy (TMA) did not complete in time
    // the one-launch forward stage's work queue: 1 + ceil(nsub * kc / 2) words (none: two launches)
    int *sync = nullptr;
    int64_t sync_n = 0;
    int nsm = 0;                     // SMs of the device
};

struct DedispArgs {
    const float4 *spec;
    const uint2 *nco;     // uniform: [ntile][nsub][nchan*M] (a, b)
    const double *ktab;   // non-uniform: [nsub][nchan*M] K (cycles per unit DM)
    const double *dm_list;
    const float2 *tw_a, *tw_b;
    float *out;
    int64_t k0;           // segment index of the chunk's first segment in the output time axis
    int64_t nout;         // output row stride (floats)
    int nsub, kc, nchan, ndm, dm_tile, nd, nint, r;
    bool uniform;
    float scale;
    const int *round_dev = nullptr;  // batches: skip segments round * kc + kk >= nseg
    int64_t nseg = 0;
    // DM range: DMs dm_off .. dm_off + dm_cnt - 1 of every tile (dm_cnt 0: the whole tile); output
    // row of DM j of tile t's range: t * dm_cnt + j
    int dm_off = 0, dm_cnt = 0;
    int64_t tlim = INT64_MAX;   // output positions (k0 + kk) * seglen + u >= tlim are not stored
};

struct TcArgs {
    const float4 *spec;
    const uint2 *nco;
    const double *ktab;
    const double *dm_list;
    const uint4 *bmat;    // F_P, the (M/64)-point DFT matrix, K-major canonical layout (hi [, lo])
    const uint4 *bmat64;  // F_64, the 64-point DFT matrix, same layout (equal to bmat when M = 4096)
    const float2 *twq;    // W_M^{j_lo m0}, pairs of m0: [m0 / 2][j_lo] (cos, cos', sin, sin')
    int lm;               // log2 M: 12 or 11
    float *out;
    int *status;          // set to 1 by a CTA whose tensor-core wait timed out
    int64_t k0, nout;
    int nsub, kc, nchan, ndm, dm_tile, nd, nint;
    int nsm;              // SMs of the device: persistent grid size
    int ab;               // 0 FP16, 1 BF16 hi/lo
    bool uniform;
    float scale;
    int dm_off = 0, dm_cnt = 0;   // DM range within every tile, as in DedispArgs
    int64_t tlim = INT64_MAX;     // output positions >= tlim are not stored, as in DedispArgs
};

// one beam of a batch, as the persistent tensor-core kernel sees it
struct TcBeam {
    const float4 *spec;   // [nsub][kc][nchan][4096] forward spectra of the round's segments
    const uint2 *nco;     // [ntile][nsub][nchan*4096] (phase, step) words
    float *out;           // round output: [ndm][nsub*nchan][out_stride], segment kk at kk * seglen
    int64_t out_stride;   // floats per output row in the round buffer (kc * seglen)
    int64_t nseg;         // segments of the whole input
    int nsub, kc, nchan, ndm, dm_tile, ntile, nd, nint;
    float scale;
};

cudaError_t tc_prepare(int ab);
cudaError_t tc_batch_launch(const TcBeam *beams, int nbeam, const int *round_dev, int *queue, const uint4 *bmat,
                            const float2 *twq, int *status, int ab, int nctas, cudaStream_t st);
size_t tc_smem(int ab, int lm);
cudaError_t tc_dedisperse(const TcArgs &a, cudaStream_t st);

// Plan tables shared by cdmt_plan_ex and cdmt_execute_static (defined with the planner):
// the FP32 form's twiddles (W_N line; forward and backward pass twiddles, tw_b = tw_a +
// 15 * 16 r), and the fixed-point chirp words (phase, step) of an evenly spaced DM list
// for ntile tiles whose first DMs are d_tile0[t] (device), or dm0 when d_tile0 is NULL
// (one tile); shift != 0 adds the tensor-core form's output-shift ramp.
cudaError_t enqueue_fp32_tables(float2 *tw_n, float2 *tw_af, float2 *tw_ai, int64_t nbin, int r, cudaStream_t st);
cudaError_t enqueue_nco_table(uint2 *nco, const double *d_tile0, double dm0, double ddm, double f_centre, double bw,
                              int nsub, int nchan, int64_t nbin, int ntile, int shift, int chirp, cudaStream_t st);
// Sec. 2's overlap for the lowest channel of the band at |DM| dm_abs_max (per-channel chirps); -1 if none < M.
int64_t overlap_for(int nsub, double f_centre, double bw, double dm_abs_max, int nchan, int nint, int64_t nbin);

cudaError_t fp32_prepare(int r);
// the DM stage at M = 4096 and 8192 (r = 16, 32): both polarisations per thread in packed f32x2
// arithmetic, the channel's spectrum and phase words in tensor memory (kernels_fp32_pair.cu)
cudaError_t fp32_pair_prepare(int r);
size_t fp32_pair_smem(int r);
cudaError_t fp32_dedisperse_pair(const DedispArgs &a, cudaStream_t st);
size_t fp32_dedisp_smem(int r);
cudaError_t fp32_forward(const ForwardArgs &a, cudaStream_t st);
cudaError_t fp32_dedisperse(const DedispArgs &a, cudaStream_t st);

}  // namespace cdmt
