// Internal definition of a plan (shared by the host translation units).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cmath>

#include <string>
#include <vector>

#include "cdmt_internal.h"

namespace cdmt {

// A named NVTX range over the host code that enqueues a stage, for tools that
// trace (ncu --nvtx, Nsight Systems); without such a tool attached it costs a
// branch.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

struct Staging {
    float4 *in = nullptr;   // [nsub][span_max] samples
    float *out = nullptr;   // [DMs of a range][nsub*nchan][kc_max*seglen]
    uint8_t *u8 = nullptr;  // [ndm][kc_max*seglen][nsub*nchan] codes (8-bit host output)
    cudaEvent_t in_free = nullptr, in_ready = nullptr, out_ready = nullptr, out_free = nullptr;
};


}  // namespace cdmt

struct cdmt_plan_s {
    int device = 0;
    int nsm = 148;         // SMs of the device
    int nsub = 0, nchan = 0, nint = 0, ndm = 0;
    int64_t nsamp = 0;
    double f_centre = 0, bw = 0;
    std::vector<double> dms;
    int64_t nbin = 0, mbin = 0, nd = 0, nvalid = 0, nseg = 0, nout = 0, seglen = 0;
    int r = 0;
    bool uniform = true;
    double ddm = 0;
    int dm_tile = 0, ntile = 0;
    int64_t seg_chunk = 0;
    int precision = 0, in_dtype = 0;
    int chirp = 0;         // enum cdmt_chirp
    int64_t mem_budget = 0;
    // device tables
    float2 *tw_n = nullptr, *tw_af = nullptr, *tw_bf = nullptr, *tw_ai = nullptr, *tw_bi = nullptr;
    uint2 *nco = nullptr;
    double *ktab = nullptr, *d_dm = nullptr;
    float4 *spec = nullptr;
    // tensor-core form
    uint4 *tc_bmat = nullptr;     // F_P, P = M / 64
    uint4 *tc_bmat64 = nullptr;   // F_64 (the same buffer when M = 4096)
    float2 *tc_twq = nullptr;
    int *d_status = nullptr;
    int *fwd_sync = nullptr;      // the one-launch forward stage's work queue (1 + chunks words)
    int64_t fwd_sync_n = 0;
    float2 *redig_mg = nullptr;   // redigitisation: (mean, levels / sigma) per (DM, channel)
    int32_t *inc_tab = nullptr;   // incoherent stage: shifts [ndm][nk][rows] of the last trial grid
    size_t inc_bytes = 0;
    double inc_key[2] = {NAN, NAN};   // (ddm_lo, ddm_step) of inc_tab
    int inc_nk = 0;
    int64_t inc_nt_out = 0;
    size_t inc_off = 0, inc_chg = 0;   // byte offsets of the change offsets and changes in inc_tab
    int64_t bytes = 0;
    // host-execute pipeline
    int64_t host_chunk = 0, span_max = 0, host_block_opt = 0;
    int64_t host_out_cap = 0;      // floats per output slot of the host pipeline (u8 slots: bytes)
    double sk_nsigma = 0.0;        // spectral-kurtosis flagging of the 8-bit host output (0: off)
    const float *scale_dev = nullptr;  // int8 input: DEVICE per-subband scales of the current call
    float *d_scale_buf = nullptr;      // int8 input from host memory: the scales on the device
    cdmt::Staging stage[3];        // host pipeline: three blocks in flight (copy in, compute, copy out)
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    // DM groups (cdmt_opts.dm_groups > 1): one child plan per contiguous group of DMs, each with
    // the overlap its own largest |DM| needs; this plan then holds no tables of its own
    struct Group {
        cdmt_plan_s *plan;   // DMs first .. first + plan->ndm - 1, input from sample `off` on
        int first;
        int64_t off;         // (nd - plan->nd) * nchan / 2 input samples
        int64_t kneed;       // segments that cover this plan's nout
    };
    std::vector<Group> groups;
    int64_t out_tlim = INT64_MAX;  // DM stage: output positions >= out_tlim are not stored
    // grouped plans from and to host memory: the whole input, filterbank and codes on the device
    uint8_t *grp_in = nullptr;
    float *grp_out = nullptr;
    uint8_t *grp_u8 = nullptr;
    // stage timing (cdmt_set_timing / cdmt_stage_times)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<cudaEvent_t> ev_marks;  // triples: before forward, before dedisperse, after dedisperse
    std::string last_error;
};


namespace cdmt {
// overlap n_d of Sec. 2 for a band (defined in cdmt_host.cu); -1 if none < M
int64_t overlap_for(int nsub, double f_centre, double bw, double dm_abs_max, int nchan, int nint, int64_t nbin);
// forward stage + DM stage of kc segments (defined in cdmt_host.cu)
int enqueue_chunk(cdmt_plan_s *p, const void *in, int64_t in_stride, int64_t in_k0, float *out,
                  int64_t out_stride, int64_t out_k0, int kc, cudaStream_t st);
// redigitisation of nt samples per row (rows `stride` floats apart) as one block (cdmt_redig.cu)
// Allocates the plan's per-row (mean, gain) array of the redigitisation if it is missing.
int redig_reserve(cdmt_plan_s *p);
int redig_enqueue(cdmt_plan_s *p, const float *d_fb, int64_t nt, int64_t stride, uint8_t *d_u8, float *d_stats,
                  cudaStream_t st, double sk_nsigma = 0.0, uint8_t *d_flags = nullptr, int ndm_r = 0);
// The forward stage, and the DM stage of a DM range of every tile (cdmt_host.cu).
int enqueue_forward(cdmt_plan_s *p, const void *in, int64_t in_stride, int64_t in_k0, int kc, cudaStream_t st);
int enqueue_dm(cdmt_plan_s *p, float *out, int64_t out_stride, int64_t out_k0, int kc, int dm_off, int dm_cnt,
               cudaStream_t st);
}  // namespace cdmt
