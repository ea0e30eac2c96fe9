/*
 * cdmt.h - C ABI of the GB300 coherent-dedispersion library.
 *
 * The library computes, on one GPU, the hot path of the convolving synthetic
 * filterbank with coherent dedispersion to many DM trials described by Bassa,
 * Pleunis & Hessels (2016, "cdmt"):
 *   Sec. 2 (Eq. 1, Eq. 2, Fig. 2): overlap-save segments of N_bin input samples,
 *     a forward FFT of N_bin, per-channel multiplication by the inverse of the
 *     ISM transfer function of Eq. 1, and n_c backward FFTs of M_bin = N_bin/n_c;
 *   Sec. 3 (Algorithm 1): swap halves, chirp multiply, backward FFT, transpose,
 *     unpad (n_d/2 samples per edge) and detect (Stokes I = |X|^2 + |Y|^2);
 * and it integrates nint consecutive samples into a DM x channel x time
 * filterbank.
 *
 * Conventions shared by every entry point:
 *  - Frequencies in MHz, DM in pc cm^-3, dispersion constant
 *    D = 4.148808e3 MHz^2 pc^-1 cm^3 s.  Subband s (0-based) is centred on
 *    f_centre + (s - (nsub-1)/2) * bw_sub: the band is contiguous and f_centre
 *    is the centre of the whole band.  Sample rate r = bw_sub * 1e6 complex
 *    samples per second (Nyquist-sampled complex subbands, Sec. 3).
 *  - Input layout: [nsub][nsamp] samples, each sample 16 bytes =
 *    float32 (X re, X im, Y re, Y im) (CDMT_IN_C64), or 4 bytes = int8
 *    (X re, X im, Y re, Y im) scaled by a per-subband float (CDMT_IN_I8).
 *  - Output layout: float32 [ndm][nsub * nchan][nout]; channel index
 *    s * nchan + c increases with frequency; output sample t covers input
 *    samples starting at (t * nint + nd/2) * nchan.
 *  - Transforms are unitary (1/sqrt(N) forward, 1/sqrt(M) backward), so complex
 *    white noise with E|x|^2 = sigma^2 per polarisation gives a mean output of
 *    2 sigma^2 nint.
 *  - Every function returns CDMT_OK (0) or a negative status; none aborts.
 *    The message of the last failure is kept per plan (cdmt_last_error) and,
 *    for failures before a plan exists, per thread (cdmt_last_error(NULL)).
 *  - A plan is bound to the CUDA device that was current when it was made and
 *    must be used from host threads one at a time.
 */
#ifndef CDMT_H
#define CDMT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cdmt_plan_s *cdmt_plan_t;

enum cdmt_status {
    CDMT_OK = 0,
    CDMT_EINVAL = -1,   /* an argument is out of range or inconsistent */
    CDMT_ENOMEM = -2,   /* a device or pinned-host allocation failed */
    CDMT_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
    CDMT_ETIMEOUT = -4, /* a bounded device wait expired */
    CDMT_EBUDGET = -5,  /* the plan would exceed the memory budget it was given */
    CDMT_ENOTSUP = -6   /* the combination of sizes has no kernel */
};

enum cdmt_precision {
    CDMT_PREC_FP32 = 0, /* every FFT stage on the FP32 pipes */
    CDMT_PREC_FP16 = 1, /* per-DM backward FFT as FP16 DFT-64 GEMMs on the tensor cores, FP32 accumulate */
    CDMT_PREC_BF16 = 2  /* the same with BF16 operands split into hi + lo parts (3 MMAs per step) */
};

enum cdmt_in_dtype {
    CDMT_IN_C64 = 0, /* 16 bytes per dual-pol sample */
    CDMT_IN_I8 = 1   /* 4 bytes per dual-pol sample plus a per-subband scale */
};

/* Optional plan overrides (cdmt_plan_ex).  Zero-initialise, then set fields;
 * a zero / negative field means "let the planner choose". */
/* Transfer functions (Sec. 2).  CDMT_CHIRP_CHANNEL: Eq. 1 evaluated about each
 * channel's centre, the paper's choice; it removes the dispersion within each
 * channel and leaves the inter-channel delays for a later incoherent stage, with
 * an overlap that holds one channel's sweep.  CDMT_CHIRP_SUBBAND: Eq. 1 about
 * the subband centre for every bin, the alternative the paper sets it against;
 * it removes the dispersion across the whole subband (its channels line up in
 * time) and needs an overlap that holds the whole subband's sweep (n_c^2 times
 * the channel's, roughly). */
enum cdmt_chirp { CDMT_CHIRP_CHANNEL = 0, CDMT_CHIRP_SUBBAND = 1 };

typedef struct cdmt_opts {
    int64_t nbin;        /* forward FFT length N_bin (power of two); 0 = choose */
    int64_t nd;          /* overlap n_d in channel samples; < 0 = rule of Sec. 2 */
    int32_t dm_tile;     /* DM trials per work item (forward spectrum reuse); 0 = choose */
    int32_t precision;   /* enum cdmt_precision */
    int32_t in_dtype;    /* enum cdmt_in_dtype */
    int32_t chirp;       /* enum cdmt_chirp: transfer function per channel (default) or per subband */
    int64_t seg_chunk;   /* segments per internal chunk (workspace size); 0 = choose */
    int64_t mem_budget;  /* bytes of device memory the plan may hold; 0 = no limit */
    int64_t host_block;  /* segments per block of the host pipeline (cdmt_execute_host*): the unit of its
                            copies and, for 8-bit output, the block the statistics cover (Sec. 3);
                            0 = choose (about 4 blocks for float32 output, 16 for 8-bit output, each
                            at least 16 work items per SM) */
    double sk_nsigma;    /* cdmt_execute_host_u8: spectral-kurtosis RFI flagging of each block's rows
                            (see cdmt_redigitise_sk); 0 = off */
    int32_t dm_groups;   /* > 1: split the DM list into this many contiguous groups of near-equal size
                            (group g: DMs g*ndm/G .. (g+1)*ndm/G - 1), each with the overlap its own
                            largest |DM| needs (the per-DM overlap of Sec. 5, taken per group), the
                            ungrouped time axis and length kept (see cdmt_plan_group); 0 or 1 = one
                            overlap for the whole list */
    int32_t group_nbin;  /* with dm_groups > 1: 1 = each group also picks its own N_bin (Sec. 5: digifil
                            chooses the FFT size per DM; see cdmt_plan_group_nbin); 0 = every group
                            uses the plan's N_bin */
    int64_t reserved[3];
} cdmt_opts;

/* Derived sizes of a plan (cdmt_plan_info). */
typedef struct cdmt_info {
    int64_t nsamp;        /* input samples per subband */
    int64_t nbin;         /* N_bin */
    int64_t mbin;         /* M_bin = N_bin / nchan */
    int64_t nd;           /* overlap n_d (channel samples) */
    int64_t nvalid;       /* S = N_bin - nd * nchan valid input samples per segment */
    int64_t nseg;         /* segments per subband = floor((nsamp - N_bin) / S) + 1 */
    int64_t nout;         /* output samples per channel = nseg * (M_bin - nd) / nint */
    int64_t seg_chunk;    /* segments per internal chunk */
    int64_t workspace_bytes; /* device memory the plan holds */
    int64_t in_bytes;     /* bytes of one input block: 16 per sample, 4 for CDMT_IN_I8 */
    int64_t out_bytes;    /* bytes of one output filterbank */
    double units;         /* DM-trial x input samples consumed per execute = ndm * nsub * nseg * S */
    int32_t nsub, nchan, nint, ndm;
    int32_t dm_tile;      /* DM trials per work item */
    int32_t uniform_dm;   /* 1 if the DM list is evenly spaced (integer phase accumulator) */
    int32_t precision, in_dtype;
    int32_t device;
    int32_t dm_groups;    /* DM groups with their own overlap (1: none); nd, nvalid and nseg above are
                             then those of the group with the largest overlap, nd of the whole list */
    int32_t reserved[6];
} cdmt_info;

/*
 * cdmt_plan - validate a problem and prepare everything an execute needs.
 *
 * Follows the initialisation of Sec. 3 / Algorithm 1 ("compute transfer
 * function for DM[idm]"): N_bin and n_d are fixed for all subbands and channels
 * (Sec. 3), n_d follows Sec. 2 (n_d = r t_d / n_c, t_d of Eq. 2 for the lowest
 * channel at the largest |DM|; rounded up to an even number with (M - n_d)
 * divisible by nint), and the per-channel chirp phases of Eq. 1 are computed on
 * the GPU in FP64 and stored as 32-bit fixed-point phase and phase step per
 * frequency bin and DM tile.
 *
 *   plan          out: the new plan (NULL on failure)
 *   nsub          number of subbands, >= 1
 *   nsamp         input samples per subband, >= N_bin
 *   f_centre_mhz  centre of the whole band (MHz); the lowest channel must be > 0
 *   bw_sub_mhz    subband width = complex sample rate / 1e6, > 0
 *   dm_list       host array of ndm trial DMs (copied; any order; any sign)
 *   ndm           >= 1
 *   nchan         channels per subband n_c, a power of two 2..32
 *   nint          output integration factor, >= 1
 * Errors: CDMT_EINVAL (bad argument, N_bin <= n_d n_c, nsamp < N_bin;
 *         cdmt_opts.dm_groups outside 0..ndm), CDMT_ENOTSUP (M_bin outside
 *         512..8192 in the FP32 form, e.g. Sec. 4's N_bin = 65536 with n_c = 8;
 *         tensor-core precisions need M_bin = 2048 or 4096 and nint dividing 32),
 *         CDMT_ENOMEM, CDMT_EBUDGET (cdmt_opts.mem_budget), CDMT_ECUDA.  Without
 *         cdmt_opts.nbin the plan picks M_bin in 512..4096.
 * Allocates device memory (tables and workspace); the plan owns all of it.
 */
int cdmt_plan(cdmt_plan_t *plan, int nsub, int64_t nsamp, double f_centre_mhz,
              double bw_sub_mhz, const double *dm_list, int ndm, int nchan, int nint);

/* cdmt_plan with overrides (opts may be NULL = cdmt_plan).  Parity tests use
 * opts->nbin and opts->nd to fix the segment grid, since the filterbank of the
 * brick-wall channeliser depends on N_bin. */
int cdmt_plan_ex(cdmt_plan_t *plan, int nsub, int64_t nsamp, double f_centre_mhz,
                 double bw_sub_mhz, const double *dm_list, int ndm, int nchan, int nint,
                 const cdmt_opts *opts);

/* cdmt_plan_info - copy the derived sizes of a plan into *info (host memory).
 * Errors: CDMT_EINVAL if plan or info is NULL. */
int cdmt_plan_info(cdmt_plan_t plan, cdmt_info *info);

/* cdmt_plan_group - the layout of DM group g of a plan made with
 * cdmt_opts.dm_groups > 1 (g < cdmt_info.dm_groups; a plan without groups has
 * one group, g = 0, of all DMs with the plan's overlap and no offset).
 *
 * Sec. 2 sizes the overlap n_d for the largest |DM| of the list; digifil
 * (Sec. 5) sizes it per DM.  A grouped plan gives group g the smallest overlap
 * nd_g that (a) holds the sweep of its own largest |DM| by the rule of Sec. 2
 * (even, (M - nd_g) divisible by nint), and (b) whose segments cover the whole
 * ungrouped output length; nd_g <= n_d of the whole list, which satisfies both.
 * The filterbank keeps the ungrouped time axis: group g's overlap-save segments
 * start off_g = (n_d - nd_g) * nchan / 2 input samples into each subband, so
 * that its first kept sample is the ungrouped first kept sample.  The rows of
 * group g are its own overlap-save filterbank; they differ from the ungrouped
 * rows by the wrap-around of the shorter segments (about 1 % rms, largest at
 * small overlaps), and the DM stage runs on nseg_g = (nsamp - off_g - N_bin) /
 * (N_bin - nd_g * nchan) + 1 segments of S_g = N_bin - nd_g * nchan instead.
 *
 *   dm_first, ndm  out (may be NULL): the group's first DM index and DM count
 *   nd, offset     out (may be NULL): nd_g (channel samples) and off_g (input samples)
 *   nseg           out (may be NULL): segments the group's DM stage runs on per execute
 * Errors: CDMT_EINVAL for a NULL plan or g out of range. */
int cdmt_plan_group(cdmt_plan_t plan, int g, int *dm_first, int *ndm, int64_t *nd, int64_t *offset,
                    int64_t *nseg);

/* cdmt_plan_group_nbin - the forward FFT length N_g of DM group g (the plan's
 * N_bin unless the plan was made with cdmt_opts.group_nbin = 1).
 *
 * Sec. 5 notes that digifil chooses the FFT size as well as the overlap for the
 * DM and frequency at hand, which pays at low DMs.  With group_nbin = 1 group g
 * takes, among the channel lengths M = N / nchan its precision runs (512..8192
 * in the FP32 form, 2048 and 4096 in the tensor-core forms) for which an
 * overlap nd_g <= n_d exists as in cdmt_plan_group (the group's own rule at
 * that M, grown until its segments cover the ungrouped output length) and one
 * segment fits the input from off_g on, the M with the least nominal FFT work
 * per DM-trial x input sample, 10 N log2(M) / S_g = 10 nchan M log2(M) /
 * (nchan (M - nd_g)), the plan's own M on a tie.  The time axis and off_g do not
 * depend on N_g (channel samples keep their rate), so the filterbank layout is
 * that of cdmt_plan_group.  The rule counts flops only: a length whose kernel
 * runs at a lower rate can make the plan slower (measured on GB300: FP32 groups
 * that take M = 8192, or FP16 groups that take M = 2048, lose more to the
 * kernels' rate than they save in work).
 *   nbin  out: N_g
 * Errors: CDMT_EINVAL for a NULL plan or nbin, or g out of range. */
int cdmt_plan_group_nbin(cdmt_plan_t plan, int g, int64_t *nbin);

/*
 * cdmt_execute - compute the whole filterbank of one input block.
 *
 * Algorithm 1's block loop without disk I/O: forward FFT of every segment of
 * every subband (Sec. 3 "unpack, segment and pad", "forward FFT", "swap halves
 * per subband"), then for each DM trial the chirp multiply, backward FFTs,
 * unpad, detection (Sec. 3) and nint-sample integration.
 *
 *   d_in         DEVICE pointer to the input block (layout above), caller-owned,
 *                16-byte aligned (CDMT_IN_I8: 4-byte aligned); read only
 *   d_out        DEVICE pointer to float32 [ndm][nsub*nchan][nout], caller-owned,
 *                4-byte aligned; fully overwritten
 *   d_scale      DEVICE pointer to nsub float scales for CDMT_IN_I8 input: sample
 *                value = int8 value x scale[subband], in FP32 (required; ignored,
 *                may be NULL, for CDMT_IN_C64)
 *   cuda_stream  cudaStream_t to enqueue on (NULL = legacy default stream)
 * Asynchronous with respect to the host: returns after enqueueing.  The plan's
 * workspace is reused by every execute, so executes of ONE plan must not
 * overlap on different streams.
 * Errors: CDMT_EINVAL (NULL pointers, misaligned input, int8 input without
 * scales), CDMT_ECUDA.
 */
int cdmt_execute(cdmt_plan_t plan, const void *d_in, float *d_out, const float *d_scale,
                 void *cuda_stream);

/*
 * cdmt_execute_host - the same computation from and to HOST memory.
 *
 * Copies the input block host->device, computes, and copies the filterbank
 * device->host, pipelining the copies of segment chunks with the compute of
 * others (Algorithm 1: "copy to device" ... "copy to host").  h_in and h_out
 * should be page-locked (cudaHostAlloc / cudaHostRegister) for full speed;
 * pageable memory works but the copies are then synchronous.  Blocks until
 * h_out holds the result.  h_scale is a host array of nsub floats for
 * CDMT_IN_I8 input (required then; the input is then 4 bytes per sample, so
 * its copy to the device is 4x smaller).  A plan with DM groups
 * (cdmt_opts.dm_groups) copies the whole input in, runs cdmt_execute and copies
 * the whole filterbank out, without overlapping copies and compute (its groups
 * segment the input differently), on device buffers it keeps until
 * cdmt_destroy: about the input plus five times the filterbank's bytes (the
 * float32 filterbank, and its 8-bit codes once cdmt_execute_host_u8 has run),
 * which cdmt_info.workspace_bytes does not include.
 * On an error the call waits for the copies it had queued before it returns,
 * so that the caller may free or reuse h_in and h_out at once.
 * Errors: CDMT_EINVAL, CDMT_ENOMEM (staging buffers), CDMT_EBUDGET (a staging
 * or DM-group buffer would exceed cdmt_opts.mem_budget), CDMT_ECUDA.
 */
/* cdmt_execute_host_u8 - the pipeline of Algorithm 1 up to "redigitize" and
 * "copy to host": like cdmt_execute_host, but each block of segments
 * (cdmt_opts.host_block, or the plan's choice) is a data block whose filterbank
 * is redigitised on the device (cdmt_redigitise: the mean and sigma of each
 * (DM, channel) over the block; with cdmt_opts.sk_nsigma > 0 also the
 * spectral-kurtosis flagging of cdmt_redigitise_sk, flagged rows coded 128)
 * and copied back as 8-bit codes, 4x fewer bytes than float32.  h_u8: host
 * (pinned for overlap) uint8 [ndm][nout][nsub*nchan], spectra in decreasing
 * frequency.  *block_segments (may be NULL) receives the segments per block
 * (the last block may be shorter).  A plan with DM groups redigitises its whole
 * filterbank as one block (*block_segments = nseg of cdmt_plan_info).  Errors as cdmt_execute_host (a
 * CDMT_IN_I8 plan needs cdmt_execute_host_u8_ex, which takes the scales). */
int cdmt_execute_host_u8(cdmt_plan_t plan, const void *h_in, uint8_t *h_u8, int64_t *block_segments,
                         void *cuda_stream);

/* cdmt_execute_host_u8_ex - cdmt_execute_host_u8 with h_scale, a host array of
 * nsub floats for CDMT_IN_I8 input (ignored, may be NULL, for CDMT_IN_C64):
 * the paper's own I/O, 8-bit voltages in and an 8-bit filterbank out.  Errors
 * as cdmt_execute_host. */
int cdmt_execute_host_u8_ex(cdmt_plan_t plan, const void *h_in, const float *h_scale, uint8_t *h_u8,
                            int64_t *block_segments, void *cuda_stream);

int cdmt_execute_host(cdmt_plan_t plan, const void *h_in, float *h_out, const float *h_scale,
                      void *cuda_stream);

/* cdmt_device_status - wait for the plan's device work and report whether
 * any tensor-core wait in it gave up (CDMT_ETIMEOUT; its outputs are then
 * incomplete).  The flag is cleared.  Returns CDMT_OK otherwise, CDMT_ECUDA on
 * a CUDA error, CDMT_EINVAL for a NULL plan. */
int cdmt_device_status(cdmt_plan_t plan);

/* cdmt_selftest_wait - run the bounded wait of the tensor-core kernels (the
 * wait between a GEMM's commit to an mbarrier and its read-out: a limit on the
 * GPU's global timer plus a cap on polls) on a barrier that nothing arrives on,
 * in a one-warp kernel of its own.  It must give up after limit_ms and leave the
 * context usable; with arrive != 0 one arrival completes the barrier's phase
 * first, and the wait must succeed at once.  No fault, trap or hang is involved.
 *   limit_ms   the wait's time limit, in (0, 1000]
 *   gave_up    out: 1 if the wait gave up, 0 if the phase completed
 *   waited_ms  out: the wait's duration on the global timer
 * Errors: CDMT_EINVAL (NULL outputs, limit out of range), CDMT_ENOMEM, CDMT_ECUDA. */
int cdmt_selftest_wait(double limit_ms, int arrive, int *gave_up, double *waited_ms);

/* cdmt_inject_timeout - mark the plan's device status word (every group's, for a
 * plan with DM groups) as a tensor-core kernel does when one of its waits gives
 * up: host-side injection for tests of the recovery path.  Until
 * cdmt_device_status reports CDMT_ETIMEOUT and clears the word, every launch of
 * the tensor-core DM stage of this plan returns at once, before it allocates
 * tensor memory, and leaves its outputs unwritten; the FP32 form does not read
 * the word.  Errors: CDMT_EINVAL for a NULL plan, CDMT_ECUDA. */
int cdmt_inject_timeout(cdmt_plan_t plan);

/* cdmt_set_timing - when on != 0, later executes record CUDA events on their
 * stream around the forward stage (Sec. 3 "forward FFT" and "swap halves per
 * subband": two kernels per chunk) and around the dedispersion kernel (chirp
 * multiply through integration: one kernel per chunk), for cdmt_stage_times.
 * Off by default; recording costs one event per stage boundary.
 * Errors: CDMT_EINVAL for a NULL plan. */
int cdmt_set_timing(cdmt_plan_t plan, int on);

/* cdmt_stage_times - wait for the events recorded since the previous call and
 * return the summed device time in milliseconds of the forward stage (ms[0])
 * and of the dedispersion kernel (ms[1]), and the number of kernel launches of
 * each (launches[0], launches[1]).  ms and launches are host arrays of two
 * elements (launches may be NULL).  Clears the record.
 * Errors: CDMT_EINVAL (NULL plan or ms), CDMT_ECUDA. */
int cdmt_stage_times(cdmt_plan_t plan, double *ms, int64_t *launches);

/* ------------------------------------------------------------------------
 * Redigitisation to 8 bits (Sec. 3: "compute block sums", "compute channel
 * statistics", "redigitize" of Algorithm 1).  The paper computes data offsets
 * and scales from the mean and standard deviation of each channel's time
 * series in the block and converts the floating-point filterbank to 8-bit
 * integers packed as spectra in decreasing frequency order.
 *
 * For every DM trial d and channel row r (r = s*nchan + c, increasing
 * frequency) of a plan's float32 filterbank fb[ndm][nsub*nchan][nout]:
 *   mu, sigma = mean and (population) standard deviation of the row's nout
 *               samples (sums of I and I^2; FP32 within a thread, FP64 across);
 *   code      = clamp(rint(fmaf(I - mu, g, 128)), 0, 255),  g = CDMT_REDIG_LEVELS / sigma
 *               (g = 0 for a constant row), in FP32: mu and sigma rounded to FP32
 *               (the values d_stats reports) and g divided in FP32, so that the
 *               codes of a row follow from its reported (mu, sigma) alone.
 * The mapping is this library's choice (the paper leaves it open): 128 is the
 * mean and 16 code steps span one sigma, so -8 .. +7.9 sigma are kept.
 *
 * cdmt_redigitise - d_fb: device, the plan's filterbank (as cdmt_execute
 * writes it); d_u8: device, uint8 [ndm][nout][nsub*nchan] with row r at
 * position nsub*nchan - 1 - r; d_stats: device float [ndm][nsub*nchan][2]
 * (mu, sigma), or NULL.  Asynchronous on cuda_stream; the plan keeps an
 * (mu, g) array of ndm*nsub*nchan float2.  Errors: CDMT_EINVAL (NULL
 * pointers), CDMT_ENOMEM, CDMT_ENOTSUP (more than 65535 DM trials or 64-row
 * tiles), CDMT_ECUDA. */
#define CDMT_REDIG_LEVELS 16.0
int cdmt_redigitise(cdmt_plan_t plan, const float *d_fb, uint8_t *d_u8, float *d_stats, void *cuda_stream);

/* cdmt_redigitise_sk - cdmt_redigitise with spectral-kurtosis RFI flagging
 * (Sec. 6 names spectral kurtosis for the statistics step as future work and
 * gives no definition; this is the generalised SK estimator).  For every
 * (DM, channel) row of n = nout samples, each a sum of k = 2 nint squared
 * magnitudes (two polarisations, nint time samples),
 *   SK = (n k + 1) / (n - 1) * (n S2 / S1^2 - 1),  S1 = sum I, S2 = sum I^2,
 * which averages 1 for Gaussian voltages with a large-n standard deviation of
 * sqrt(2 (k + 1) / (k n)).  A row with |SK - 1| > sk_nsigma times that
 * deviation is flagged: all its codes are 128 (its mean) and d_flags[dm][row]
 * is 1 (0 otherwise).  Rows without power have SK = 0; rows of fewer than two
 * samples are never flagged.  sk_nsigma = 0 disables flagging (then this is
 * cdmt_redigitise).  d_flags: DEVICE uint8 [ndm][nsub*nchan], may be NULL.
 * Errors: as cdmt_redigitise; CDMT_EINVAL for a negative or NaN sk_nsigma. */
int cdmt_redigitise_sk(cdmt_plan_t plan, const float *d_fb, uint8_t *d_u8, float *d_stats, double sk_nsigma,
                       uint8_t *d_flags, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Incoherent dedispersion of the coherent filterbanks (Sec. 4: in the
 * semi-coherent search every coherently dedispersed filterbank is then
 * incoherently dedispersed at fine DM steps around its coherent DM; Sec. 1:
 * incoherent dedispersion shifts each channel's time series by its delay).
 *
 * The channels of a coherent filterbank still carry the delays between their
 * reference frequencies nu_r (channel centres; subband centres for
 * CDMT_CHIRP_SUBBAND), so for coherent DM trial c (DM_c, the plan's list), fine
 * trial k (total DM = DM_c + ddm_lo + k ddm_step) and row r the shift in output
 * samples of t_samp = nint * nchan / (bw_sub * 1e6) seconds is
 *     d(c, k, r) = rint(D (DM_c + ddm_lo + k ddm_step) (nu_r^-2 - nu_top^-2) / t_samp)
 * (FP64 on the host; nu_top the highest reference frequency), and with d_lo,
 * d_hi the extreme shifts over all (c, k, r):
 *     out[c][k][t] = sum_r fb[c][r][t + d(c, k, r) - d_lo],   t < nt_out = nout - (d_hi - d_lo)
 * summed in FP32.  Output sample t is at the top frequency's time t + d_lo.
 *
 * cdmt_incoherent_info - nt_out for the fine-trial grid, and (h_delays, host,
 * may be NULL) the shifts d - d_lo as int32 [ndm][nk][nsub*nchan].
 * cdmt_incoherent - d_fb: device, the plan's filterbank [ndm][nsub*nchan][nout]
 * (as cdmt_execute writes it); d_out: device float32 [ndm][nk][nt_out].
 * Asynchronous on cuda_stream, except that a new trial grid uploads the plan's
 * shift table synchronously.  Errors: CDMT_EINVAL (NULL pointers, nk < 1, no
 * output sample left), CDMT_ENOMEM, CDMT_ENOTSUP (more than 65535 coherent DMs
 * or 1024-sample blocks), CDMT_ECUDA. */
int cdmt_incoherent_info(cdmt_plan_t plan, double ddm_lo, double ddm_step, int nk, int64_t *nt_out, int32_t *h_delays);
int cdmt_incoherent(cdmt_plan_t plan, const float *d_fb, double ddm_lo, double ddm_step, int nk, float *d_out,
                    void *cuda_stream);

/* Bytes of the device array that backs cdmt_execute_static (64 MiB). */
#define CDMT_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)

/*
 * cdmt_execute_static - cdmt_plan + cdmt_execute in one call that allocates no
 * memory at all.  The paper has no counterpart: it serves callers that must not
 * call cudaMalloc / cudaFree, for example because their device memory belongs
 * to another framework's pool, or because a real-time loop cannot pay the
 * device-wide synchronisation those calls imply.
 *
 * Computes the FP32-form filterbank of one input block (same kernels and
 * results as a plan with precision CDMT_PREC_FP32, nbin and nd given) for the
 * evenly spaced DM list dm_first + i * dm_step, i < ndm.  nd < 0 applies the
 * overlap rule of Sec. 2.  d_in / d_out are the caller's DEVICE buffers in the
 * layouts above (d_out: float32 [ndm][nsub*nchan][nout] with nout =
 * nseg * (M - nd) / nint); enqueued on cuda_stream, asynchronous.
 *
 * All other memory it uses (twiddles, chirp-phase words, the forward spectrum
 * of a chunk of segments) is one file-scope __device__ array of
 * CDMT_STATIC_SCRATCH_BYTES, which every GPU that loads this part of the
 * library keeps until the process exits.  Limit: about 24 * nsub * nbin bytes
 * must fit in it (e.g. nsub <= 42 at nbin = 65536); larger problems return
 * CDMT_EBUDGET with the sizes in cdmt_last_error(NULL), and need cdmt_plan.
 * The first call on a device looks up the array's device address (and sets the
 * kernels' shared-memory attributes) with that device current; make that first
 * call before any stream capture.  Every call writes every scratch byte it
 * later reads, so nothing carries over from a previous call, but all calls on a
 * device share the one array: calls whose work overlaps on the GPU (different
 * streams, or host threads racing) corrupt each other's results.
 * Errors: CDMT_EINVAL, CDMT_ENOTSUP (M_bin outside 512..8192), CDMT_EBUDGET,
 * CDMT_ECUDA; messages via cdmt_last_error(NULL).
 */
int cdmt_execute_static(int nsub, int64_t nsamp, double f_centre_mhz, double bw_sub_mhz, double dm_first,
                        double dm_step, int ndm, int nchan, int nint, int64_t nbin, int64_t nd, const void *d_in,
                        float *d_out, void *cuda_stream);

/* cdmt_destroy - free every resource of a plan (NULL is accepted).  Waits for
 * the plan's device work to finish first. */
int cdmt_destroy(cdmt_plan_t plan);

/* cdmt_strerror - static text for a status code. */
const char *cdmt_strerror(int status);

/* cdmt_last_error - message of the last failure on this plan, or, for
 * plan == NULL, of the last failure on this host thread before a plan existed.
 * The pointer stays valid until the next call on the same plan / thread. */
const char *cdmt_last_error(cdmt_plan_t plan);

/* ------------------------------------------------------------------------
 * Batches of beams of uneven shapes.
 *
 * A batch runs several beams, each with its own subbands, samples, channel
 * count, integration and evenly spaced DM list, through ONE CUDA graph per
 * "round".  A round is a chunk of consecutive overlap-save segments of every
 * beam (the block loop of Algorithm 1, Sec. 3, with N_FFT chosen so that the
 * round outputs of all beams fit the output budget).  Each graph launch runs
 * the forward stage of every beam and then one persistent tensor-core launch
 * that takes (beam, subband, segment, channel, DM tile) items from a device
 * queue; beams the autotuner assigns to the FP32 form get their own DM-stage
 * kernel in the same graph.  The round number lives in device memory and the
 * graph advances it, so one graph serves every round.
 */
typedef struct cdmt_batch_s *cdmt_batch_t;

typedef struct cdmt_beam {
    int32_t nsub;          /* subbands */
    int32_t ndm;           /* DM trials: dm_first + i * dm_step, i < ndm */
    int64_t nsamp;         /* samples per subband */
    double f_centre_mhz;   /* centre of the beam's band */
    double bw_sub_mhz;     /* subband width */
    double dm_first, dm_step;
    int32_t nchan, nint;
    const void *d_in;      /* DEVICE input [nsub][nsamp] 16-byte samples, caller-owned, valid for the
                              batch's lifetime (its address is captured in the graph) */
} cdmt_beam;

typedef struct cdmt_batch_opts {
    int64_t out_budget;    /* bytes for the round outputs of all beams (0: 16 GiB) */
    int32_t autotune;      /* 0: FP16 tensor-core form with one DM tile; 1: time candidates */
    int32_t reserved0;
    const char *tune_cache;/* text file of tuned choices (read, and appended to), or NULL */
    int64_t reserved[6];
} cdmt_batch_opts;

/* per-beam choice of the autotuner */
typedef struct cdmt_batch_tune {
    int32_t precision;     /* enum cdmt_precision */
    int32_t dm_tile;
    int64_t nbin;
    double units_per_s;    /* measured DM-trial samples/s on the sample (0 if not measured) */
    int32_t from_cache;
    int32_t reserved;
} cdmt_batch_tune;

typedef struct cdmt_batch_beam_info {
    cdmt_info plan;        /* the beam's plan (nbin, nd, nseg, nout, ...) */
    cdmt_batch_tune tune;
    int32_t nround;        /* rounds to cover every beam's input */
    int32_t reserved0;
    int64_t seg_per_round; /* segments of this beam per round; round r covers segments
                              [r * seg_per_round, ...) (fewer or none near the end) */
    float *d_out;          /* DEVICE round output, owned by the batch: float32
                              [ndm][nsub*nchan][out_row_stride]; segment kk of the round at
                              columns [kk * seglen, (kk + 1) * seglen), seglen = (M - nd) / nint;
                              overwritten by every round */
    int64_t out_row_stride;
    int64_t out_bytes_total; /* round output bytes of all beams */
} cdmt_batch_beam_info;

/* cdmt_batch_create - tune, plan and capture a batch.  beams: host array of
 * nbeam descriptors (copied).  stream: used for autotuning runs.  Allocates
 * device memory (plans, round outputs).
 * Errors: CDMT_EINVAL, CDMT_EBUDGET (one segment of every beam does not fit the
 * output budget), CDMT_ENOMEM, CDMT_ECUDA, and the plan errors of a beam. */
int cdmt_batch_create(cdmt_batch_t *batch, int nbeam, const cdmt_beam *beams, const cdmt_batch_opts *opts,
                      void *stream);

/* cdmt_batch_info - sizes, tuned choices and the round output buffer of one beam. */
int cdmt_batch_info(cdmt_batch_t batch, int beam, cdmt_batch_beam_info *info);

/* cdmt_batch_run_round - enqueue round r (0 <= r < nround) on stream: one graph
 * launch.  The round outputs are valid once the stream reaches that point and
 * until the next round is enqueued. */
int cdmt_batch_run_round(cdmt_batch_t batch, int round, void *stream);

/* cdmt_batch_run - enqueue every round in order (each overwrites the round
 * outputs): throughput runs, or a consumer that drains by stream order. */
int cdmt_batch_run(cdmt_batch_t batch, void *stream);

/* cdmt_batch_copy_out - copy beam's whole round output buffer
 * (ndm * nsub*nchan * out_row_stride floats) to dst (host or device memory,
 * cudaMemcpyDefault), ordered on stream after the rounds enqueued there. */
int cdmt_batch_copy_out(cdmt_batch_t batch, int beam, void *dst, void *stream);

/* cdmt_batch_status - wait for the batch's device work; CDMT_ETIMEOUT if a
 * tensor-core wait gave up (flag cleared), else CDMT_OK. */
int cdmt_batch_status(cdmt_batch_t batch);

/* cdmt_batch_last_error - message of the last failure on the batch (NULL:
 * this thread's last failure before a batch existed). */
const char *cdmt_batch_last_error(cdmt_batch_t batch);

/* cdmt_batch_destroy - free the batch (waits for the device first). */
int cdmt_batch_destroy(cdmt_batch_t batch);

/* ------------------------------------------------------------------------
 * Streaming server: real-time blocks of several beams, continuously batched.
 *
 * Each beam added to a server keeps its plan, its overlap tail (the input
 * samples that do not yet complete an overlap-save segment, Sec. 2) in two
 * staging buffers, and for int8 blocks two block buffers, resident on the device
 * (a block's copy to the device, on its own stream, overlaps the compute of the
 * block before; complex64 blocks from host memory are copied straight behind
 * the tail).  Submitted blocks are
 * queued; a
 * scheduler thread dispatches them in arrival order across beams whenever an
 * output slot is free (blocks of one beam stay in order on that beam's CUDA
 * stream; blocks of different beams overlap on the GPU).  The slot pool is sized
 * from the HBM budget left after the resident beam state, so new blocks are
 * admitted as slots and memory free up.  A block's filterbank holds every
 * segment the block completes (Algorithm 1's block loop run per beam).  A beam
 * with out_dtype CDMT_OUT_U8 runs Algorithm 1 through "redigitize" for every
 * block: the float32 filterbank goes to a scratch slot of the pool, which is
 * free again once the block completes, and the 8-bit codes and the row
 * statistics occupy the output slot.
 */
typedef struct cdmt_server_s *cdmt_server_t;

typedef struct cdmt_server_opts {
    int64_t hbm_budget;    /* bytes the server may hold (0: 120 GiB) */
    int32_t max_slots;     /* upper bound on output slots (0: 64) */
    int32_t reserved0;
    int64_t reserved[6];
} cdmt_server_opts;

typedef struct cdmt_stream_desc {
    int32_t nsub, ndm;
    int64_t block_len;     /* samples per subband per block */
    double f_centre_mhz, bw_sub_mhz;
    double dm_first, dm_step;
    int32_t nchan, nint;
    int32_t precision;     /* enum cdmt_precision */
    int32_t in_dtype;      /* CDMT_IN_C64: 16-byte samples; CDMT_IN_I8: 4 int8 per sample + nsub float scales */
    int64_t nbin;          /* 0: 4096 * nchan */
    int32_t dm_tile;       /* DM trials per work item (0: the plan's choice) */
    int32_t out_dtype;     /* enum cdmt_out_dtype: the block's filterbank as float32, or redigitised to
                              8 bits per block (Sec. 3, as cdmt_redigitise) */
    double sk_nsigma;      /* CDMT_OUT_U8: spectral-kurtosis flagging of each block's rows, as
                              cdmt_redigitise_sk (0 = off) */
    int64_t reserved[3];
} cdmt_stream_desc;

/* Output type of a served block. */
enum cdmt_out_dtype {
    CDMT_OUT_F32 = 0, /* float32 [ndm][nsub*nchan][row_stride] in d_out */
    CDMT_OUT_U8 = 1   /* 8-bit codes [ndm][samples][nsub*nchan] (spectra in decreasing frequency) in d_u8,
                         per-row (mean, sigma) of the block's samples in d_stats */
};

typedef struct cdmt_block_result {
    int32_t beam;
    int32_t reserved0;
    int64_t index;         /* block number within the beam (submission order) */
    float *d_out;          /* CDMT_OUT_F32 beams: DEVICE slot, float32 [ndm][nsub*nchan][row_stride], this
                              block's samples in columns [0, samples); valid until cdmt_server_release.
                              NULL for 8-bit beams */
    int64_t nseg;          /* overlap-save segments this block completed (0 while the stream fills) */
    int64_t first_sample;  /* output-sample index (per channel, since the stream start) of column 0 */
    int64_t samples;       /* output samples per row in this block = nseg * (M - nd) / nint */
    int64_t row_stride;    /* floats between rows of d_out: max segments per block x (M - nd) / nint, rounded
                              up to a multiple of 4 */
    double latency_ms;     /* submit -> completion */
    uint8_t *d_u8;         /* CDMT_OUT_U8 beams: DEVICE slot, [ndm][samples][nsub*nchan] codes (row r of the
                              filterbank at position nsub*nchan-1-r); NULL for float32 beams */
    float *d_stats;        /* CDMT_OUT_U8 beams: DEVICE, [ndm][nsub*nchan][2] (mean, sigma) of each row over
                              this block's samples; both valid until cdmt_server_release, and only when
                              samples > 0 */
    uint8_t *d_flags;      /* CDMT_OUT_U8 beams: DEVICE, [ndm][nsub*nchan] spectral-kurtosis flags of this
                              block's rows (all 0 when sk_nsigma is 0); NULL for float32 beams */
} cdmt_block_result;

typedef struct cdmt_server_stats {
    int64_t blocks_done, blocks_queued, blocks_running;
    double latency_p50_ms, latency_p99_ms, latency_max_ms;
    double wall_s;          /* first submit to last completion */
    double data_s;          /* seconds of voltage data completed, summed over beams */
    double realtime_factor; /* data_s / wall_s */
    double units_per_s;     /* DM-trial x samples per second */
    int64_t hbm_bytes;      /* resident beam state + output slots */
    int32_t slots;
    int32_t reserved0;
} cdmt_server_stats;

/* create / destroy a server (destroy waits for its GPU work; output slots and
 * beam state are freed) */
int cdmt_server_create(cdmt_server_t *server, const cdmt_server_opts *opts);
int cdmt_server_destroy(cdmt_server_t server);

/* cdmt_server_add_beam - admit a beam: plans it and allocates its resident
 * state; CDMT_EBUDGET if that state plus one output slot does not fit the HBM
 * budget.  *beam_id receives the beam's index. */
int cdmt_server_add_beam(cdmt_server_t server, const cdmt_stream_desc *desc, int *beam_id);

/* cdmt_server_submit - queue the next block of a beam.  block: [nsub][block_len]
 * samples in host (pinned for asynchronous copies) or device memory; scale:
 * nsub floats (host or device) for int8 blocks.  Both must stay valid until the
 * block completes.  Returns at once with *request_id. */
int cdmt_server_submit(cdmt_server_t server, int beam, const void *block, const float *scale, int64_t *request_id);

/* cdmt_server_wait - wait up to timeout_s for a block (CDMT_ETIMEOUT after) and
 * describe its output in *result (may be NULL). */
int cdmt_server_wait(cdmt_server_t server, int64_t request_id, double timeout_s, cdmt_block_result *result);

/* cdmt_server_release - give a completed block's output slot back. */
int cdmt_server_release(cdmt_server_t server, int64_t request_id);

/* cdmt_server_save_beam - checkpoint of a beam's stream: the overlap tail that
 * its next block is appended to (the last N_bin - S samples it has not yet
 * completed into segments, Sec. 2), its segment and block counters, and the
 * shape the beam was made with.  A stream restored from it into a beam of the
 * same shape continues exactly: the next block's filterbank equals the one the
 * original beam would have produced, at the same output position.
 *   host   out: the checkpoint (host memory), or NULL to query its size
 *   bytes  in: the size of host; out: the checkpoint's size
 * Every block submitted to the beam must be done (waited for or not).
 * Errors: CDMT_EINVAL (NULL server or bytes, no such beam, blocks queued or
 * running, host smaller than the checkpoint), CDMT_ECUDA. */
int cdmt_server_save_beam(cdmt_server_t srv, int beam, void *host, int64_t *bytes);

/* cdmt_server_restore_beam - continue a stream from a checkpoint of
 * cdmt_server_save_beam (host memory, `bytes` long) in a beam with the same
 * subbands, block length, band, DM grid, channels, nint, N_bin and overlap (the
 * precision, input and output types may differ).  The beam must have no block
 * queued or running; its tail and counters are replaced.
 * Errors: CDMT_EINVAL (NULL pointers, no such beam, blocks queued or running,
 * not a checkpoint, another shape, truncated), CDMT_ECUDA. */
int cdmt_server_restore_beam(cdmt_server_t srv, int beam, const void *host, int64_t bytes);

/* cdmt_server_get_stats - latency percentiles, real-time factor and throughput of
 * the blocks completed since the start (or the last reset). */
int cdmt_server_get_stats(cdmt_server_t server, cdmt_server_stats *stats);
int cdmt_server_reset_stats(cdmt_server_t server);

/* cdmt_server_last_error - message of the last failure on the server. */
const char *cdmt_server_last_error(cdmt_server_t server);

#ifdef __cplusplus
}
#endif

#endif /* CDMT_H */
