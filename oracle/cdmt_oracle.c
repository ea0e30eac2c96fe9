/*
 * FP64 CPU oracle for coherent dedispersion with a convolving synthetic
 * filterbank (Bassa, Pleunis & Hessels 2016, "cdmt").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is read, built and run by the test
 * suite, by the smoke check and by the CPU-baseline leg of the benchmark.
 * The GPU library never links, includes or calls it, and it shares no code
 * (kernels, headers, tables, constants generators) with the GPU library.
 *
 * What it computes, per subband s, overlap-save segment k, DM trial and
 * polarisation (paper Sec. 2, Eq. 1, Eq. 2, Fig. 2; Sec. 3, Algorithm 1):
 *   1. x_n = in[s][k*S + n][pol], n < N  (S = N - nd*nchan valid samples)
 *   2. X = unitary forward DFT_N(x) (e^{-2 pi i}/sqrt(N)), halves swapped so
 *      bins run in increasing frequency (Sec. 3, "swap halves per subband").
 *   3. channel c takes bins [c*M, (c+1)*M), M = N/nchan, and multiplies them
 *      by the conjugate of Eq. 1 evaluated at the channel centre nu_c with
 *      offset nu = (j - M/2) * bw / N  (Sec. 2: each channel gets its own
 *      transfer function; Sec. 3: "complex multiplication with transfer
 *      function").  The *_m entry points also offer one transfer function
 *      for the whole subband (chirp = 1: Eq. 1 about the subband centre), the
 *      alternative that Sec. 2 sets the per-channel choice against.  Dedispersion is the convolution with the INVERSE of the
 *      ISM transfer function (Sec. 1, Sec. 2), i.e. multiplication by
 *      exp(-2 pi i phi), phi = 1e6 * D * DM * nu^2 / (nu_c^2 (nu_c + nu)).
 *   4. halves of each channel swapped back, unitary inverse DFT_M
 *      (e^{+2 pi i}/sqrt(M)) (Sec. 3, "backward FFT").
 *   5. nd/2 samples dropped at each edge, |y_X|^2 + |y_Y|^2 (Stokes I)
 *      (Sec. 3, "transpose, unpad and detect").
 *   6. nint consecutive samples summed into out[dm][s*nchan + c][t].
 *   7. (orc_redigitise) per DM and channel, mean and standard deviation of the
 *      block's samples, then 8-bit codes in decreasing-frequency, time-major
 *      order (Sec. 3, "compute block sums", "compute channel statistics",
 *      "redigitize").
 *   8. (orc_incoherent) incoherent dedispersion of the coherent filterbanks
 *      over fine DM trials (Sec. 4, semi-coherent search).
 *   9. (orc_spectral_kurtosis, orc_redigitise_sk) spectral-kurtosis flags of
 *      the rows of a block and redigitisation with flagged rows set to 128
 *      (Sec. 6, future work; generalised SK estimator).
 *
 * Readings where the paper is silent: D = 4.148808e3 MHz^2 pc^-1 cm^3 s
 * (the paper quotes 1/2.41e-4); transforms unitary; channel index increases
 * with frequency; nd = the smallest even integer >= r*t_d/nchan (Eq. 2 for the
 * lowest channel at the largest |DM|) with (M - nd) divisible by nint.
 *
 * The FFT is an iterative radix-2 Cooley-Tukey transform with each twiddle
 * evaluated directly from cos/sin (no recurrences).  A naive O(N^2) DFT is
 * provided for the tests that pin the FFT.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_D 4.148808e3 /* MHz^2 pc^-1 cm^3 s */
#define ORC_PI 3.14159265358979323846

typedef double complex cplx;

/* Eq. 2: dispersion sweep across [nu_min, nu_max] (MHz) at the given DM. */
double orc_sweep(double nu_min, double nu_max, double dm)
{
    return ORC_D * (1.0 / (nu_min * nu_min) - 1.0 / (nu_max * nu_max)) * dm;
}

/* Centre frequency (MHz) of subband s: the band is contiguous and f_centre is
 * the centre of the whole band. */
double orc_subband_centre(int nsub, double f_centre, double bw, int s)
{
    return f_centre + ((double)s - 0.5 * (double)(nsub - 1)) * bw;
}

/* Centre frequency (MHz) of channel c of a subband centred on nu_s. */
double orc_channel_centre(double nu_s, double bw, int nchan, int c)
{
    return nu_s - 0.5 * bw + ((double)c + 0.5) * bw / (double)nchan;
}

/* Overlap rule of Sec. 2: nd = r t_d / nchan with t_d (Eq. 2) for the lowest
 * channel, at the largest |DM| of the list.  Rounded up to an even integer
 * and then up until (M - nd) is a multiple of nint.  Returns -1 if no nd < M
 * exists.  chirp = 1 (one transfer function for the whole subband): t_d is
 * the sweep across the lowest subband. */
int64_t orc_overlap_m(int nsub, double f_centre, double bw, const double *dm,
                      int ndm, int nchan, int nint, int64_t nbin, int chirp)
{
    double dmax = 0.0;
    for (int i = 0; i < ndm; i++)
        if (fabs(dm[i]) > dmax) dmax = fabs(dm[i]);
    double nu_s0 = orc_subband_centre(nsub, f_centre, bw, 0);
    double lo = nu_s0 - 0.5 * bw;
    double hi = lo + (chirp ? bw : bw / (double)nchan);
    double td = orc_sweep(lo, hi, dmax);
    double r = bw * 1e6;
    double want = r * td / (double)nchan;
    int64_t nd = (int64_t)ceil(want);
    if (nd % 2) nd++;
    int64_t m = nbin / nchan;
    while (nd < m && (m - nd) % nint != 0) nd += 2;
    if (nd >= m) return -1;
    return nd;
}

int64_t orc_overlap(int nsub, double f_centre, double bw, const double *dm,
                    int ndm, int nchan, int nint, int64_t nbin)
{
    return orc_overlap_m(nsub, f_centre, bw, dm, ndm, nchan, nint, nbin, 0);
}

/* In-place iterative radix-2 FFT, unnormalised, kernel exp(sign*2*pi*i*nk/n). */
void orc_fft(cplx *x, int64_t n, int sign)
{
    for (int64_t i = 1, j = 0; i < n; i++) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            cplx t = x[i];
            x[i] = x[j];
            x[j] = t;
        }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t h = len >> 1;
        for (int64_t k = 0; k < h; k++) {
            double ang = (double)sign * 2.0 * ORC_PI * (double)k / (double)len;
            cplx w = cos(ang) + I * sin(ang);
            for (int64_t i = 0; i < n; i += len) {
                cplx u = x[i + k];
                cplx v = x[i + k + h] * w;
                x[i + k] = u + v;
                x[i + k + h] = u - v;
            }
        }
    }
}

/* Naive O(n^2) DFT, unnormalised: y[k] = sum_n x[n] exp(sign*2*pi*i*n*k/n). */
void orc_dft(const cplx *x, cplx *y, int64_t n, int sign)
{
    for (int64_t k = 0; k < n; k++) {
        cplx acc = 0.0;
        for (int64_t j = 0; j < n; j++) {
            int64_t p = (j * k) % n; /* exact reduction of the angle */
            double ang = (double)sign * 2.0 * ORC_PI * (double)p / (double)n;
            acc += x[j] * (cos(ang) + I * sin(ang));
        }
        y[k] = acc;
    }
}

/* Forward spectrum of one segment (step 2): unitary DFT_N with halves swapped
 * so that output bin i has frequency offset (i - N/2) * bw / N. */
static void spectrum(const cplx *x, cplx *xs, cplx *tmp, int64_t n)
{
    memcpy(tmp, x, sizeof(cplx) * (size_t)n);
    orc_fft(tmp, n, -1);
    double sc = 1.0 / sqrt((double)n);
    for (int64_t i = 0; i < n; i++) xs[i] = tmp[(i + n / 2) % n] * sc;
}

/* Steps 3-4 for one channel: chirp multiply, swap halves back, unitary inverse
 * DFT_M.  xs: the swapped forward spectrum of the segment (length N).  The
 * chirp is Eq. 1 about the reference frequency nu_r; bin j of the channel lies
 * at nu_r + dnu + (j - M/2) bw / N (per-channel chirp: nu_r = nu_c, dnu = 0;
 * one chirp for the subband: nu_r = nu_s, dnu = nu_c - nu_s). */
static void channel_series(const cplx *xs, int64_t n, int nchan, int c,
                           double nu_r, double dnu, double bw, double dm, cplx *y, cplx *w)
{
    int64_t m = n / nchan;
    for (int64_t j = 0; j < m; j++) {
        double nu = dnu + ((double)j - 0.5 * (double)m) * bw / (double)n;
        double phi = 1e6 * ORC_D * dm * nu * nu / (nu_r * nu_r * (nu_r + nu));
        cplx h = cos(2.0 * ORC_PI * phi) - I * sin(2.0 * ORC_PI * phi); /* exp(-2 pi i phi) */
        y[j] = xs[(int64_t)c * m + j] * h;
    }
    for (int64_t j = 0; j < m; j++) w[j] = y[(j + m / 2) % m];
    orc_fft(w, m, +1);
    double sc = 1.0 / sqrt((double)m);
    for (int64_t j = 0; j < m; j++) y[j] = w[j] * sc;
}

/* Complex channelised, dedispersed time series of ONE polarisation of ONE
 * segment, before any samples are discarded (steps 2-4).
 * x: N complex samples; y: [nchan][M] complex output. */
void orc_segment_channels_m(const cplx *x, int64_t n, int nchan, double nu_s,
                            double bw, double dm, cplx *y, int chirp)
{
    int64_t m = n / nchan;
    cplx *xs = malloc(sizeof(cplx) * (size_t)n);
    cplx *tmp = malloc(sizeof(cplx) * (size_t)n);
    spectrum(x, xs, tmp, n);
    for (int c = 0; c < nchan; c++) {
        double nu_c = orc_channel_centre(nu_s, bw, nchan, c);
        channel_series(xs, n, nchan, c, chirp ? nu_s : nu_c, chirp ? nu_c - nu_s : 0.0, bw, dm,
                       y + (int64_t)c * m, tmp);
    }
    free(xs);
    free(tmp);
}

void orc_segment_channels(const cplx *x, int64_t n, int nchan, double nu_s,
                          double bw, double dm, cplx *y)
{
    orc_segment_channels_m(x, n, nchan, nu_s, bw, dm, y, 0);
}

/* Plan quantities (overlap-save segment grid). Returns 0 on success. */
int orc_grid(int64_t nsamp, int64_t nbin, int nchan, int64_t nd, int nint,
             int64_t *nvalid, int64_t *nseg, int64_t *nout)
{
    int64_t m = nbin / nchan;
    int64_t s = nbin - nd * nchan;
    if (s <= 0 || nsamp < nbin || (m - nd) % nint != 0) return -1;
    *nvalid = s;
    *nseg = (nsamp - nbin) / s + 1;
    *nout = *nseg * (m - nd) / nint;
    return 0;
}

/* Filterbank rows of one (subband s, segment k) for the DM trials listed in
 * dm_idx.  in: float32 [nsub][nsamp][4] = (Xre, Xim, Yre, Yim) per sample.
 * out: double [ndm_total][nsub*nchan][nout]; only the samples of segment k
 * in rows of subband s and the listed DMs are written. */
static void segment_rows(const float *in, int nsub, int64_t nsamp, double f_centre,
                         double bw, const double *dm, int ndm_total,
                         const int *dm_idx, int ndm_sel, int nchan, int nint,
                         int64_t nbin, int64_t nd, int s, int64_t k, double *out,
                         int64_t nout, int chirp)
{
    int64_t m = nbin / nchan;
    int64_t sv = nbin - nd * nchan;
    int64_t l = (m - nd) / nint;
    double nu_s = orc_subband_centre(nsub, f_centre, bw, s);
    cplx *x = malloc(sizeof(cplx) * (size_t)nbin);
    cplx *xs[2];
    cplx *tmp = malloc(sizeof(cplx) * (size_t)nbin);
    cplx *y = malloc(sizeof(cplx) * (size_t)m);
    double *pw = malloc(sizeof(double) * (size_t)m);
    for (int p = 0; p < 2; p++) {
        xs[p] = malloc(sizeof(cplx) * (size_t)nbin);
        const float *src = in + ((size_t)s * (size_t)nsamp + (size_t)(k * sv)) * 4;
        for (int64_t i = 0; i < nbin; i++)
            x[i] = (double)src[i * 4 + 2 * p] + I * (double)src[i * 4 + 2 * p + 1];
        spectrum(x, xs[p], tmp, nbin);
    }
    (void)ndm_total;
    for (int q = 0; q < ndm_sel; q++) {
        int idm = dm_idx[q];
        for (int c = 0; c < nchan; c++) {
            double nu_c = orc_channel_centre(nu_s, bw, nchan, c);
            for (int64_t i = 0; i < m; i++) pw[i] = 0.0;
            for (int p = 0; p < 2; p++) {
                channel_series(xs[p], nbin, nchan, c, chirp ? nu_s : nu_c, chirp ? nu_c - nu_s : 0.0, bw,
                               dm[idm], y, tmp);
                for (int64_t i = 0; i < m; i++) {
                    double re = creal(y[i]), im = cimag(y[i]);
                    pw[i] += re * re + im * im;
                }
            }
            double *row = out + ((size_t)idm * (size_t)nsub * (size_t)nchan +
                                 (size_t)s * (size_t)nchan + (size_t)c) * (size_t)nout;
            for (int64_t u = 0; u < l; u++) {
                double acc = 0.0;
                for (int qq = 0; qq < nint; qq++) acc += pw[nd / 2 + u * nint + qq];
                row[k * l + u] = acc;
            }
        }
    }
    for (int p = 0; p < 2; p++) free(xs[p]);
    free(x);
    free(tmp);
    free(y);
    free(pw);
}

/* Whole filterbank: out double [ndm][nsub*nchan][nout]. nthreads <= 0 means
 * the OpenMP default.  chirp: 0 per-channel transfer functions, 1 one per
 * subband.  Returns 0 on success, -1 on bad arguments. */
int orc_filterbank_m(const float *in, int nsub, int64_t nsamp, double f_centre,
                     double bw, const double *dm, int ndm, int nchan, int nint,
                     int64_t nbin, int64_t nd, double *out, int nthreads, int chirp)
{
    int64_t sv, nseg, nout;
    if (nbin % nchan || orc_grid(nsamp, nbin, nchan, nd, nint, &sv, &nseg, &nout))
        return -1;
    int *idx = malloc(sizeof(int) * (size_t)ndm);
    for (int i = 0; i < ndm; i++) idx[i] = i;
    int64_t npair = (int64_t)nsub * nseg;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t pr = 0; pr < npair; pr++) {
        int s = (int)(pr / nseg);
        int64_t k = pr % nseg;
        segment_rows(in, nsub, nsamp, f_centre, bw, dm, ndm, idx, ndm, nchan, nint,
                     nbin, nd, s, k, out, nout, chirp);
    }
    free(idx);
    return 0;
}

int orc_filterbank(const float *in, int nsub, int64_t nsamp, double f_centre,
                   double bw, const double *dm, int ndm, int nchan, int nint,
                   int64_t nbin, int64_t nd, double *out, int nthreads)
{
    return orc_filterbank_m(in, nsub, nsamp, f_centre, bw, dm, ndm, nchan, nint, nbin, nd, out, nthreads, 0);
}

/* Sampled tiles: for each tile t, the filterbank samples of segment seg[t] in
 * the rows of subband sub[t] and DM index dmi[t], written to
 * out[t][nchan][(M - nd)/nint].  Each tile depends only on its own segment of
 * input, so this reproduces the corresponding slice of orc_filterbank. */
int orc_tiles_m(const float *in, int nsub, int64_t nsamp, double f_centre, double bw,
                const double *dm, int ndm, int nchan, int nint, int64_t nbin,
                int64_t nd, int ntile, const int *sub, const int64_t *seg,
                const int *dmi, double *out, int nthreads, int chirp)
{
    int64_t sv, nseg, nout;
    if (nbin % nchan || orc_grid(nsamp, nbin, nchan, nd, nint, &sv, &nseg, &nout))
        return -1;
    int64_t l = (nbin / nchan - nd) / nint;
    for (int t = 0; t < ntile; t++)
        if (sub[t] < 0 || sub[t] >= nsub || seg[t] < 0 || seg[t] >= nseg ||
            dmi[t] < 0 || dmi[t] >= ndm)
            return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int t = 0; t < ntile; t++) {
        /* a private one-subband, one-DM view: rows land in a scratch filterbank
         * whose time axis is the segment's own l samples */
        double *scratch = malloc(sizeof(double) * (size_t)nchan * (size_t)l);
        const float *src = in + (size_t)sub[t] * (size_t)nsamp * 4 +
                           (size_t)(seg[t] * sv) * 4;
        segment_rows(src, 1, nbin, orc_subband_centre(nsub, f_centre, bw, sub[t]),
                     bw, dm + dmi[t], 1, (const int[]){0}, 1, nchan, nint, nbin, nd,
                     0, 0, scratch, l, chirp);
        memcpy(out + (size_t)t * (size_t)nchan * (size_t)l, scratch,
               sizeof(double) * (size_t)nchan * (size_t)l);
        free(scratch);
    }
    return 0;
}

int orc_tiles(const float *in, int nsub, int64_t nsamp, double f_centre, double bw,
              const double *dm, int ndm, int nchan, int nint, int64_t nbin,
              int64_t nd, int ntile, const int *sub, const int64_t *seg,
              const int *dmi, double *out, int nthreads)
{
    return orc_tiles_m(in, nsub, nsamp, f_centre, bw, dm, ndm, nchan, nint, nbin, nd, ntile, sub, seg, dmi, out,
                       nthreads, 0);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Redigitisation to 8 bits (Sec. 3, the steps "compute block sums", "compute
 * channel statistics", "redigitize" of Algorithm 1).  For every DM trial and
 * every channel row of a float filterbank fb[ndm][rows][nt] (one data block):
 *   mu = (1/nt) sum_t I_t,  sigma = sqrt((1/nt) sum_t I_t^2 - mu^2)   (FP64);
 * the offset and scale of the row are mu and sigma rounded to FP32 and the
 * gain g = LEVELS / sigma divided in FP32 (g = 0 when sigma = 0), and each
 * sample becomes (orc_codes)
 *   code = clamp(rint(fmaf(I - mu, g, 128)), 0, 255)
 * in FP32 (the paper leaves the mapping open: 128 is the mean and LEVELS = 16
 * code steps span one sigma).  Codes are written in the paper's filterbank
 * order (Sec. 3): per DM, time-major spectra in decreasing frequency,
 * u8[ndm][nt][rows] with row r at position rows - 1 - r.
 * stats (may be NULL) receives (mu, sigma) per (dm, row) in FP64.
 */
#define ORC_LEVELS 16.0f

/* The code step of the redigitisation alone, given each row's statistics:
 * musig[2 i] = mu, musig[2 i + 1] = sigma (FP32) of row i = d rows + r, and
 * (may be NULL) flags[i] != 0 for rows coded 128 whatever their samples.  The
 * codes of a row are unique given these two numbers, so a redigitiser that
 * reports the statistics it used can be checked code for code. */
void orc_codes(const float *fb, int ndm, int rows, int64_t nt, const float *musig, const uint8_t *flags, uint8_t *out)
{
    for (int d = 0; d < ndm; d++) {
        for (int r = 0; r < rows; r++) {
            const size_t i = (size_t)d * rows + r;
            const float *row = fb + i * (size_t)nt;
            const float muf = musig[2 * i], sgf = musig[2 * i + 1];
            const float g = (flags && flags[i]) || !(sgf > 0.0f) ? 0.0f : ORC_LEVELS / sgf;
            for (int64_t t = 0; t < nt; t++) {
                float x = rintf(fmaf(row[t] - muf, g, 128.0f));
                if (x < 0.0f) x = 0.0f;
                if (x > 255.0f) x = 255.0f;
                out[((size_t)d * (size_t)nt + (size_t)t) * rows + (size_t)(rows - 1 - r)] = (uint8_t)x;
            }
        }
    }
}

void orc_redigitise(const float *fb, int ndm, int rows, int64_t nt, uint8_t *out, double *stats)
{
    float *musig = (float *)malloc(sizeof(float) * 2 * (size_t)ndm * rows);
    for (int d = 0; d < ndm; d++) {
        for (int r = 0; r < rows; r++) {
            const size_t i = (size_t)d * rows + r;
            const float *row = fb + i * (size_t)nt;
            double s1 = 0.0, s2 = 0.0;
            for (int64_t t = 0; t < nt; t++) {
                s1 += (double)row[t];
                s2 += (double)row[t] * (double)row[t];
            }
            const double mu = nt > 0 ? s1 / (double)nt : 0.0;
            double var = nt > 0 ? s2 / (double)nt - mu * mu : 0.0;
            if (var < 0.0) var = 0.0;
            const double sigma = sqrt(var);
            if (stats) {
                stats[2 * i] = mu;
                stats[2 * i + 1] = sigma;
            }
            musig[2 * i] = (float)mu;
            musig[2 * i + 1] = (float)sigma;
        }
    }
    orc_codes(fb, ndm, rows, nt, musig, NULL, out);
    free(musig);
}

/*
 * Spectral-kurtosis RFI flags.  Sec. 6 names spectral kurtosis for RFI
 * excision in the statistics step as future work and gives no definition;
 * this takes the generalised spectral-kurtosis estimator.  For one (DM,
 * channel) row of a block of n filterbank samples I_t, each the sum of k
 * squared magnitudes (k = 2 nint: two polarisations, nint time samples),
 *   SK = (n k + 1) / (n - 1) * (n S2 / S1^2 - 1),   S1 = sum I, S2 = sum I^2.
 * For Gaussian voltages I ~ Gamma(k) and SK is 1 on average, with standard
 * deviation sqrt(2 (k + 1) / (k n)) for large n (delta method on the sample
 * variance over the squared sample mean).  A row is flagged when
 * |SK - 1| > nsigma times that deviation.  Rows without power (S1 = 0) have
 * SK = 0; rows of fewer than two samples are never flagged (SK = 1).
 */
double orc_sk_sigma(int64_t n, int k)
{
    return sqrt(2.0 * (double)(k + 1) / ((double)k * (double)n));
}

void orc_spectral_kurtosis(const float *fb, int ndm, int rows, int64_t nt, int k, double nsigma, double *sk,
                           uint8_t *flags)
{
    const double thr = nt > 1 ? nsigma * orc_sk_sigma(nt, k) : 0.0;
    for (int d = 0; d < ndm; d++) {
        for (int r = 0; r < rows; r++) {
            const float *row = fb + ((size_t)d * rows + r) * (size_t)nt;
            double s1 = 0.0, s2 = 0.0;
            for (int64_t t = 0; t < nt; t++) {
                s1 += (double)row[t];
                s2 += (double)row[t] * (double)row[t];
            }
            double v = 1.0;
            if (nt > 1) {
                const double n = (double)nt;
                v = s1 > 0.0 ? (n * k + 1.0) / (n - 1.0) * (n * s2 / (s1 * s1) - 1.0) : 0.0;
            }
            const size_t i = (size_t)d * rows + r;
            if (sk) sk[i] = v;
            if (flags) flags[i] = (uint8_t)(nt > 1 && fabs(v - 1.0) > thr);
        }
    }
}

/* orc_redigitise with spectral-kurtosis flagging: flagged rows get gain 0,
 * i.e. every code 128 (the row's mean). */
void orc_redigitise_sk(const float *fb, int ndm, int rows, int64_t nt, int k, double nsigma, uint8_t *out,
                       double *stats, uint8_t *flags)
{
    orc_redigitise(fb, ndm, rows, nt, out, stats);
    uint8_t *fl = (uint8_t *)malloc((size_t)ndm * rows);
    orc_spectral_kurtosis(fb, ndm, rows, nt, k, nsigma, NULL, fl);
    for (int d = 0; d < ndm; d++)
        for (int r = 0; r < rows; r++) {
            const size_t i = (size_t)d * rows + r;
            if (flags) flags[i] = fl[i];
            if (!fl[i]) continue;
            for (int64_t t = 0; t < nt; t++) out[((size_t)d * (size_t)nt + (size_t)t) * rows + (size_t)(rows - 1 - r)] = 128;
        }
    free(fl);
}

/*
 * Incoherent dedispersion of the coherent filterbanks (Sec. 4, the
 * semi-coherent search: each coherently dedispersed filterbank is
 * incoherently dedispersed over fine DM trials around its coherent DM; Sec. 1
 * describes incoherent dedispersion as shifting each channel's time series by
 * its dispersive delay).  The channels of a coherent filterbank still carry
 * the delays between their reference frequencies nu_r (channel centres, or
 * subband centres for one transfer function per subband), so the shift of row
 * r for total DM = DM_c + ddm_k, in output samples of t_samp seconds, is
 *   d(c, k, r) = rint(D (DM_c + ddm_k) (nu_r^-2 - nu_top^-2) / t_samp),
 * nu_top the highest reference frequency of the band.  With d_lo and d_hi the
 * smallest and largest shift over all (c, k, r), the output is
 *   out[c][k][t] = sum_r fb[c][r][t + d(c, k, r) - d_lo],  t < nt - (d_hi - d_lo)
 * (sums in FP64).  delays (may be NULL) receives d(c, k, r) - d_lo as int32
 * [ndm][nk][rows].  Returns nt_out, or -1 if no output sample remains.
 */
int64_t orc_incoherent(const float *fb, int ndm, int nsub, int nchan, int64_t nt, double f_centre, double bw,
                       int nint, int chirp, const double *dm_c, double ddm_lo, double ddm_step, int nk,
                       double *out, int32_t *delays)
{
    const int rows = nsub * nchan;
    double *nu = malloc(sizeof(double) * (size_t)rows);
    double top = 0.0;
    for (int s = 0; s < nsub; s++) {
        double nu_s = orc_subband_centre(nsub, f_centre, bw, s);
        for (int c = 0; c < nchan; c++) {
            nu[s * nchan + c] = chirp ? nu_s : orc_channel_centre(nu_s, bw, nchan, c);
            if (nu[s * nchan + c] > top) top = nu[s * nchan + c];
        }
    }
    const double tsamp = (double)nint * (double)nchan / (bw * 1e6);
    const size_t nd_tab = (size_t)ndm * (size_t)nk * (size_t)rows;
    int64_t *d = malloc(sizeof(int64_t) * nd_tab);
    int64_t dlo = 0, dhi = 0;
    for (int i = 0; i < ndm; i++)
        for (int k = 0; k < nk; k++)
            for (int r = 0; r < rows; r++) {
                double dm = dm_c[i] + ddm_lo + (double)k * ddm_step;
                int64_t v = (int64_t)llrint(ORC_D * dm * (1.0 / (nu[r] * nu[r]) - 1.0 / (top * top)) / tsamp);
                d[((size_t)i * nk + k) * rows + r] = v;
                if ((i | k | r) == 0 || v < dlo) dlo = v;
                if ((i | k | r) == 0 || v > dhi) dhi = v;
            }
    const int64_t nt_out = nt - (dhi - dlo);
    if (nt_out > 0 && out) {
        for (int i = 0; i < ndm; i++)
            for (int k = 0; k < nk; k++) {
                double *o = out + ((size_t)i * nk + k) * (size_t)nt_out;
                for (int64_t t = 0; t < nt_out; t++) o[t] = 0.0;
                for (int r = 0; r < rows; r++) {
                    const float *row = fb + ((size_t)i * rows + r) * (size_t)nt;
                    const int64_t sh = d[((size_t)i * nk + k) * rows + r] - dlo;
                    for (int64_t t = 0; t < nt_out; t++) o[t] += (double)row[t + sh];
                }
            }
    }
    if (delays)
        for (size_t q = 0; q < nd_tab; q++) delays[q] = (int32_t)(d[q] - dlo);
    free(d);
    free(nu);
    return nt_out > 0 ? nt_out : -1;
}
