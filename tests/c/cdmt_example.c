/*
 * A C caller of the library, with no Python in between: plans a small
 * coherent-dedispersion problem, fills the input with seeded complex noise,
 * runs the FP32 and FP16 forms through cdmt_execute, and writes both
 * filterbanks (float32, [ndm][nsub*nchan][nout]) to the files named on the
 * command line and the input (float32 [nsub][nsamp][4]) to OUT_FP32.input.
 * Exit status 0 on success; errors are printed with the library's message.
 *
 *   cdmt_example OUT_FP32 OUT_FP16
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "cdmt.h"

#define NSUB 2
#define NSAMP ((1 << 15) + 123)
#define NCHAN 8
#define NINT 4

static int check(int rc, cdmt_plan_t p, const char *what)
{
    if (rc != CDMT_OK) fprintf(stderr, "%s: %s (%s)\n", what, cdmt_strerror(rc), cdmt_last_error(p));
    return rc;
}

/* 64-bit LCG and Box-Muller: complex Gaussian samples with E|x|^2 = 1 per polarisation */
static double uniform(uint64_t *s)
{
    *s = *s * 6364136223846793005ULL + 1442695040888963407ULL;
    return ((*s >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static int run(int precision, const float *d_in, const char *path)
{
    const double dms[3] = {0.0, 4.0, 8.0};
    cdmt_opts o = {0};
    o.nbin = 1 << 14;
    o.nd = -1;
    o.precision = precision;
    cdmt_plan_t p = NULL;
    if (check(cdmt_plan_ex(&p, NSUB, NSAMP, 140.0, 0.1953125, dms, 3, NCHAN, NINT, &o), NULL, "cdmt_plan_ex")) return 1;
    cdmt_info inf;
    if (check(cdmt_plan_info(p, &inf), p, "cdmt_plan_info")) return 1;
    const size_t n = (size_t)inf.ndm * NSUB * NCHAN * (size_t)inf.nout;
    float *d_out = NULL;
    if (cudaMalloc((void **)&d_out, n * sizeof(float)) != cudaSuccess) return 1;
    if (check(cdmt_execute(p, d_in, d_out, NULL, NULL), p, "cdmt_execute")) return 1;
    float *h = (float *)malloc(n * sizeof(float));
    if (!h || cudaMemcpy(h, d_out, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    if (check(cdmt_device_status(p), p, "cdmt_device_status")) return 1;
    FILE *f = fopen(path, "wb");
    if (!f || fwrite(h, sizeof(float), n, f) != n) return 1;
    fclose(f);
    printf("%s form: %lld DMs x %d rows x %lld samples -> %s\n", precision == CDMT_PREC_FP32 ? "FP32" : "FP16",
           (long long)inf.ndm, NSUB * NCHAN, (long long)inf.nout, path);
    free(h);
    cudaFree(d_out);
    return check(cdmt_destroy(p), NULL, "cdmt_destroy") != CDMT_OK;
}

int main(int argc, char **argv)
{
    if (argc != 3) {
        fprintf(stderr, "usage: %s OUT_FP32 OUT_FP16\n", argv[0]);
        return 2;
    }
    const size_t nf = (size_t)NSUB * NSAMP * 4;
    float *x = (float *)malloc(nf * sizeof(float));
    uint64_t s = 12345;
    for (size_t i = 0; i < nf; i += 2) {
        /* Box-Muller with radius sqrt(-ln u): real and imaginary parts N(0, 1/2) */
        const double r = sqrt(-log(uniform(&s))), a = 6.283185307179586 * uniform(&s);
        x[i] = (float)(r * cos(a));
        x[i + 1] = (float)(r * sin(a));
    }
    float *d_in = NULL;
    if (cudaMalloc((void **)&d_in, nf * sizeof(float)) != cudaSuccess ||
        cudaMemcpy(d_in, x, nf * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
        fprintf(stderr, "device memory\n");
        return 1;
    }
    /* the input goes next to the first output, for a checker that recomputes it */
    char inpath[4096];
    snprintf(inpath, sizeof inpath, "%s.input", argv[1]);
    FILE *fi = fopen(inpath, "wb");
    if (!fi || fwrite(x, sizeof(float), nf, fi) != nf) return 1;
    fclose(fi);
    int rc = run(CDMT_PREC_FP32, d_in, argv[1]);
    if (!rc) rc = run(CDMT_PREC_FP16, d_in, argv[2]);
    cudaFree(d_in);
    free(x);
    return rc;
}
