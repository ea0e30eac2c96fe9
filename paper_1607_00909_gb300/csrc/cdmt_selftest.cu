// Checks of the failure paths of the tensor-core kernels that need no fault.
//
// cdmt_selftest_wait runs the bounded mbarrier wait those kernels use between a
// GEMM's commit and its read-out (tc::mbar_wait: a time limit on the global
// timer plus a cap on polls) on a barrier that nothing arrives on, and reports
// that the wait gave up and how long it took; with `arrive` set, one arrival
// completes the phase first and the wait must succeed.  cdmt_inject_timeout
// marks a plan's status word as a kernel whose wait gave up does, so that the
// host-side recovery (later DM-stage launches return before they allocate tensor
// memory; cdmt_device_status reports and clears) can be exercised.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cdmt.h"
#include "cdmt_plan_impl.h"
#include "tc_ptx.cuh"

namespace {

__global__ void k_wait_selftest(uint64_t limit_ns, int arrive, unsigned long long *res)
{
    __shared__ uint64_t mb;
    if (threadIdx.x == 0) {
        cdmt::tc::mbar_init(&mb, 1);
        cdmt::tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (arrive) {
        uint64_t state;
        asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(cdmt::tc::smem_addr(&mb)) : "memory");
        (void)state;
    }
    const uint64_t t0 = cdmt::tc::globaltimer_ns();
    const bool done = cdmt::tc::mbar_wait(&mb, 0, limit_ns, 1u << 26);
    res[0] = done ? 0ull : 1ull;
    res[1] = cdmt::tc::globaltimer_ns() - t0;
}

}  // namespace

extern "C" {

int cdmt_selftest_wait(double limit_ms, int arrive, int *gave_up, double *waited_ms)
{
    if (!gave_up || !waited_ms || !(limit_ms > 0.0) || limit_ms > 1000.0) return CDMT_EINVAL;
    unsigned long long *d = nullptr, h[2] = {0, 0};
    if (cudaMalloc(&d, sizeof h) != cudaSuccess) {
        cudaGetLastError();
        return CDMT_ENOMEM;
    }
    k_wait_selftest<<<1, 32>>>((uint64_t)(limit_ms * 1e6), arrive, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return CDMT_ECUDA;
    *gave_up = (int)h[0];
    *waited_ms = (double)h[1] * 1e-6;
    return CDMT_OK;
}

int cdmt_inject_timeout(cdmt_plan_t p)
{
    if (!p) return CDMT_EINVAL;
    const int one = 1;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device && cudaSetDevice(p->device) != cudaSuccess) return CDMT_ECUDA;
    cudaError_t e = cudaSuccess;
    if (p->groups.empty()) e = cudaMemcpy(p->d_status, &one, sizeof one, cudaMemcpyHostToDevice);
    for (auto &g : p->groups)
        if (e == cudaSuccess) e = cudaMemcpy(g.plan->d_status, &one, sizeof one, cudaMemcpyHostToDevice);
    if (cur != p->device) cudaSetDevice(cur);
    return e == cudaSuccess ? CDMT_OK : CDMT_ECUDA;
}

}  // extern "C"
