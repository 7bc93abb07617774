// Device allocation with a fault-injection hook (rt_debug_fail_alloc): the
// failure is produced on the host, before any device call, so tests of the
// out-of-memory paths never disturb the GPU.  And a probe of the sweeps'
// bounded copy waits (rt_debug_wait_probe): a barrier armed for a copy that
// is never issued, so the wait runs out and reports, with nothing in flight.
#include <mutex>

#include "rt.h"
#include "rt_internal.h"
#include "sweep_tma.cuh"

namespace {
// Allocations to let through before failures start (-1: off) and how many
// consecutive allocations then fail (-1: all of them).
std::mutex g_mu;
long long g_fail_after = -1, g_fail_count = 0;
}  // namespace

namespace rtk {

cudaError_t dev_alloc(void **p, size_t bytes)
{
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_fail_after > 0) {
            --g_fail_after;
        } else if (g_fail_after == 0 && g_fail_count != 0) {
            if (g_fail_count > 0 && --g_fail_count == 0) g_fail_after = -1;
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}

}  // namespace rtk

extern "C" rt_status rt_debug_fail_alloc_n(int after, int count)
{
    std::lock_guard<std::mutex> lk(g_mu);
    const bool on = after >= 0 && count != 0;
    g_fail_after = on ? (long long)after : -1;
    g_fail_count = on ? (count < 0 ? -1 : (long long)count) : 0;
    return RT_OK;
}

extern "C" rt_status rt_debug_fail_alloc(int after) { return rt_debug_fail_alloc_n(after, 1); }

namespace rtk {

// One block: stage barrier 0 (and 1 when `drain`, standing for the next
// item's copy) armed for 16 bytes that no copy delivers, then the sweeps'
// own stage wait.  Each wait gives up after its limit (2 s).
__global__ void k_wait_probe(int *err, int drain)
{
    __shared__ __align__(8) uint64_t bar[2];
    init_stage_barriers(bar);
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar[0], 16u);
        if (drain) mbar_arrive_expect_tx(&bar[1], 16u);
    }
    __syncthreads();
    stage_wait_or_abort(bar, 0, drain != 0, err);
}

}  // namespace rtk

extern "C" rt_status rt_debug_wait_probe(int drain, int *device_status)
{
    using namespace rtk;
    if (!device_status) return RT_EINVAL;
    *device_status = 0;
    int *err = nullptr;
    if (dev_alloc(&err, sizeof(int)) != cudaSuccess) return RT_ENOMEM;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 64, 0, s>>>(err, drain ? 1 : 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(device_status, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (s) cudaStreamDestroy(s);
    cudaFree(err);
    return e == cudaSuccess ? RT_OK : RT_ECUDA;
}
