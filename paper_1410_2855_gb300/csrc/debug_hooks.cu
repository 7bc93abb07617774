// Device allocation with a fault-injection hook (rt_debug_fail_alloc): the
// failure is produced on the host, before any device call, so tests of the
// out-of-memory paths never disturb the GPU.
#include <atomic>

#include "rt.h"
#include "rt_internal.h"

namespace {
std::atomic<long long> g_fail_after{-1};  // allocations to let through before one fails; -1: off
}  // namespace

namespace rtk {

cudaError_t dev_alloc(void **p, size_t bytes)
{
    long long k = g_fail_after.load();
    while (k >= 0) {
        if (g_fail_after.compare_exchange_weak(k, k - 1)) {
            if (k == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

}  // namespace rtk

extern "C" rt_status rt_debug_fail_alloc(int after)
{
    g_fail_after.store(after < 0 ? -1 : (long long)after);
    return RT_OK;
}
