// Device allocation with a fault-injection hook (rt_debug_fail_alloc): the
// failure is produced on the host, before any device call, so tests of the
// out-of-memory paths never disturb the GPU.
#include <mutex>

#include "rt.h"
#include "rt_internal.h"

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
