// Autotuning of the column sweep's tile width (include/rt.h, rt_autotune).
#include "engine.h"
#include "fft_core.cuh"

using namespace rtk;

extern "C" {

rt_status rt_autotune(int n, int reps, int *best_col_tile, double *best_us)
{
    if (!best_col_tile || !best_us || reps <= 0 || n < 32 || n > 4096 || (n & (n - 1))) return RT_EINVAL;
    const int logn = log2_of(n);
    const size_t P = (size_t)n * n;
    const int orders = radix_orders(logn);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return RT_ECUDA;
    cudaEvent_t a = nullptr, b = nullptr;
    float2 *E = nullptr, *h = nullptr, *tw[3] = {nullptr, nullptr, nullptr};
    int *err = nullptr;
    rt_status st = RT_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && st == RT_OK) st = e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;
        return st == RT_OK;
    };
    // a scratch field (a smooth-phase start is not needed: the timing does
    // not depend on the values) with the propagator and every order's twiddles
    if (ok(cudaEventCreate(&a)) && ok(cudaEventCreate(&b)) && ok(dev_alloc(&E, P * sizeof(float2))) &&
        ok(dev_alloc(&h, n * sizeof(float2))) && ok(dev_alloc(&err, sizeof(int))) &&
        ok(cudaMemsetAsync(E, 0, P * sizeof(float2), s)) && ok(cudaMemsetAsync(err, 0, sizeof(int), s)))
        for (int o = 0; o < orders && st == RT_OK; ++o)
            if (ok(dev_alloc(&tw[o], (size_t)(twiddle_entries(logn) + 1) * sizeof(float2))))
                ok(o == 0 ? launch_tables32(n, 0.5, tw[0], h, s) : launch_twiddles32(n, o, tw[o], s));
    int best = 0, best_order = 0;
    double best_t = 1e300;
    for (int colC : {2, 4, 8, 16}) {
        if (st != RT_OK || !col_tile_ok32(logn, colC)) continue;
        alignas(64) unsigned char map[128];
        if (!ok(make_col_tensor_map(map, E, n, colC))) break;
        for (int o = 0; o < col_orders32(logn, colC) && st == RT_OK; ++o) {
            for (int r = 0; r < 3 && st == RT_OK; ++r) ok(launch_col_diffract32(logn, colC, E, tw[o], h, map, err, s, o));
            ok(cudaEventRecord(a, s));
            for (int r = 0; r < reps && st == RT_OK; ++r) ok(launch_col_diffract32(logn, colC, E, tw[o], h, map, err, s, o));
            ok(cudaEventRecord(b, s));
            float ms = 0.0f;
            if (ok(cudaEventSynchronize(b)) && ok(cudaEventElapsedTime(&ms, a, b))) {
                const double us = 1e3 * ms / reps;
                if (us < best_t) {
                    best_t = us;
                    best = colC;
                    best_order = o;
                }
            }
        }
    }
    int kerr = 0;
    if (st == RT_OK && ok(cudaMemcpy(&kerr, err, sizeof(int), cudaMemcpyDeviceToHost)) && kerr) st = (rt_status)kerr;
    for (float2 *p : tw)
        if (p) cudaFree(p);
    if (E) cudaFree(E);
    if (h) cudaFree(h);
    if (err) cudaFree(err);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaStreamDestroy(s);
    if (st != RT_OK) return st;
    if (!best) return RT_EINVAL;
    set_tuned_col_tile32(logn, best);
    set_tuned_col_order32(logn, best_order);
    *best_col_tile = best;
    *best_us = best_t;
    return RT_OK;
}

rt_status rt_tune_set_order(int n, int order)
{
    if (n < 32 || n > 4096 || (n & (n - 1))) return RT_EINVAL;
    return set_tuned_col_order32(log2_of(n), order) ? RT_OK : RT_EINVAL;
}

rt_status rt_tune_get_order(int n, int *order, int *orders)
{
    if (!order || !orders || n < 32 || n > 4096 || (n & (n - 1))) return RT_EINVAL;
    *order = tuned_col_order32(log2_of(n));
    *orders = radix_orders(log2_of(n));
    return RT_OK;
}

rt_status rt_tune_set(int n, int col_tile)
{
    if (n < 32 || n > 4096 || (n & (n - 1))) return RT_EINVAL;
    return set_tuned_col_tile32(log2_of(n), col_tile) ? RT_OK : RT_EINVAL;
}

rt_status rt_tune_get(int n, int *col_tile, int *tuned)
{
    if (!col_tile || !tuned || n < 32 || n > 4096 || (n & (n - 1))) return RT_EINVAL;
    const int logn = log2_of(n);
    *tuned = tuned_col_tile32(logn) > 0;
    *col_tile = default_col_tile32(logn);
    return RT_OK;
}

rt_status rt_tune_set_batch_mixed(int mixed)
{
    if (mixed != 0 && mixed != 1) return RT_EINVAL;
    set_batch_mixed(mixed == 1);
    return RT_OK;
}

rt_status rt_tune_get_batch_mixed(int *mixed)
{
    if (!mixed) return RT_EINVAL;
    *mixed = batch_mixed() ? 1 : 0;
    return RT_OK;
}

}  // extern "C"
