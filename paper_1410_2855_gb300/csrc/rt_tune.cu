// Autotuning of the column sweep's tile width and radix order (include/rt.h,
// rt_autotune: the sweep alone; rt_autotune_concurrent: whole bounces of
// resonators running together).
#include <chrono>
#include <vector>

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

rt_status rt_autotune_concurrent(int n, int resonators, int bounces, int reps, int *best_col_tile, int *best_order,
                                 double *best_rate)
{
    if (!best_col_tile || !best_order || !best_rate || n < 32 || n > 4096 || (n & (n - 1)) || resonators < 1 ||
        resonators > 16 || bounces < 1 || bounces > 100000 || reps < 1)
        return RT_EINVAL;
    const int logn = log2_of(n);
    const int keep_tile = tuned_col_tile32(logn), keep_order = tuned_col_order32(logn);
    std::vector<cudaStream_t> streams(resonators, nullptr);
    rt_status st = RT_OK;
    for (cudaStream_t &s : streams)
        if (st == RT_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) st = RT_ECUDA;
    int best = 0, best_o = 0;
    double best_r = 0.0;
    for (int colC : {2, 4, 8, 16}) {
        if (st != RT_OK || !col_tile_ok32(logn, colC)) continue;
        for (int o = 0; o < col_orders32(logn, colC) && st == RT_OK; ++o) {
            // handles created with col_tile = 0 take the tuned pair
            set_tuned_col_tile32(logn, colC);
            set_tuned_col_order32(logn, o);
            std::vector<rt_handle *> hs(resonators, nullptr);
            for (int i = 0; i < resonators && st == RT_OK; ++i) {
                rt_opts op;
                rt_opts_default(&op);
                op.cuda_stream = streams[i];
                op.chunk = bounces;
                op.history_cap = 0;
                op.seed += (unsigned long long)i;
                st = rt_create(n, 1000.0, nullptr, 0.3, 1e4, 0.9, &op, &hs[i]);
            }
            auto run = [&]() {
                for (rt_handle *h : hs)
                    if (st == RT_OK) st = rt_step(h, bounces);
                for (rt_handle *h : hs)
                    if (st == RT_OK) st = rt_sync(h);
            };
            run();  // warm-up: graph capture, first touch
            double t = 1e300;
            for (int r = 0; r < reps && st == RT_OK; ++r) {
                const auto t0 = std::chrono::steady_clock::now();
                run();
                const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                t = dt < t ? dt : t;
            }
            for (rt_handle *h : hs) rt_destroy(h);
            if (st != RT_OK) break;
            const double rate = (double)resonators * bounces / t;
            if (rate > best_r) {
                best_r = rate;
                best = colC;
                best_o = o;
            }
        }
    }
    for (cudaStream_t s : streams)
        if (s) cudaStreamDestroy(s);
    if (st != RT_OK || !best) {  // leave the earlier choice in force
        set_tuned_col_tile32(logn, keep_tile);
        set_tuned_col_order32(logn, keep_order);
        return st != RT_OK ? st : RT_EINVAL;
    }
    set_tuned_col_tile32(logn, best);
    set_tuned_col_order32(logn, best_o);
    *best_col_tile = best;
    *best_order = best_o;
    *best_rate = best_r;
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

rt_status rt_tune_set_batch_split(int parts)
{
    if (parts < 0 || parts > 8) return RT_EINVAL;
    set_batch_split(parts);
    return RT_OK;
}

rt_status rt_tune_get_batch_split(int *parts)
{
    if (!parts) return RT_EINVAL;
    *parts = batch_split_setting();
    return RT_OK;
}

rt_status rt_tune_get_batch_mixed(int *mixed)
{
    if (!mixed) return RT_EINVAL;
    *mixed = batch_mixed() ? 1 : 0;
    return RT_OK;
}

}  // extern "C"
