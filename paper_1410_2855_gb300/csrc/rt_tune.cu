// Autotuning of the column sweep's tile width (include/rt.h, rt_autotune).
#include "engine.h"

using namespace rtk;

extern "C" {

rt_status rt_autotune(int n, int reps, int *best_col_tile, double *best_us)
{
    if (!best_col_tile || !best_us || reps <= 0 || n < 32 || n > 4096 || (n & (n - 1))) return RT_EINVAL;
    const int logn = log2_of(n);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return RT_ECUDA;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int best = 0;
    double best_t = 1e300;
    rt_status st = RT_OK;
    for (int colC : {2, 4, 8, 16}) {
        if (!col_tile_ok32(logn, colC)) continue;
        rt_opts o;
        rt_opts_default(&o);
        o.col_tile = colC;
        o.chunk = 0;
        o.history_cap = 0;
        o.cuda_stream = s;
        rt_handle *h = nullptr;
        if ((st = rt_create(n, 100.0, nullptr, 0.2, 1000.0, 0.95, &o, &h)) != RT_OK) break;
        rt_step(h, 3);
        cudaEventRecord(a, s);
        for (int r = 0; r < reps && st == RT_OK; ++r) st = rt_sweep(h, RT_SWEEP_COLUMNS);
        cudaEventRecord(b, s);
        if (st == RT_OK && cudaEventSynchronize(b) != cudaSuccess) st = RT_ECUDA;
        float ms = 0.0f;
        if (st == RT_OK) cudaEventElapsedTime(&ms, a, b);
        rt_destroy(h);
        if (st != RT_OK) break;
        const double us = 1e3 * ms / reps;
        if (us < best_t) {
            best_t = us;
            best = colC;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(s);
    if (st != RT_OK) return st;
    if (!best) return RT_EINVAL;
    set_tuned_col_tile32(logn, best);
    *best_col_tile = best;
    *best_us = best_t;
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

}  // extern "C"
