// FP32 fused path, batched sweeps (all resonators of one grid size per
// persistent launch): launchers and instantiations.
#include "launch.cuh"

namespace rtk {

template <int LOGN, int C, int ORDER>
static cudaError_t col_batch_launch(const BatchRes *res, int nres, const float2 *tw, int *err, cudaStream_t s)
{
    using F = ColForm<LOGN, C>;
    auto k = [] {
        if constexpr (ORDER == 0) return F::batch_kernel();
        else return k_col_pair1_batch<LOGN, C, ORDER>;
    }();
    constexpr int threads = F::threads;
    static std::atomic<unsigned long long> mask{0};
    static std::atomic<int> per_sm{0};
    cudaError_t e = ensure_smem(k, F::smem, mask);
    if (e != cudaSuccess) return e;
    const int items = nres * ((1 << LOGN) / C);
    const int grid = persistent_grid(k, threads, F::smem, items, per_sm);
    k<<<grid, threads, F::smem, s>>>(res, nres, tw, err);
    return cudaGetLastError();
}

// order: radix order of the column transforms (the one-stage form; tw is
// that order's table).
template <int LOGN, int C>
static cudaError_t col_batch32_c(const BatchRes *res, int nres, const float2 *tw, int *err, cudaStream_t s, int order)
{
    if constexpr (!col_tma_fits<LOGN, C>()) {
        return cudaErrorInvalidValue;
    } else {
        if (order == 0) return col_batch_launch<LOGN, C, 0>(res, nres, tw, err, s);
        if constexpr (ColForm<LOGN, C>::form == 2 && radix_orders(LOGN) > 1) {
            if (order == 1) return col_batch_launch<LOGN, C, 1>(res, nres, tw, err, s);
            if constexpr (radix_orders(LOGN) > 2) {
                if (order == 2) return col_batch_launch<LOGN, C, 2>(res, nres, tw, err, s);
            }
        }
        return cudaErrorInvalidValue;
    }
}

template <int LOGN>
static cudaError_t col_batch32(int colC, const BatchRes *res, int nres, const float2 *tw, int *err, cudaStream_t s,
                               int order)
{
    switch (colC) {
    case 2: return col_batch32_c<LOGN, 2>(res, nres, tw, err, s, order);
    case 4: return col_batch32_c<LOGN, 4>(res, nres, tw, err, s, order);
    case 8: return col_batch32_c<LOGN, 8>(res, nres, tw, err, s, order);
    case 16: return col_batch32_c<LOGN, 16>(res, nres, tw, err, s, order);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_batch32(int logn, int colC, const BatchRes *res, int nres, const float2 *tw, int *err,
                               cudaStream_t s, int order)
{
    if (nres <= 0) return cudaSuccess;
    RTK_LOGN_CASES(col_batch32, colC, res, nres, tw, err, s, order)
}

template <int LOGN>
static cudaError_t row_batch32(const BatchRes *res, int nres, const float2 *tw, int *err, cudaStream_t s)
{
    constexpr int LPC = tma_lpc<LOGN>();
    using L = RowPlan<LOGN, LPC>;
    auto k = k_row_tma_batch<LOGN, LPC>;
    static std::atomic<unsigned long long> mask{0};
    static std::atomic<int> per_sm{0};
    cudaError_t e = ensure_smem(k, L::total, mask);
    if (e != cudaSuccess) return e;
    const int items = nres * ((1 << LOGN) / LPC);
    const int grid = persistent_grid(k, LPC * Plan<LOGN>::T, L::total, items, per_sm);
    k<<<grid, LPC * Plan<LOGN>::T, L::total, s>>>(res, nres, tw, err);
    return cudaGetLastError();
}

cudaError_t launch_row_batch32(int logn, const BatchRes *res, int nres, const float2 *tw, int *err, cudaStream_t s)
{
    if (nres <= 0) return cudaSuccess;
    RTK_LOGN_CASES(row_batch32, res, nres, tw, err, s)
}

template <int LOGN> static int row_groups_impl() { return (1 << LOGN) / tma_lpc<LOGN>(); }
int row_groups32(int logn) { RTK_LOGN_CASES(row_groups_impl) }

template <int LOGN, int C, int ORDER> static cudaError_t col_batch_prep_o()
{
    static std::atomic<unsigned long long> mask{0};
    if constexpr (ORDER == 0) return ensure_smem(ColForm<LOGN, C>::batch_kernel(), ColForm<LOGN, C>::smem, mask);
    else return ensure_smem(k_col_pair1_batch<LOGN, C, ORDER>, ColForm<LOGN, C>::smem, mask);
}

template <int LOGN, int C> static cudaError_t col_batch_prep_c(int order)
{
    if constexpr (!col_tma_fits<LOGN, C>()) {
        return cudaErrorInvalidValue;
    } else {
        if (order == 0) return col_batch_prep_o<LOGN, C, 0>();
        if constexpr (ColForm<LOGN, C>::form == 2 && radix_orders(LOGN) > 1) {
            if (order == 1) return col_batch_prep_o<LOGN, C, 1>();
            if constexpr (radix_orders(LOGN) > 2) {
                if (order == 2) return col_batch_prep_o<LOGN, C, 2>();
            }
        }
        return cudaErrorInvalidValue;
    }
}

template <int LOGN> static cudaError_t batch_prep32(int colC, int order)
{
    static std::atomic<unsigned long long> mask{0};
    constexpr int LPC = tma_lpc<LOGN>();
    cudaError_t e = ensure_smem(k_row_tma_batch<LOGN, LPC>, RowPlan<LOGN, LPC>::total, mask);
    if (e != cudaSuccess) return e;
    switch (colC) {
    case 2: return col_batch_prep_c<LOGN, 2>(order);
    case 4: return col_batch_prep_c<LOGN, 4>(order);
    case 8: return col_batch_prep_c<LOGN, 8>(order);
    case 16: return col_batch_prep_c<LOGN, 16>(order);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_batch32(int logn, int colC, int order) { RTK_LOGN_CASES(batch_prep32, colC, order) }

}  // namespace rtk
