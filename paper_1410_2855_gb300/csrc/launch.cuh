// Host-side launch helpers shared by the FP32 translation units: dispatch on
// log2(n), persistent grid sizing, and which column tiles fit.
#pragma once

#include <atomic>

#include "sweep.cuh"
#include "sweep_tma.cuh"

namespace rtk {

#define RTK_LOGN_CASES(F, ...)              \
    switch (logn) {                         \
    case 5: return F<5>(__VA_ARGS__);       \
    case 6: return F<6>(__VA_ARGS__);       \
    case 7: return F<7>(__VA_ARGS__);       \
    case 8: return F<8>(__VA_ARGS__);       \
    case 9: return F<9>(__VA_ARGS__);       \
    case 10: return F<10>(__VA_ARGS__);     \
    case 11: return F<11>(__VA_ARGS__);     \
    case 12: return F<12>(__VA_ARGS__);     \
    default: return cudaErrorInvalidValue;  \
    }

// A column tile of C columns fits one block (threads, shared memory).
template <int LOGN, int C> constexpr bool col_fits32()
{
    return C <= (1 << LOGN) && C * Plan<LOGN>::T <= 1024 && col_smem_bytes<float, LOGN, C>() <= 227 * 1024;
}

// Form of the persistent column sweeps: 0 one column per thread
// (k_col_tma), 1 column pairs with two stages and register tables
// (k_col_pair), 2 column pairs with one stage, two or more blocks per SM
// (k_col_pair1).  All three give the same bits.
#ifndef RTK_COL_FORM
#define RTK_COL_FORM 2
#endif
template <int LOGN, int C> struct ColForm {
    static constexpr int form = RTK_COL_FORM;
    static constexpr int threads = (form == 0 ? C : C / 2) * Plan<LOGN>::T;
    static constexpr size_t smem = form == 2 ? ColStage1<LOGN, C>::total : ColPlan<LOGN, C>::total;
    // the handle kernel of form 2 may also stage its tables (ColStage1::tabs_fit)
    static constexpr size_t smem_handle = form == 2 ? ColStage1<LOGN, C>::total_tabs : smem;
    static constexpr auto kernel()
    {
        if constexpr (form == 2) return k_col_pair1<LOGN, C>;
        else if constexpr (form == 1) return k_col_pair<LOGN, C>;
        else return k_col_tma<LOGN, C>;
    }
    static constexpr auto batch_kernel()
    {
        if constexpr (form == 2) return k_col_pair1_batch<LOGN, C>;
        else if constexpr (form == 1) return k_col_pair_batch<LOGN, C>;
        else return k_col_tma_batch<LOGN, C>;
    }
};

// ... and its copy-engine-fed persistent form (the one built) fits too.
template <int LOGN, int C> constexpr bool col_tma_fits()
{
    return col_fits32<LOGN, C>() && C >= 2 && ColForm<LOGN, C>::smem <= 227 * 1024;
}

// Rows per block of the persistent row sweeps: one row from n = 1024 up,
// else enough rows for 64 threads.
template <int LOGN> constexpr int tma_lpc() { return Plan<LOGN>::T >= 64 ? 1 : 64 / Plan<LOGN>::T; }

inline int sm_count()
{
    static std::atomic<int> cached{0};
    int v = cached.load();
    if (v > 0) return v;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
    cached.store(v);
    return v;
}

// Blocks of a persistent launch: resident blocks per SM x SMs, capped by the work.
template <typename K>
inline int persistent_grid(K kernel, int threads, size_t smem, int work, std::atomic<int> &per_sm)
{
    int b = per_sm.load();
    if (b <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess || b <= 0) b = 1;
        per_sm.store(b);
    }
    const int g = b * sm_count();
    return g < work ? g : work;
}

}  // namespace rtk
