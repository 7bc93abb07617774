// FP32 fused path, column sweep: launchers and instantiations, the field's
// column-tile tensor map, and the column tile width (built in or tuned).
#include <cudaTypedefs.h>

#include "launch.cuh"

namespace rtk {

// Tensor map over the complex64 field viewed as an n x 2n float matrix; one
// box is BR rows x C complex columns (2C floats, >= 16 bytes for C >= 2).
cudaError_t make_col_tensor_map(void *map, float2 *E, int n, int colC)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)2 * n, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)2 * n * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * colC), (cuuint32_t)(n < 256 ? n : 256)};
    const cuuint32_t es[2] = {1, 1};
    CUresult r = encode(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, E, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Persistent copy-engine-fed sweep where the tile fits it; otherwise (wide
// tiles at large n) one block per tile, loading straight from global memory.
// order: radix order of the transforms (the one-stage form only; tw must be
// that order's table).
template <int LOGN, int C, int ORDER>
static cudaError_t col_launch32(float2 *E, const float2 *tw, const float2 *h, const void *tmap, int *err,
                                cudaStream_t s)
{
    using F = ColForm<LOGN, C>;
    auto k = [] {
        if constexpr (ORDER == 0) return F::kernel();
        else return k_col_pair1<LOGN, C, ORDER>;
    }();
    constexpr int threads = F::threads;
    constexpr size_t smem = F::smem_handle;
    static std::atomic<unsigned long long> mask{0};
    static std::atomic<int> per_sm{0};
    cudaError_t e = ensure_smem(k, smem, mask);
    if (e != cudaSuccess) return e;
    const int ntiles = (1 << LOGN) / C;
    const int grid = persistent_grid(k, threads, smem, ntiles, per_sm);
    k<<<grid, threads, smem, s>>>(E, tw, h, *static_cast<const CUtensorMap *>(tmap), ntiles, err);
    return cudaGetLastError();
}

template <int LOGN, int C>
static cudaError_t col_diff32_c(float2 *E, const float2 *tw, const float2 *h, const void *tmap, int *err,
                                cudaStream_t s, int order)
{
    if constexpr (!col_fits32<LOGN, C>()) {
        return cudaErrorInvalidValue;
    } else if constexpr (col_tma_fits<LOGN, C>()) {
        if (order == 0) return col_launch32<LOGN, C, 0>(E, tw, h, tmap, err, s);
        if constexpr (ColForm<LOGN, C>::form == 2 && radix_orders(LOGN) > 1) {
            if (order == 1) return col_launch32<LOGN, C, 1>(E, tw, h, tmap, err, s);
            if constexpr (radix_orders(LOGN) > 2) {
                if (order == 2) return col_launch32<LOGN, C, 2>(E, tw, h, tmap, err, s);
            }
        }
        return cudaErrorInvalidValue;
    } else {
        if (order != 0) return cudaErrorInvalidValue;
        cudaError_t e = col_attr<float, LOGN, C, MODE_DIFF>();
        if (e != cudaSuccess) return e;
        k_col<float, LOGN, C, MODE_DIFF>
            <<<(1 << LOGN) / C, C * Plan<LOGN>::T, col_smem_bytes<float, LOGN, C>(), s>>>(E, tw, h);
        return cudaGetLastError();
    }
}

template <int LOGN>
static cudaError_t col_diff32(int colC, float2 *E, const float2 *tw, const float2 *h, const void *tmap, int *err,
                              cudaStream_t s, int order)
{
    switch (colC) {
    case 2: return col_diff32_c<LOGN, 2>(E, tw, h, tmap, err, s, order);
    case 4: return col_diff32_c<LOGN, 4>(E, tw, h, tmap, err, s, order);
    case 8: return col_diff32_c<LOGN, 8>(E, tw, h, tmap, err, s, order);
    case 16: return col_diff32_c<LOGN, 16>(E, tw, h, tmap, err, s, order);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_diffract32(int logn, int colC, float2 *E, const float2 *tw, const float2 *h, const void *tmap,
                                  int *err, cudaStream_t s, int order)
{
    RTK_LOGN_CASES(col_diff32, colC, E, tw, h, tmap, err, s, order)
}

// Radix orders the column sweep of side 2^logn offers at tile width colC.
template <int LOGN> static int col_orders_impl(int colC)
{
    auto orders = [](bool tma) { return RTK_COL_FORM == 2 && tma ? radix_orders(LOGN) : 1; };
    switch (colC) {
    case 2: return col_fits32<LOGN, 2>() ? orders(col_tma_fits<LOGN, 2>()) : 0;
    case 4: return col_fits32<LOGN, 4>() ? orders(col_tma_fits<LOGN, 4>()) : 0;
    case 8: return col_fits32<LOGN, 8>() ? orders(col_tma_fits<LOGN, 8>()) : 0;
    case 16: return col_fits32<LOGN, 16>() ? orders(col_tma_fits<LOGN, 16>()) : 0;
    default: return 0;
    }
}

int col_orders32(int logn, int colC) { RTK_LOGN_CASES(col_orders_impl, colC) }

template <int LOGN, int C> static cudaError_t col_prep32_c()
{
    if constexpr (!col_fits32<LOGN, C>()) {
        return cudaErrorInvalidValue;
    } else if constexpr (col_tma_fits<LOGN, C>()) {
        static std::atomic<unsigned long long> mask{0};
        return ensure_smem(ColForm<LOGN, C>::kernel(), ColForm<LOGN, C>::smem_handle, mask);
    } else {
        return col_attr<float, LOGN, C, MODE_DIFF>();
    }
}

template <int LOGN> static cudaError_t col_prep32(int colC)
{
    switch (colC) {
    case 2: return col_prep32_c<LOGN, 2>();
    case 4: return col_prep32_c<LOGN, 4>();
    case 8: return col_prep32_c<LOGN, 8>();
    case 16: return col_prep32_c<LOGN, 16>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_col32(int logn, int colC) { RTK_LOGN_CASES(col_prep32, colC) }

// ---- column tile width ------------------------------------------------------------

template <int LOGN> static int col_ok32(int colC)
{
    switch (colC) {
    case 2: return col_fits32<LOGN, 2>();
    case 4: return col_fits32<LOGN, 4>();
    case 8: return col_fits32<LOGN, 8>();
    case 16: return col_fits32<LOGN, 16>();
    default: return 0;
    }
}

int col_tile_ok32(int logn, int colC) { RTK_LOGN_CASES(col_ok32, colC) }

// Tile widths chosen by the autotuner (0: not tuned), per log2 n.
static std::atomic<int> g_tuned_col[13];

// Built-in widths: the autotuner's choices on GB300 (2 at 4096, 4 at
// 1024-2048, 8 below; 16 only where 8 does not fit a whole warp's rows).
int builtin_col_tile32(int logn) { return logn >= 12 ? 2 : (logn >= 10 ? 4 : (logn >= 6 ? 8 : 16)); }

int default_col_tile32(int logn)
{
    if (logn >= 0 && logn < 13) {
        const int t = g_tuned_col[logn].load();
        if (t > 0 && col_tile_ok32(logn, t)) return t;
    }
    return builtin_col_tile32(logn);
}

int set_tuned_col_tile32(int logn, int colC)
{
    if (logn < 5 || logn > 12 || (colC != 0 && !col_tile_ok32(logn, colC))) return 0;
    g_tuned_col[logn].store(colC);
    return 1;
}

int tuned_col_tile32(int logn) { return (logn >= 0 && logn < 13) ? g_tuned_col[logn].load() : 0; }

// Radix orders chosen by the autotuner (0: the built-in sequence), per log2 n.
static std::atomic<int> g_tuned_order[13];

int set_tuned_col_order32(int logn, int order)
{
    if (logn < 5 || logn > 12 || order < 0 || order >= radix_orders(logn)) return 0;
    g_tuned_order[logn].store(order);
    return 1;
}

int tuned_col_order32(int logn) { return (logn >= 0 && logn < 13) ? g_tuned_order[logn].load() : 0; }

}  // namespace rtk
