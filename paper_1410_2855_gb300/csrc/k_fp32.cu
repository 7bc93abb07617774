// FP32 fused path: launchers and instantiations of the two bounce sweeps and
// of the FP32 set-up and spectrum kernels.
#include <cudaTypedefs.h>

#include "setup_kernels.cuh"
#include "sweep.cuh"
#include "sweep_tma.cuh"

// 1: persistent copy-engine-fed sweeps (default); 0: one block per line group.
#ifndef RTK_PERSISTENT
#define RTK_PERSISTENT 1
#endif

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

template <int LOGN, int C> constexpr bool col_fits32()
{
    return C <= (1 << LOGN) && C * Plan<LOGN>::T <= 1024 && col_smem_bytes<float, LOGN, C>() <= 227 * 1024;
}

// ---- persistent launch geometry -------------------------------------------------

static int sm_count()
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
static int persistent_grid(K kernel, int threads, size_t smem, int work, std::atomic<int> &per_sm)
{
    int b = per_sm.load();
    if (b <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess || b <= 0) b = 1;
        per_sm.store(b);
    }
    const int g = b * sm_count();
    return g < work ? g : work;
}

template <int LOGN> constexpr int tma_lpc() { return Plan<LOGN>::T >= 64 ? 1 : 64 / Plan<LOGN>::T; }

template <int LOGN, int C> constexpr bool col_tma_fits()
{
    return col_fits32<LOGN, C>() && C >= 2 && ColPlan<LOGN, C>::total <= 227 * 1024;
}

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

// ---- column sweep ---------------------------------------------------------------

template <int LOGN, int C>
static cudaError_t col_tma32_c(float2 *E, const float2 *tw, const float2 *h, const void *tmap, int *err,
                               cudaStream_t s)
{
    if constexpr (!col_tma_fits<LOGN, C>()) {
        return cudaErrorInvalidValue;
    } else {
        using L = ColPlan<LOGN, C>;
        auto k = k_col_tma<LOGN, C>;
        static std::atomic<unsigned long long> mask{0};
        static std::atomic<int> per_sm{0};
        cudaError_t e = ensure_smem(k, L::total, mask);
        if (e != cudaSuccess) return e;
        const int ntiles = (1 << LOGN) / C;
        const int grid = persistent_grid(k, C * Plan<LOGN>::T, L::total, ntiles, per_sm);
        k<<<grid, C * Plan<LOGN>::T, L::total, s>>>(E, tw, h, *static_cast<const CUtensorMap *>(tmap), ntiles, err);
        return cudaGetLastError();
    }
}

template <int LOGN, int C>
static cudaError_t col_diff32_c(float2 *E, const float2 *tw, const float2 *h, const void *tmap, int *err,
                                cudaStream_t s)
{
    if constexpr (!col_fits32<LOGN, C>()) {
        return cudaErrorInvalidValue;
    } else if constexpr (RTK_PERSISTENT && col_tma_fits<LOGN, C>()) {
        return col_tma32_c<LOGN, C>(E, tw, h, tmap, err, s);
    } else {
        cudaError_t e = col_attr<float, LOGN, C, MODE_DIFF>();
        if (e != cudaSuccess) return e;
        k_col<float, LOGN, C, MODE_DIFF>
            <<<(1 << LOGN) / C, C * Plan<LOGN>::T, col_smem_bytes<float, LOGN, C>(), s>>>(E, tw, h);
        return cudaGetLastError();
    }
}

template <int LOGN>
static cudaError_t col_diff32(int colC, float2 *E, const float2 *tw, const float2 *h, const void *tmap, int *err,
                              cudaStream_t s)
{
    switch (colC) {
    case 2: return col_diff32_c<LOGN, 2>(E, tw, h, tmap, err, s);
    case 4: return col_diff32_c<LOGN, 4>(E, tw, h, tmap, err, s);
    case 8: return col_diff32_c<LOGN, 8>(E, tw, h, tmap, err, s);
    case 16: return col_diff32_c<LOGN, 16>(E, tw, h, tmap, err, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_diffract32(int logn, int colC, float2 *E, const float2 *tw, const float2 *h, const void *tmap,
                                  int *err, cudaStream_t s)
{
    RTK_LOGN_CASES(col_diff32, colC, E, tw, h, tmap, err, s)
}

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

// ---- row sweep (diffraction along x + local map) --------------------------------

template <int LOGN, int PE>
static cudaError_t row_tma32_pe(float2 *E, float *N, const float2 *tw, const float2 *h, const GainParams<float> &g,
                                const StatParams &st, cudaStream_t s)
{
    constexpr int LPC = tma_lpc<LOGN>();
    using L = RowStage<LOGN, LPC, RTK_ROW_PP, PE == PE_TABLE>;
    auto k = k_row_tma<LOGN, LPC, PE>;
    static std::atomic<unsigned long long> mask{0};
    static std::atomic<int> per_sm{0};
    cudaError_t e = ensure_smem(k, L::total, mask);
    if (e != cudaSuccess) return e;
    const int ngroups = (1 << LOGN) / LPC;
    const int grid = persistent_grid(k, LPC * Plan<LOGN>::T, L::total, ngroups, per_sm);
    k<<<grid, LPC * Plan<LOGN>::T, L::total, s>>>(E, N, tw, h, g, st, ngroups);
    return cudaGetLastError();
}

template <int LOGN, int PE>
static cudaError_t row_dg32_pe(float2 *E, float *N, const float2 *tw, const float2 *h, const GainParams<float> &g,
                               const StatParams &st, cudaStream_t s)
{
    if constexpr (RTK_PERSISTENT) return row_tma32_pe<LOGN, PE>(E, N, tw, h, g, st, s);
    cudaError_t e = row_attr<float, LOGN, MODE_DIFF_GAIN, PE>();
    if (e != cudaSuccess) return e;
    constexpr int LPC = row_lpc<LOGN>();
    k_row<float, LOGN, MODE_DIFF_GAIN, PE>
        <<<(1 << LOGN) / LPC, LPC * Plan<LOGN>::T, row_smem_bytes<float, LOGN>(), s>>>(E, E, N, tw, h, g, st);
    return cudaGetLastError();
}

template <int LOGN>
static cudaError_t row_dg32(int pe, float2 *E, float *N, const float2 *tw, const float2 *h,
                            const GainParams<float> &g, const StatParams &st, cudaStream_t s)
{
    switch (pe) {
    case PE_SG10: return row_dg32_pe<LOGN, PE_SG10>(E, N, tw, h, g, st, s);
    case PE_UNIFORM: return row_dg32_pe<LOGN, PE_UNIFORM>(E, N, tw, h, g, st, s);
    case PE_TABLE: return row_dg32_pe<LOGN, PE_TABLE>(E, N, tw, h, g, st, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_row_diffract_gain32(int logn, int pe, float2 *E, float *N, const float2 *tw, const float2 *h,
                                       const GainParams<float> &g, const StatParams &st, cudaStream_t s)
{
    RTK_LOGN_CASES(row_dg32, pe, E, N, tw, h, g, st, s)
}

template <int LOGN> static int row_blocks_impl() { return (1 << LOGN) / row_lpc<LOGN>(); }
int row_blocks32(int logn) { RTK_LOGN_CASES(row_blocks_impl) }

// ---- batched sweeps (resonators of one grid size per launch) -----------------

template <int LOGN, int C>
static cudaError_t col_batch32_c(const BatchRes *res, int nres, const float2 *tw, int *err, cudaStream_t s)
{
    if constexpr (!col_tma_fits<LOGN, C>()) {
        return cudaErrorInvalidValue;
    } else {
        using L = ColPlan<LOGN, C>;
        auto k = k_col_tma_batch<LOGN, C>;
        static std::atomic<unsigned long long> mask{0};
        static std::atomic<int> per_sm{0};
        cudaError_t e = ensure_smem(k, L::total, mask);
        if (e != cudaSuccess) return e;
        const int items = nres * ((1 << LOGN) / C);
        const int grid = persistent_grid(k, C * Plan<LOGN>::T, L::total, items, per_sm);
        k<<<grid, C * Plan<LOGN>::T, L::total, s>>>(res, nres, tw, err);
        return cudaGetLastError();
    }
}

template <int LOGN>
static cudaError_t col_batch32(int colC, const BatchRes *res, int nres, const float2 *tw, int *err, cudaStream_t s)
{
    switch (colC) {
    case 2: return col_batch32_c<LOGN, 2>(res, nres, tw, err, s);
    case 4: return col_batch32_c<LOGN, 4>(res, nres, tw, err, s);
    case 8: return col_batch32_c<LOGN, 8>(res, nres, tw, err, s);
    case 16: return col_batch32_c<LOGN, 16>(res, nres, tw, err, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_batch32(int logn, int colC, const BatchRes *res, int nres, const float2 *tw, int *err,
                               cudaStream_t s)
{
    if (nres <= 0) return cudaSuccess;
    RTK_LOGN_CASES(col_batch32, colC, res, nres, tw, err, s)
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

template <int LOGN, int C> static cudaError_t col_batch_prep_c()
{
    if constexpr (!col_tma_fits<LOGN, C>()) {
        return cudaErrorInvalidValue;
    } else {
        static std::atomic<unsigned long long> mask{0};
        return ensure_smem(k_col_tma_batch<LOGN, C>, ColPlan<LOGN, C>::total, mask);
    }
}

template <int LOGN> static cudaError_t batch_prep32(int colC)
{
    static std::atomic<unsigned long long> mask{0};
    constexpr int LPC = tma_lpc<LOGN>();
    cudaError_t e = ensure_smem(k_row_tma_batch<LOGN, LPC>, RowPlan<LOGN, LPC>::total, mask);
    if (e != cudaSuccess) return e;
    switch (colC) {
    case 2: return col_batch_prep_c<LOGN, 2>();
    case 4: return col_batch_prep_c<LOGN, 4>();
    case 8: return col_batch_prep_c<LOGN, 8>();
    case 16: return col_batch_prep_c<LOGN, 16>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_batch32(int logn, int colC) { RTK_LOGN_CASES(batch_prep32, colC) }

// ---- plain line transforms (spectrum readout) -----------------------------------

template <int LOGN>
static cudaError_t row_fft32(const float2 *in, float2 *out, const float2 *tw, int dir, cudaStream_t s)
{
    constexpr size_t sm = row_smem_bytes<float, LOGN>();
    constexpr int LPC = row_lpc<LOGN>();
    const GainParams<float> g{};
    const StatParams st{};
    cudaError_t e;
    if (dir < 0) {
        if ((e = row_attr<float, LOGN, MODE_FWD>()) != cudaSuccess) return e;
        k_row<float, LOGN, MODE_FWD, PE_SG10>
            <<<(1 << LOGN) / LPC, LPC * Plan<LOGN>::T, sm, s>>>(in, out, nullptr, tw, nullptr, g, st);
    } else {
        if ((e = row_attr<float, LOGN, MODE_INV>()) != cudaSuccess) return e;
        k_row<float, LOGN, MODE_INV, PE_SG10>
            <<<(1 << LOGN) / LPC, LPC * Plan<LOGN>::T, sm, s>>>(in, out, nullptr, tw, nullptr, g, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_row_fft32(int logn, const float2 *in, float2 *out, const float2 *tw, int dir, cudaStream_t s)
{
    RTK_LOGN_CASES(row_fft32, in, out, tw, dir, s)
}

// Column tile of the readout transforms: 16 columns up to n = 512, then fewer.
template <int LOGN> constexpr int fft_col_c32() { return LOGN >= 12 ? 2 : (LOGN >= 11 ? 4 : (LOGN >= 10 ? 8 : 16)); }

template <int LOGN>
static cudaError_t col_fft32(float2 *X, const float2 *tw, int dir, cudaStream_t s)
{
    constexpr int C = fft_col_c32<LOGN>();
    constexpr size_t sm = col_smem_bytes<float, LOGN, C>();
    cudaError_t e;
    if (dir < 0) {
        if ((e = col_attr<float, LOGN, C, MODE_FWD>()) != cudaSuccess) return e;
        k_col<float, LOGN, C, MODE_FWD><<<(1 << LOGN) / C, C * Plan<LOGN>::T, sm, s>>>(X, tw, nullptr);
    } else {
        if ((e = col_attr<float, LOGN, C, MODE_INV>()) != cudaSuccess) return e;
        k_col<float, LOGN, C, MODE_INV><<<(1 << LOGN) / C, C * Plan<LOGN>::T, sm, s>>>(X, tw, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_col_fft32(int logn, float2 *X, const float2 *tw, int dir, cudaStream_t s)
{
    RTK_LOGN_CASES(col_fft32, X, tw, dir, s)
}

// ---- preparation before graph capture -------------------------------------------

template <int LOGN, int C> static cudaError_t col_prep32_c()
{
    if constexpr (!col_fits32<LOGN, C>()) {
        return cudaErrorInvalidValue;
    } else if constexpr (RTK_PERSISTENT && col_tma_fits<LOGN, C>()) {
        static std::atomic<unsigned long long> mask{0};
        return ensure_smem(k_col_tma<LOGN, C>, ColPlan<LOGN, C>::total, mask);
    } else {
        return col_attr<float, LOGN, C, MODE_DIFF>();
    }
}

template <int LOGN, int PE> static cudaError_t row_prep32()
{
    if constexpr (RTK_PERSISTENT) {
        static std::atomic<unsigned long long> mask{0};
        return ensure_smem(k_row_tma<LOGN, tma_lpc<LOGN>(), PE>,
                           RowStage<LOGN, tma_lpc<LOGN>(), RTK_ROW_PP, PE == PE_TABLE>::total, mask);
    } else {
        return row_attr<float, LOGN, MODE_DIFF_GAIN, PE>();
    }
}

template <int LOGN> static cudaError_t prep32(int colC, int pe)
{
    cudaError_t e;
    switch (pe) {
    case PE_SG10: e = row_prep32<LOGN, PE_SG10>(); break;
    case PE_UNIFORM: e = row_prep32<LOGN, PE_UNIFORM>(); break;
    case PE_TABLE: e = row_prep32<LOGN, PE_TABLE>(); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    switch (colC) {
    case 2: return col_prep32_c<LOGN, 2>();
    case 4: return col_prep32_c<LOGN, 4>();
    case 8: return col_prep32_c<LOGN, 8>();
    case 16: return col_prep32_c<LOGN, 16>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_bounce32(int logn, int colC, int pe) { RTK_LOGN_CASES(prep32, colC, pe) }

// ---- set-up and readout -------------------------------------------------------

int twiddle_entries(int logn) { return twiddle_count(logn); }

cudaError_t launch_tables32(int n, double alpha, float2 *tw, float2 *h, cudaStream_t s)
{
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    const int total = twiddle_count(logn);
    k_prop_table<float2><<<(n + 255) / 256, 256, 0, s>>>(n, alpha, h);
    if (total > 0) k_twiddles<float2><<<(total + 255) / 256, 256, 0, s>>>(logn, total, tw);
    return cudaGetLastError();
}

cudaError_t launch_noise32(int n, unsigned long long seed, double amp, float2 *E, cudaStream_t s)
{
    k_noise<float2><<<grid_for((size_t)n * n, 256, 2048), 256, 0, s>>>(n, seed, amp, E);
    return cudaGetLastError();
}

cudaError_t launch_pump32(int n, int kind, double g0, double order, double radius, const double *profile,
                          float *out, cudaStream_t s)
{
    k_pump<float><<<grid_for((size_t)n * n, 256, 2048), 256, 0, s>>>(n, kind, g0, order, radius, profile, out);
    return cudaGetLastError();
}

cudaError_t launch_power32(int n, const float2 *X, float *S, cudaStream_t s)
{
    const size_t P = (size_t)n * n;
    k_power<float2, float><<<grid_for(P, 256, 2048), 256, 0, s>>>(P, X, S);
    return cudaGetLastError();
}

int peak_blocks(int n) { return grid_for((size_t)n * n, 256, 1024); }

cudaError_t launch_peak32(int n, int ring, const float *S, double *part_val, long long *part_idx, unsigned int *count,
                          PeakResult *out, cudaStream_t s)
{
    k_peak<float><<<peak_blocks(n), 256, 0, s>>>(n, ring, S, part_val, part_idx, count, out);
    return cudaGetLastError();
}

}  // namespace rtk
