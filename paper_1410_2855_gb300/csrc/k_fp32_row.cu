// FP32 fused path, row sweep (diffraction along x + local map): launchers and
// instantiations, one per grid size, pump evaluation and aperture form.
#include "launch.cuh"

namespace rtk {

template <int LOGN, int PE, int FEAT>
static cudaError_t row_dg32_k(float2 *E, float *N, const float2 *tw, const float2 *h, const GainParams<float> &g,
                              const StatParams &st, cudaStream_t s)
{
    constexpr int LPC = tma_lpc<LOGN>();
    using L = RowStage<LOGN, LPC, RTK_ROW_PP, PE == PE_TABLE>;
    auto k = k_row_tma<LOGN, LPC, PE, FEAT>;
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
    switch (feature_form(g)) {
    case FEAT_TABLE: return row_dg32_k<LOGN, PE, FEAT_TABLE>(E, N, tw, h, g, st, s);
    case FEAT_TABLE_EXACT: return row_dg32_k<LOGN, PE, FEAT_TABLE_EXACT>(E, N, tw, h, g, st, s);
    default: return row_dg32_k<LOGN, PE, FEAT_PLAIN>(E, N, tw, h, g, st, s);
    }
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

// The persistent grid never exceeds the number of row groups.
template <int LOGN> static int row_blocks_impl() { return (1 << LOGN) / tma_lpc<LOGN>(); }
int row_blocks32(int logn) { RTK_LOGN_CASES(row_blocks_impl) }

template <int LOGN, int PE, int FEAT> static cudaError_t row_prep32_k()
{
    static std::atomic<unsigned long long> mask{0};
    constexpr int LPC = tma_lpc<LOGN>();
    return ensure_smem(k_row_tma<LOGN, LPC, PE, FEAT>, RowStage<LOGN, LPC, RTK_ROW_PP, PE == PE_TABLE>::total, mask);
}

template <int LOGN, int PE> static cudaError_t row_prep32_pe(int feat)
{
    switch (feat) {
    case FEAT_TABLE: return row_prep32_k<LOGN, PE, FEAT_TABLE>();
    case FEAT_TABLE_EXACT: return row_prep32_k<LOGN, PE, FEAT_TABLE_EXACT>();
    default: return row_prep32_k<LOGN, PE, FEAT_PLAIN>();
    }
}

template <int LOGN> static cudaError_t row_prep32(int pe, int feat)
{
    switch (pe) {
    case PE_SG10: return row_prep32_pe<LOGN, PE_SG10>(feat);
    case PE_UNIFORM: return row_prep32_pe<LOGN, PE_UNIFORM>(feat);
    case PE_TABLE: return row_prep32_pe<LOGN, PE_TABLE>(feat);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_row32(int logn, int pe, int feat) { RTK_LOGN_CASES(row_prep32, pe, feat) }

cudaError_t prepare_bounce32(int logn, int colC, int pe, int feat)
{
    cudaError_t e = prepare_row32(logn, pe, feat);
    return e != cudaSuccess ? e : prepare_col32(logn, colC);
}

}  // namespace rtk
