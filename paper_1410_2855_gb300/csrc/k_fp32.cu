// FP32 fused path: launchers and instantiations of the two bounce sweeps and
// of the FP32 set-up and spectrum kernels.
#include "setup_kernels.cuh"
#include "sweep.cuh"

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

// ---- column sweep ---------------------------------------------------------------

template <int LOGN, int C>
static cudaError_t col_diff32_c(float2 *E, const float2 *tw, const float2 *h, cudaStream_t s)
{
    if constexpr (!col_fits32<LOGN, C>()) {
        return cudaErrorInvalidValue;
    } else {
        cudaError_t e = col_attr<float, LOGN, C, MODE_DIFF>();
        if (e != cudaSuccess) return e;
        k_col<float, LOGN, C, MODE_DIFF>
            <<<(1 << LOGN) / C, C * Plan<LOGN>::T, col_smem_bytes<float, LOGN, C>(), s>>>(E, tw, h);
        return cudaGetLastError();
    }
}

template <int LOGN>
static cudaError_t col_diff32(int colC, float2 *E, const float2 *tw, const float2 *h, cudaStream_t s)
{
    switch (colC) {
    case 2: return col_diff32_c<LOGN, 2>(E, tw, h, s);
    case 4: return col_diff32_c<LOGN, 4>(E, tw, h, s);
    case 8: return col_diff32_c<LOGN, 8>(E, tw, h, s);
    case 16: return col_diff32_c<LOGN, 16>(E, tw, h, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_diffract32(int logn, int colC, float2 *E, const float2 *tw, const float2 *h, cudaStream_t s)
{
    RTK_LOGN_CASES(col_diff32, colC, E, tw, h, s)
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

// ---- row sweep (diffraction along x + local map) --------------------------------

template <int LOGN, int PE>
static cudaError_t row_dg32_pe(float2 *E, float *N, const float2 *tw, const float2 *h, const GainParams<float> &g,
                               const StatParams &st, cudaStream_t s)
{
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
    if constexpr (!col_fits32<LOGN, C>()) return cudaErrorInvalidValue;
    else return col_attr<float, LOGN, C, MODE_DIFF>();
}

template <int LOGN> static cudaError_t prep32(int colC, int pe)
{
    cudaError_t e;
    switch (pe) {
    case PE_SG10: e = row_attr<float, LOGN, MODE_DIFF_GAIN, PE_SG10>(); break;
    case PE_UNIFORM: e = row_attr<float, LOGN, MODE_DIFF_GAIN, PE_UNIFORM>(); break;
    case PE_TABLE: e = row_attr<float, LOGN, MODE_DIFF_GAIN, PE_TABLE>(); break;
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
