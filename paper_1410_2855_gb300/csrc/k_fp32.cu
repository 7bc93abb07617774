// FP32 fused path: set-up tables, noise, pump, aperture phase, and the
// spectrum readout (plain line transforms, power, folded argmax).  The two
// bounce sweeps are in k_fp32_col.cu, k_fp32_row.cu and k_fp32_batch.cu.
#include "launch.cuh"
#include "setup_kernels.cuh"

namespace rtk {

// ---- plain line transforms (spectrum readout) -----------------------------------

template <int LOGN>
static cudaError_t row_fft32(const float2 *in, float2 *out, const float2 *tw, int dir, cudaStream_t s)
{
    constexpr size_t sm = row_smem_bytes<float, LOGN>();
    constexpr int LPC = row_lpc<LOGN>();
    cudaError_t e;
    if (dir < 0) {
        if ((e = row_attr<float, LOGN, MODE_FWD>()) != cudaSuccess) return e;
        k_row<float, LOGN, MODE_FWD><<<(1 << LOGN) / LPC, LPC * Plan<LOGN>::T, sm, s>>>(in, out, tw, nullptr);
    } else {
        if ((e = row_attr<float, LOGN, MODE_INV>()) != cudaSuccess) return e;
        k_row<float, LOGN, MODE_INV><<<(1 << LOGN) / LPC, LPC * Plan<LOGN>::T, sm, s>>>(in, out, tw, nullptr);
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

// ---- plain diffraction (intracavity readout) ----------------------------------

template <int LOGN>
static cudaError_t row_diff_plain32(const float2 *in, float2 *out, const float2 *tw, const float2 *h, cudaStream_t s)
{
    constexpr int LPC = row_lpc<LOGN>();
    cudaError_t e = row_attr<float, LOGN, MODE_DIFF>();
    if (e != cudaSuccess) return e;
    k_row<float, LOGN, MODE_DIFF>
        <<<(1 << LOGN) / LPC, LPC * Plan<LOGN>::T, row_smem_bytes<float, LOGN>(), s>>>(in, out, tw, h);
    return cudaGetLastError();
}

cudaError_t launch_row_diffract_plain32(int logn, const float2 *in, float2 *out, const float2 *tw, const float2 *h,
                                        cudaStream_t s)
{
    RTK_LOGN_CASES(row_diff_plain32, in, out, tw, h, s)
}

template <int LOGN>
static cudaError_t col_diff_plain32(float2 *X, const float2 *tw, const float2 *h, cudaStream_t s)
{
    constexpr int C = fft_col_c32<LOGN>();
    cudaError_t e = col_attr<float, LOGN, C, MODE_DIFF>();
    if (e != cudaSuccess) return e;
    k_col<float, LOGN, C, MODE_DIFF>
        <<<(1 << LOGN) / C, C * Plan<LOGN>::T, col_smem_bytes<float, LOGN, C>(), s>>>(X, tw, h);
    return cudaGetLastError();
}

cudaError_t launch_col_diffract_plain32(int logn, float2 *X, const float2 *tw, const float2 *h, cudaStream_t s)
{
    RTK_LOGN_CASES(col_diff_plain32, X, tw, h, s)
}

// ---- set-up and readout -------------------------------------------------------

// The most entries a table of any radix order of side 2^logn needs.
int twiddle_entries(int logn)
{
    int m = 0;
    for (int o = 0; o < radix_orders(logn); ++o) m = twiddle_count(logn, o) > m ? twiddle_count(logn, o) : m;
    return m;
}

cudaError_t launch_twiddles32(int n, int order, float2 *tw, cudaStream_t s)
{
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    if (order < 0 || order >= radix_orders(logn)) return cudaErrorInvalidValue;
    const int total = twiddle_count(logn, order);
    if (total > 0) k_twiddles<float2><<<(total + 255) / 256, 256, 0, s>>>(logn, order, total, tw);
    return cudaGetLastError();
}

cudaError_t launch_tables32(int n, double alpha, float2 *tw, float2 *h, cudaStream_t s)
{
    k_prop_table<float2><<<(n + 255) / 256, 256, 0, s>>>(n, alpha, h);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? launch_twiddles32(n, 0, tw, s) : e;
}

cudaError_t launch_prop32(int n, double alpha, float2 *h, cudaStream_t s)
{
    k_prop_table<float2><<<(n + 255) / 256, 256, 0, s>>>(n, alpha, h);
    return cudaGetLastError();
}

cudaError_t launch_noise32(int n, unsigned long long seed, double amp, float2 *E, cudaStream_t s)
{
    k_noise<float2><<<grid_for((size_t)n * n, 256, 2048), 256, 0, s>>>(n, seed, amp, E);
    return cudaGetLastError();
}

double lens_curvature(double alpha, double z_over_F) { return 3.14159265358979323846 / (4.0 * alpha) * z_over_F; }

cudaError_t launch_lens32(int n, double c, int edge, int taper, float2 *lens, cudaStream_t s)
{
    k_lens_table<float2><<<(n + 255) / 256, 256, 0, s>>>(n, c / 3.14159265358979323846, edge, taper, lens);
    return cudaGetLastError();
}

cudaError_t launch_phase32(int n, double c, int edge, int taper, const double *psi, float2 *phase, cudaStream_t s)
{
    k_phase_table<float2><<<grid_for((size_t)n * n, 256, 2048), 256, 0, s>>>(n, c / 3.14159265358979323846, edge,
                                                                              taper, psi, phase);
    return cudaGetLastError();
}

cudaError_t launch_pattern32(int n, int kind, int q, int alt, double w, double env, double curv, double amp,
                             float2 *E, cudaStream_t s)
{
    k_pattern<float2><<<grid_for((size_t)n * n, 256, 2048), 256, 0, s>>>(n, kind, q, alt, w, env, curv, amp, E);
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
