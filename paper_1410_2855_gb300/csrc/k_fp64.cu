// Plain FP64 path: the bounce as six separate sweeps (row FFT, column FFT,
// propagator multiply, column inverse FFT, row inverse FFT, local map), each
// one pass over HBM in complex128.  It is the unfused comparison form and the
// FP64 reference of the library; plus the FP64 set-up and spectrum kernels.
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

template <int LOGN>
static cudaError_t row_fft64(const double2 *in, double2 *out, const double2 *tw, int dir, cudaStream_t s)
{
    constexpr size_t sm = row_smem_bytes<double, LOGN>();
    constexpr int LPC = row_lpc<LOGN>();
    if (dir < 0) {
        cudaError_t e = row_attr<double, LOGN, MODE_FWD>();
        auto k = k_row<double, LOGN, MODE_FWD>;
        if (e != cudaSuccess) return e;
        k<<<(1 << LOGN) / LPC, LPC * Plan<LOGN>::T, sm, s>>>(in, out, tw, nullptr);
    } else {
        cudaError_t e = row_attr<double, LOGN, MODE_INV>();
        auto k = k_row<double, LOGN, MODE_INV>;
        if (e != cudaSuccess) return e;
        k<<<(1 << LOGN) / LPC, LPC * Plan<LOGN>::T, sm, s>>>(in, out, tw, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_row_fft64(int logn, const double2 *in, double2 *out, const double2 *tw, int dir, cudaStream_t s)
{
    RTK_LOGN_CASES(row_fft64, in, out, tw, dir, s)
}

// Column tile: 8 columns up to n = 512, then fewer (shared memory, registers).
template <int LOGN> constexpr int col_c64() { return LOGN >= 11 ? 2 : (LOGN >= 10 ? 4 : 8); }

template <int LOGN>
static cudaError_t col_fft64(double2 *X, const double2 *tw, int dir, cudaStream_t s)
{
    constexpr int C = col_c64<LOGN>();
    constexpr size_t sm = col_smem_bytes<double, LOGN, C>();
    if (dir < 0) {
        cudaError_t e = col_attr<double, LOGN, C, MODE_FWD>();
        auto k = k_col<double, LOGN, C, MODE_FWD>;
        if (e != cudaSuccess) return e;
        k<<<(1 << LOGN) / C, C * Plan<LOGN>::T, sm, s>>>(X, tw, nullptr);
    } else {
        cudaError_t e = col_attr<double, LOGN, C, MODE_INV>();
        auto k = k_col<double, LOGN, C, MODE_INV>;
        if (e != cudaSuccess) return e;
        k<<<(1 << LOGN) / C, C * Plan<LOGN>::T, sm, s>>>(X, tw, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_col_fft64(int logn, double2 *X, const double2 *tw, int dir, cudaStream_t s)
{
    RTK_LOGN_CASES(col_fft64, X, tw, dir, s)
}

// Plain diffraction of a copy of the field (intracavity readout).
template <int LOGN>
static cudaError_t row_diff_plain64(const double2 *in, double2 *out, const double2 *tw, const double2 *h,
                                    cudaStream_t s)
{
    constexpr int LPC = row_lpc<LOGN>();
    cudaError_t e = row_attr<double, LOGN, MODE_DIFF>();
    if (e != cudaSuccess) return e;
    k_row<double, LOGN, MODE_DIFF>
        <<<(1 << LOGN) / LPC, LPC * Plan<LOGN>::T, row_smem_bytes<double, LOGN>(), s>>>(in, out, tw, h);
    return cudaGetLastError();
}

cudaError_t launch_row_diffract_plain64(int logn, const double2 *in, double2 *out, const double2 *tw,
                                        const double2 *h, cudaStream_t s)
{
    RTK_LOGN_CASES(row_diff_plain64, in, out, tw, h, s)
}

template <int LOGN>
static cudaError_t col_diff_plain64(double2 *X, const double2 *tw, const double2 *h, cudaStream_t s)
{
    constexpr int C = col_c64<LOGN>();
    cudaError_t e = col_attr<double, LOGN, C, MODE_DIFF>();
    if (e != cudaSuccess) return e;
    k_col<double, LOGN, C, MODE_DIFF>
        <<<(1 << LOGN) / C, C * Plan<LOGN>::T, col_smem_bytes<double, LOGN, C>(), s>>>(X, tw, h);
    return cudaGetLastError();
}

cudaError_t launch_col_diffract_plain64(int logn, double2 *X, const double2 *tw, const double2 *h, cudaStream_t s)
{
    RTK_LOGN_CASES(col_diff_plain64, X, tw, h, s)
}

// E[y, x] *= h[x] h[y]: the separable transfer function, 1/n^2 included.
__global__ void __launch_bounds__(256) k_mul_h64(int n, double2 *E, const double2 *__restrict__ h)
{
    const size_t P = (size_t)n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)(i / n);
        E[i] = cmul(E[i], cmul(h[x], h[y]));
    }
}

cudaError_t launch_mul_h64(int n, double2 *E, const double2 *h, cudaStream_t s)
{
    k_mul_h64<<<grid_for((size_t)n * n, 256, 2048), 256, 0, s>>>(n, E, h);
    return cudaGetLastError();
}

// Local map in FP64 (gain, mirror with its aperture phase, absorbing edge,
// inversion relaxation) and the mean intensity of the new field.
__global__ void __launch_bounds__(256) k_gain64(int n, double2 *E, double *__restrict__ N, GainParams<double> g,
                                               StatParams st)
{
    const size_t P = (size_t)n * n;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)(i / n);
        const double nn = N[i];
        double2 e = E[i];
        const double inten = e.x * e.x + e.y * e.y;
        const bool inside = x >= g.edge && x < n - g.edge && y >= g.edge && y < n - g.edge;
        const double gain = inside ? g.sqrtR * exp(0.5 * nn) : 0.0;
        e = cscale(e, gain);
        if (g.phase) e = cmul(e, g.phase[i]);
        else if (g.lens) e = cmul(e, cmul(g.lens[x], g.lens[y]));
        const double yc = (double)(y - n / 2) * (2.0 / (double)n);
        const double n0 = pump_value(g, x, y, n, yc * yc);
        const double a = 1.0 + inten * g.invIsat;
        if (g.relax_exact) {
            const double nss = n0 / a;
            N[i] = nss + (nn - nss) * exp(-a * g.invT1);
        } else {
            N[i] = nn + (n0 - nn * a) * g.invT1;
        }
        E[i] = e;
        acc += e.x * e.x + e.y * e.y;
    }
    finish_mean<256>(acc, st, 1.0 / (double)P);
}

int gain_blocks64(int n) { return grid_for((size_t)n * n, 256, 1216); }

cudaError_t launch_gain64(int n, double2 *E, double *N, const GainParams<double> &g, const StatParams &st,
                          cudaStream_t s)
{
    k_gain64<<<gain_blocks64(n), 256, 0, s>>>(n, E, N, g, st);
    return cudaGetLastError();
}

// ---- set-up and readout -------------------------------------------------------

cudaError_t launch_tables64(int n, double alpha, double2 *tw, double2 *h, cudaStream_t s)
{
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    const int total = twiddle_count(logn);
    k_prop_table<double2><<<(n + 255) / 256, 256, 0, s>>>(n, alpha, h);
    if (total > 0) k_twiddles<double2><<<(total + 255) / 256, 256, 0, s>>>(logn, 0, total, tw);
    return cudaGetLastError();
}

cudaError_t launch_prop64(int n, double alpha, double2 *h, cudaStream_t s)
{
    k_prop_table<double2><<<(n + 255) / 256, 256, 0, s>>>(n, alpha, h);
    return cudaGetLastError();
}

cudaError_t launch_noise64(int n, unsigned long long seed, double amp, double2 *E, cudaStream_t s)
{
    k_noise<double2><<<grid_for((size_t)n * n, 256, 2048), 256, 0, s>>>(n, seed, amp, E);
    return cudaGetLastError();
}

cudaError_t launch_lens64(int n, double c, int edge, int taper, double2 *lens, cudaStream_t s)
{
    k_lens_table<double2><<<(n + 255) / 256, 256, 0, s>>>(n, c / 3.14159265358979323846, edge, taper, lens);
    return cudaGetLastError();
}

cudaError_t launch_phase64(int n, double c, int edge, int taper, const double *psi, double2 *phase,
                           cudaStream_t s)
{
    k_phase_table<double2><<<grid_for((size_t)n * n, 256, 2048), 256, 0, s>>>(n, c / 3.14159265358979323846, edge,
                                                                               taper, psi, phase);
    return cudaGetLastError();
}

cudaError_t launch_pattern64(int n, int kind, int q, int alt, double w, double env, double curv, double amp,
                             double2 *E, cudaStream_t s)
{
    k_pattern<double2><<<grid_for((size_t)n * n, 256, 2048), 256, 0, s>>>(n, kind, q, alt, w, env, curv, amp, E);
    return cudaGetLastError();
}

cudaError_t launch_pump64(int n, int kind, double g0, double order, double radius, const double *profile,
                          double *out, cudaStream_t s)
{
    k_pump<double><<<grid_for((size_t)n * n, 256, 2048), 256, 0, s>>>(n, kind, g0, order, radius, profile, out);
    return cudaGetLastError();
}

cudaError_t launch_power64(int n, const double2 *X, double *S, cudaStream_t s)
{
    const size_t P = (size_t)n * n;
    k_power<double2, double><<<grid_for(P, 256, 2048), 256, 0, s>>>(P, X, S);
    return cudaGetLastError();
}

cudaError_t launch_peak64(int n, int ring, const double *S, double *part_val, long long *part_idx,
                          unsigned int *count, PeakResult *out, cudaStream_t s)
{
    k_peak<double><<<peak_blocks(n), 256, 0, s>>>(n, ring, S, part_val, part_idx, count, out);
    return cudaGetLastError();
}

}  // namespace rtk

namespace rtk {

template <int LOGN> static cudaError_t prep64()
{
    constexpr int C = col_c64<LOGN>();
    cudaError_t e;
    if ((e = row_attr<double, LOGN, MODE_FWD>()) != cudaSuccess) return e;
    if ((e = row_attr<double, LOGN, MODE_INV>()) != cudaSuccess) return e;
    if ((e = col_attr<double, LOGN, C, MODE_FWD>()) != cudaSuccess) return e;
    return col_attr<double, LOGN, C, MODE_INV>();
}

cudaError_t prepare_bounce64(int logn) { RTK_LOGN_CASES(prep64) }

}  // namespace rtk
