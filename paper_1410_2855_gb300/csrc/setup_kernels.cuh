// Set-up and readout kernels, generic over the storage precision.  All of
// their arithmetic is FP64 (tables, noise, pump); results are stored in the
// path's precision.
#pragma once

#include <climits>

#include "fft_core.cuh"
#include "rt_internal.h"

namespace rtk {

#ifndef RTK_UNIT_TABLES
#define RTK_UNIT_TABLES 1
#endif

// Stores the FP64 factor (re, im) of squared modulus mod2 in the path's
// precision.  For FP32, of the (at most four) pairs formed from the floats
// just below and above re and im, the one whose squared modulus is closest
// to mod2 (ties keep round-to-nearest); each component stays within one ulp.
// The tables are applied to the same paths every bounce, so a modulus that
// rounding left above or below 1 would scale those paths' power by the same
// factor each time; this keeps that factor within about 1e-8 of exact.
template <typename V> __device__ __forceinline__ V store_factor(double re, double im, double mod2)
{
    (void)mod2;
    return cmk<V>(re, im);
}
#if RTK_UNIT_TABLES
template <> __device__ __forceinline__ float2 store_factor<float2>(double re, double im, double mod2)
{
    const float rc[2] = {__double2float_rn(re), __double2float_rd(re) == __double2float_rn(re) ? __double2float_ru(re)
                                                                                               : __double2float_rd(re)};
    const float ic[2] = {__double2float_rn(im), __double2float_rd(im) == __double2float_rn(im) ? __double2float_ru(im)
                                                                                               : __double2float_rd(im)};
    float2 best = make_float2(rc[0], ic[0]);
    double err = fabs((double)rc[0] * rc[0] + (double)ic[0] * ic[0] - mod2);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const double e = fabs((double)rc[a] * rc[a] + (double)ic[b] * ic[b] - mod2);
            if (e < err) {
                err = e;
                best = make_float2(rc[a], ic[b]);
            }
        }
    return best;
}
#endif

// Per-axis propagator h[k] = exp(-i pi alpha m^2) / n, m the signed
// frequency of bin k (the 1-D factor of the transfer function of eq.
// limit_of_operators_renorm_final; the 1/n carries the inverse transform's
// normalisation for that axis).  alpha*m^2 is split into a rounded product
// and its exact FMA residual, the product is reduced modulo 2 exactly
// (fmod), and sincospi evaluates exp(-i pi t) on the reduced argument, so
// phases of thousands of radians keep full FP64 accuracy.
template <typename V>
__global__ void k_prop_table(int n, double alpha, V *h)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long m = k < n / 2 ? k : (long long)k - n;
    const double m2 = (double)(m * m);
    const double hi = alpha * m2;
    const double lo = fma(alpha, m2, -hi);
    const double t = fmod(hi, 2.0) + lo;
    double sp, cp;
    sincospi(t, &sp, &cp);
    const double inv = 1.0 / (double)n;
    h[k] = store_factor<V>(cp * inv, -sp * inv, inv * inv);
}

// Phase of the complex aperture (eq. complex_aperture2) as the library
// applies it: theta(x, y) = c (x^2 + y^2) + psi(x, y), factor exp(-i theta)
// (the conjugate of the printed exp(+i theta), matching the propagator's
// sign), with x_j = (j - n/2) / (n/2).  c / pi times x^2 (exact: x is a
// short dyadic fraction) is split into a rounded product and its FMA
// residual and reduced modulo 2 before sincospi, like the propagator.
__device__ __forceinline__ double lens_turns(double c_over_pi, double q)
{
    const double hi = c_over_pi * q;
    const double lo = fma(c_over_pi, q, -hi);
    return fmod(hi, 2.0) + lo;
}

// Aperture modulus along one axis: 0 in the absorbing band of `edge`
// pixels, then a sin^2 ramp over `taper` pixels, then 1.
__device__ __forceinline__ double aperture_modulus(int j, int n, int edge, int taper)
{
    if (j < edge || j >= n - edge) return 0.0;
    const int d = min(j - edge, n - 1 - edge - j);
    if (d >= taper) return 1.0;
    const double s = sinpi(0.5 * (double)(d + 1) / (double)(taper + 1));
    return s * s;
}

// Separable aperture factors lens[j] = A(j) exp(-i c x_j^2), one axis.
template <typename V>
__global__ void k_lens_table(int n, double c_over_pi, int edge, int taper, V *lens)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double x = (double)(j - n / 2) / (double)(n / 2);
    double sp, cp;
    sincospi(lens_turns(c_over_pi, x * x), &sp, &cp);
    const double a = aperture_modulus(j, n, edge, taper);
    lens[j] = store_factor<V>(a * cp, -a * sp, a * a);
}

// Full aperture factors A(x) A(y) exp(-i (c (x^2 + y^2) + psi[y n + x])); psi may be null.
template <typename V>
__global__ void k_phase_table(int n, double c_over_pi, int edge, int taper, const double *psi, V *phase)
{
    const size_t P = (size_t)n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)(i / n);
        const double xc = (double)(x - n / 2) / (double)(n / 2);
        const double yc = (double)(y - n / 2) / (double)(n / 2);
        double sl, cl;
        sincospi(lens_turns(c_over_pi, xc * xc + yc * yc), &sl, &cl);
        double sr = 0.0, cr = 1.0;
        if (psi) sincos(psi[i], &sr, &cr);
        const double a = aperture_modulus(x, n, edge, taper) * aperture_modulus(y, n, edge, taper);
        // exp(-i (a + b)) = (cos a cos b - sin a sin b) - i (sin a cos b + cos a sin b)
        phase[i] = store_factor<V>(a * (cl * cr - sl * sr), -a * (sl * cr + cl * sr), a * a);
    }
}

// Structured starting fields (rt_set_field_pattern): a Gaussian beam, or a
// q x q lattice of Gaussian beams or first-order vortices on the periodic
// window, times a Gaussian envelope and a phase front; FP64 arithmetic.
// Only lattice points within 10 widths can pass the cutoff, so each pixel
// visits the 2K+1 nearest indices per axis (all q when that covers them).
__device__ __forceinline__ double wrap_window(double u) { return u - 2.0 * floor(u / 2.0 + 0.5); }

template <typename V>
__global__ void k_pattern(int n, int kind, int q, int alt, double w, double env, double curv, double amp, V *E)
{
    const size_t P = (size_t)n * n;
    const double p = 2.0 / (double)q, inv2w2 = 1.0 / (2.0 * w * w);
    const int K = (int)ceil(10.0 * w / p) + 1;
    const bool all = 2 * K + 1 >= q;
    const int cnt = all ? q : 2 * K + 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)(i / n);
        const double xc = (double)(x - n / 2) / (double)(n / 2);
        const double yc = (double)(y - n / 2) / (double)(n / 2);
        const double r2 = xc * xc + yc * yc;
        double sr = 0.0, si = 0.0;
        if (kind == 0) {
            sr = exp(-r2 * inv2w2);
        } else {
            const int ax = all ? 0 : (int)floor(xc / p + 0.5) - K;
            const int by = all ? 0 : (int)floor(yc / p + 0.5) - K;
            for (int bj = 0; bj < cnt; ++bj) {
                const int b = ((by + bj) % q + q) % q;
                const double dy = wrap_window(yc - b * p);
                for (int aj = 0; aj < cnt; ++aj) {
                    const int a = ((ax + aj) % q + q) % q;
                    const double dx = wrap_window(xc - a * p);
                    const double e = (dx * dx + dy * dy) * inv2w2;
                    if (e > 50.0) continue;
                    const double sgn = (alt && ((a + b) & 1)) ? -1.0 : 1.0;
                    const double g = exp(-e);
                    if (kind == 1) {
                        sr += sgn * g;
                    } else {
                        sr += dx / w * g;
                        si += sgn * dy / w * g;
                    }
                }
            }
        }
        const double f = amp * (env > 0.0 ? exp(-r2 / (2.0 * env * env)) : 1.0);
        double sp, cp;
        sincos(-curv * r2, &sp, &cp);
        E[i] = cmk<V>(f * (cp * sr - sp * si), f * (cp * si + sp * sr));
    }
}

// Pass-major twiddle table of the line FFT of length 2^logn (layout in
// fft_core.cuh): for each pass after the first, with span Ns and radix R,
// entry (r-1)*Ns + j holds exp(-2 pi i r j / (Ns R)).  FP64 sincospi on the
// exact rational argument 2 r j / (Ns R).
// Radix sequence of a line of 2^logn points (the runtime twin of Seq in
// fft_core.cuh): passes of radix 16 and, when 4 does not divide logn, one of
// radix 2^(logn mod 4), placed last (order 0), first (1) or second (2).
__host__ __device__ inline int seq_passes(int logn) { return logn / 4 + (logn % 4 ? 1 : 0); }
__host__ __device__ inline int seq_small(int logn, int order)
{
    const int p16 = logn / 4;
    return logn % 4 == 0 ? -1 : (order == 1 ? 0 : (order == 2 && p16 >= 2 ? 1 : p16));
}
__host__ __device__ inline int seq_radix(int logn, int order, int p)
{
    return p == seq_small(logn, order) ? (1 << (logn % 4)) : 16;
}

// Pass-major twiddles of the sequence: pass p >= 1 (radix R, span Ns, the
// product of the radices before it) owns (R - 1) Ns entries, entry
// (k - 1) Ns + j = exp(-2 pi i j k / (Ns R)), computed in FP64 from the
// exact rational argument 2 j k / (Ns R).
template <typename V>
__global__ void k_twiddles(int logn, int order, int total, V *tw)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int base = 0, Ns = seq_radix(logn, order, 0), R = 16;
    for (int p = 1; p < seq_passes(logn); ++p) {
        R = seq_radix(logn, order, p);
        const int size = (R - 1) * Ns;
        if (e < base + size) break;
        base += size;
        Ns *= R;
    }
    const int local = e - base;
    const int r = local / Ns + 1, j = local % Ns;
    double s, c;
    sincospi(2.0 * (double)((long long)r * j) / ((double)Ns * R), &s, &c);
    tw[e] = store_factor<V>(c, -s, 1.0);
}

__host__ __device__ inline int twiddle_count(int logn, int order = 0)
{
    int s = 0, Ns = seq_radix(logn, order, 0);
    for (int p = 1; p < seq_passes(logn); ++p) {
        const int R = seq_radix(logn, order, p);
        s += (R - 1) * Ns;
        Ns *= R;
    }
    return s;
}

// splitmix64 (Steele, Lea & Flood 2014) as a counter-based stream: output c
// of the stream whose state starts at seed.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long c)
{
    unsigned long long z = seed + (c + 1ull) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Complex Gaussian noise by Box-Muller on two uniforms per point:
// E = amp/sqrt(2) * sqrt(-2 ln(1 - u1)) * exp(2 pi i u2).
template <typename V>
__global__ void k_noise(int n, unsigned long long seed, double amp, V *E)
{
    const size_t P = (size_t)n * n;
    const double sigma = amp * 0.70710678118654752440;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P; i += (size_t)gridDim.x * blockDim.x) {
        const double u1 = (double)(splitmix64_at(seed, 2ull * i) >> 11) * 0x1.0p-53;
        const double u2 = (double)(splitmix64_at(seed, 2ull * i + 1ull) >> 11) * 0x1.0p-53;
        const double rho = sigma * sqrt(-2.0 * log(1.0 - u1));
        double s, c;
        sincospi(2.0 * u2, &s, &c);
        E[i] = cmk<V>(rho * c, rho * s);
    }
}

// Unsaturated inversion N0 = g0 * P(x, y) in FP64.
template <typename R>
__global__ void k_pump(int n, int kind, double g0, double order, double radius, const double *profile, R *out)
{
    const size_t P = (size_t)n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P; i += (size_t)gridDim.x * blockDim.x) {
        double v;
        if (kind == PUMP_UNIFORM) {
            v = g0;
        } else if (kind == PUMP_ARRAY) {
            v = g0 * profile[i];
        } else {
            const int x = (int)(i % n), y = (int)(i / n);
            const double xc = (double)(x - n / 2) / (double)(n / 2);
            const double yc = (double)(y - n / 2) / (double)(n / 2);
            const double q = (xc * xc + yc * yc) / (radius * radius);
            v = g0 * exp(-(q > 0.0 ? pow(q, 0.5 * order) : 0.0));
        }
        out[i] = (R)v;
    }
}

template <typename V, typename R>
__global__ void k_power(size_t P, const V *X, R *S)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P; i += (size_t)gridDim.x * blockDim.x) {
        const V x = X[i];
        S[i] = x.x * x.x + x.y * x.y;
    }
}

// Folded-power argmax (see rt_spectrum_peak): bin k and its mirror -k form
// one peak filed under the smaller flat index; ties to the smaller index.
__device__ __forceinline__ bool peak_better(double v, long long k, double bv, long long bk)
{
    return v > bv || (v == bv && k < bk);
}

template <typename R>
__global__ void __launch_bounds__(256) k_peak(int n, int ring, const R *S, double *part_val, long long *part_idx,
                                              unsigned int *count, PeakResult *out)
{
    __shared__ double sv[256];
    __shared__ long long sk[256];
    __shared__ int is_last;
    const long long P = (long long)n * n;
    double bv = -1.0;
    long long bk = LLONG_MAX;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < P; k += (long long)gridDim.x * blockDim.x) {
        const int ky = (int)(k / n), kx = (int)(k % n);
        const long long kp = (long long)((n - ky) % n) * n + (n - kx) % n;
        if (kp < k) continue;
        const int mx = kx < n / 2 ? kx : kx - n, my = ky < n / 2 ? ky : ky - n;
        const int amx = mx < 0 ? -mx : mx, amy = my < 0 ? -my : my;
        if ((amx > amy ? amx : amy) < ring) continue;
        const double v = (kp == k) ? (double)S[k] : (double)S[k] + (double)S[kp];
        if (peak_better(v, k, bv, bk)) { bv = v; bk = k; }
    }
    sv[threadIdx.x] = bv;
    sk[threadIdx.x] = bk;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o && peak_better(sv[threadIdx.x + o], sk[threadIdx.x + o], sv[threadIdx.x], sk[threadIdx.x])) {
            sv[threadIdx.x] = sv[threadIdx.x + o];
            sk[threadIdx.x] = sk[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_val[blockIdx.x] = sv[0];
        part_idx[blockIdx.x] = sk[0];
        __threadfence();
        is_last = (atomicAdd(count, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    bv = -1.0;
    bk = LLONG_MAX;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 256) {
        const double v = __ldcg(part_val + i);
        const long long k = __ldcg(part_idx + i);
        if (peak_better(v, k, bv, bk)) { bv = v; bk = k; }
    }
    sv[threadIdx.x] = bv;
    sk[threadIdx.x] = bk;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o && peak_better(sv[threadIdx.x + o], sk[threadIdx.x + o], sv[threadIdx.x], sk[threadIdx.x])) {
            sv[threadIdx.x] = sv[threadIdx.x + o];
            sk[threadIdx.x] = sk[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out->value = sv[0];
        out->index = sk[0];
        *count = 0u;
    }
}

inline int grid_for(size_t P, int threads, int cap)
{
    size_t b = (P + threads - 1) / threads;
    return (int)(b < (size_t)cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace rtk
