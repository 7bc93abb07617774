// Row and column sweeps of the bounce map.
//
// The 2-D propagator exp(-i pi alpha (mx^2 + my^2)) factors into
// h(mx) h(my), h(m) = exp(-i pi alpha m^2) / n, so diffraction over one
// iterate is a 1-D diffraction along y applied to every column followed by a
// 1-D diffraction along x applied to every row.  The fused FP32 bounce is
// therefore two sweeps over HBM:
//   column sweep: forward FFT, x h(my), inverse FFT            (8 B in, 8 B out)
//   row sweep:    forward FFT, x h(mx), inverse FFT, local map (12 B in, 12 B out)
// The local map (gain against the frozen inversion, mirror, absorbing edge,
// inversion relaxation) needs the field after both diffractions, so it is
// fused into the row sweep, where the inversion row is also contiguous.
#pragma once

#include <atomic>

#include "fft_core.cuh"
#include "rt_internal.h"

namespace rtk {

enum SweepMode { MODE_FWD = 0, MODE_INV = 1, MODE_DIFF = 2 };

// Lines per block of a row sweep: about 256 threads.
template <int LOGN> constexpr int row_lpc()
{
    return Plan<LOGN>::T >= 256 ? 1 : ((256 / Plan<LOGN>::T) > (1 << LOGN) ? (1 << LOGN) : 256 / Plan<LOGN>::T);
}
// Register budget per thread of the sweeps (build-time knob); the launch
// bounds ask the compiler for as many resident blocks as that budget allows.
#ifndef RTK_REGS
#define RTK_REGS 128
#endif
constexpr int min_blocks(int threads)
{
    return 65536 / (threads * RTK_REGS) > 0 ? 65536 / (threads * RTK_REGS) : 1;
}

// exp for the FP32 local map: ex2.approx of a prescaled argument (relative
// error ~2e-7 for the small arguments here); FP64 keeps the library exp.
__device__ __forceinline__ float fexp(float x) { return __expf(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
__device__ __forceinline__ double dpow(double x, double y) { return pow(x, y); }

// Unsaturated inversion N0 for the plain FP64 gain kernel (runtime pump kind).
template <typename R>
__device__ __forceinline__ R pump_value(const GainParams<R> &g, int x, int y, int n, R yc2)
{
    if (g.pump_kind == PUMP_UNIFORM) return g.g0;
    if (g.pump_kind == PUMP_ARRAY || g.int_half_order != 5) return __ldg(g.pump_tab + (size_t)y * n + x);
    const R xc = R(x - n / 2) * (R(2) / R(n));
    const R q = (xc * xc + yc2) * g.inv_rp2;
    const R q2 = q * q;
    return g.g0 * fexp(-(q2 * q2 * q));
}

// Block sum of v, then the last block to arrive sums the block partials in a
// fixed order and records the mean: deterministic, no atomics on doubles.
template <int NT>
__device__ __forceinline__ void finish_mean(double v, const StatParams &st, double inv_points)
{
    static_assert(NT % 32 == 0, "whole warps");
    __shared__ double red[NT / 32];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red[w];
        st.part[blockIdx.x] = s;
        __threadfence();
        is_last = (atomicAdd(st.count, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) s += __ldcg(st.part + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __syncthreads();
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < NT / 32; ++w) tot += red[w];
        const double mean = tot * inv_points;
        const long long b = *st.bounce;
        if (st.hist_cap > 0) st.hist[b % st.hist_cap] = mean;
        *st.last_mean = mean;
        *st.bounce = b + 1;
        if (!isfinite(mean)) atomicExch(st.err, -4);
        *st.count = 0u;
    }
}

// Row transforms (readout and the plain FP64 path).  Each group of T threads
// owns one row.  `in` and `out` may alias (in-place): a block reads all its
// rows before it writes any.
template <typename R, int LOGN, int MODE>
__global__ void __launch_bounds__(row_lpc<LOGN>() * Plan<LOGN>::T, min_blocks(row_lpc<LOGN>() * Plan<LOGN>::T))
k_row(const cv<R> *in, cv<R> *out, const cv<R> *__restrict__ tw, const cv<R> *__restrict__ h)
{
    using V = cv<R>;
    using P = Plan<LOGN>;
    constexpr int N = P::N, T = P::T, LPC = row_lpc<LOGN>(), LS = padded_len(N);
    extern __shared__ __align__(16) unsigned char smraw[];
    V *line = reinterpret_cast<V *>(smraw) + (threadIdx.x / T) * LS;
    const int t = threadIdx.x % T;
    const int row = blockIdx.x * LPC + threadIdx.x / T;
    auto sync = []() { __syncthreads(); };
    LineBufs<V, false> lb{{line, line}, 0};

    const V *src = in + (size_t)row * N + t;
    V v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = src[s * T];

    if constexpr (MODE == MODE_INV) {
        fft_line<LOGN, +1, 1>(v, t, lb, tw, sync);
    } else if constexpr (MODE == MODE_FWD) {
        fft_line<LOGN, -1, 1>(v, t, lb, tw, sync);
    } else {  // diffraction: the propagator is applied as the forward transform ends
        fft_line<LOGN, -1, 1, false, true>(v, t, lb, tw, sync, h);
        fft_line<LOGN, +1, 1>(v, t, lb, tw, sync);
    }
    V *dst = out + (size_t)row * N + t;
#pragma unroll
    for (int s = 0; s < 16; ++s) dst[s * T] = v[s];
}

// Column sweep on a tile of C adjacent columns.  Thread (c, t) with c the
// fast index, so a warp reads C*sizeof(V) contiguous bytes from each of
// 32/C rows.  Shared layout [padded row][c].  In place.
template <typename R, int LOGN, int C, int MODE>
__global__ void __launch_bounds__(C * Plan<LOGN>::T, min_blocks(C * Plan<LOGN>::T))
k_col(cv<R> *X, const cv<R> *__restrict__ tw, const cv<R> *__restrict__ h)
{
    using V = cv<R>;
    using P = Plan<LOGN>;
    constexpr int N = P::N, T = P::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int c = threadIdx.x % C, t = threadIdx.x / C;
    V *line = reinterpret_cast<V *>(smraw) + c;
    auto sync = []() { __syncthreads(); };
    LineBufs<V, false> lb{{line, line}, 0};
    V *col = X + (size_t)t * N + blockIdx.x * C + c;

    V v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = col[(size_t)s * T * N];
    if constexpr (MODE == MODE_INV) {
        fft_line<LOGN, +1, C>(v, t, lb, tw, sync);
    } else if constexpr (MODE == MODE_FWD) {
        fft_line<LOGN, -1, C>(v, t, lb, tw, sync);
    } else {  // diffraction, as in the persistent sweeps
        fft_line<LOGN, -1, C, false, true>(v, t, lb, tw, sync, h);
        fft_line<LOGN, +1, C>(v, t, lb, tw, sync);
    }
#pragma unroll
    for (int s = 0; s < 16; ++s) col[(size_t)s * T * N] = v[s];
}

template <typename R, int LOGN> constexpr size_t row_smem_bytes()
{
    return (size_t)row_lpc<LOGN>() * padded_len(1 << LOGN) * sizeof(cv<R>);
}
template <typename R, int LOGN, int C> constexpr size_t col_smem_bytes()
{
    return (size_t)C * padded_len(1 << LOGN) * sizeof(cv<R>);
}

// Opt a kernel into more than 48 KB of dynamic shared memory, once per
// kernel and device.  Called before a launch and before graph capture.
template <typename K>
inline cudaError_t ensure_smem(K kernel, size_t bytes, std::atomic<unsigned long long> &mask)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (mask.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) mask.fetch_or(bit);
    return e;
}

template <typename R, int LOGN, int MODE>
inline cudaError_t row_attr()
{
    static std::atomic<unsigned long long> mask{0};
    return ensure_smem(k_row<R, LOGN, MODE>, row_smem_bytes<R, LOGN>(), mask);
}

template <typename R, int LOGN, int C, int MODE>
inline cudaError_t col_attr()
{
    static std::atomic<unsigned long long> mask{0};
    return ensure_smem(k_col<R, LOGN, C, MODE>, col_smem_bytes<R, LOGN, C>(), mask);
}

}  // namespace rtk
