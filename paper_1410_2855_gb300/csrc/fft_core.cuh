// Device-side building blocks of the split-step propagator: complex helpers,
// in-register DFTs of size 2..16 and a Stockham line FFT whose passes are
// exchanged through (padded) shared memory.
//
// A line of length N = 2^L is transformed by T = N/16 cooperating threads,
// each holding 16 elements in registers.  Passes are radix 16 (floor(L/4)
// of them) followed by one pass of radix 2, 4 or 8 when 4 does not divide L.
// Input and output are both in natural order with the same thread mapping:
// register slot s of thread t holds element t + T*s.  That is what lets a
// forward transform, a pointwise multiply in the Fourier domain and an
// inverse transform follow each other with no data movement in between
// (the diffraction operator of eq. limit_of_operators_renorm_final is
// diagonal in the Fourier basis).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rtk {

template <typename R> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <typename R> using cv = typename cvec<R>::type;

template <typename V> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <typename V>
__device__ __forceinline__ V cmk(typename real_of<V>::type a, typename real_of<V>::type b)
{
    V r;
    r.x = a;
    r.y = b;
    return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b)
{
    return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cscale(V a, typename real_of<V>::type s)
{
    return cmk<V>(a.x * s, a.y * s);
}

// exp(DIR * 2 pi i k / 16), k a constant after unrolling; multiples of 4
// are done with swaps and negations only.
template <int DIR, typename V>
__device__ __forceinline__ V rot16(V a, int k)
{
    using R = typename real_of<V>::type;
    k &= 15;
    if (k == 0) return a;
    if (k == 4) return DIR > 0 ? cmk<V>(-a.y, a.x) : cmk<V>(a.y, -a.x);
    if (k == 8) return cmk<V>(-a.x, -a.y);
    if (k == 12) return DIR > 0 ? cmk<V>(a.y, -a.x) : cmk<V>(-a.y, a.x);
    const R c8 = R(0.92387953251128675613), s8 = R(0.38268343236508977173), r2 = R(0.70710678118654752440);
    const R C[16] = {R(1), c8, r2, s8, R(0), -s8, -r2, -c8, R(-1), -c8, -r2, -s8, R(0), s8, r2, c8};
    const R S[16] = {R(0), s8, r2, c8, R(1), c8, r2, s8, R(0), -s8, -r2, -c8, R(-1), -c8, -r2, -s8};
    const R c = C[k], s = DIR > 0 ? S[k] : -S[k];
    return cmk<V>(a.x * c - a.y * s, a.x * s + a.y * c);
}

// In-register DFT of size RAD (2, 4, 8, 16): X[k] = sum_j x[j] exp(DIR 2 pi i jk/RAD).
// Radix-2 decimation in frequency, then a compile-time reordering (register
// renaming) back to natural order.
template <int RAD, int DIR, typename V>
__device__ __forceinline__ void dft(V (&v)[RAD])
{
#pragma unroll
    for (int half = RAD / 2; half >= 1; half >>= 1) {
#pragma unroll
        for (int s = 0; s < RAD; s += 2 * half) {
#pragma unroll
            for (int k = 0; k < half; ++k) {
                V a = v[s + k], b = v[s + k + half];
                v[s + k] = cadd(a, b);
                v[s + k + half] = rot16<DIR>(csub(a, b), k * (16 / (2 * half)));
            }
        }
    }
    V t[RAD];
#pragma unroll
    for (int k = 0; k < RAD; ++k) {
        int r = 0;
#pragma unroll
        for (int b = 1, kk = k; b < RAD; b <<= 1, kk >>= 1) r = (r << 1) | (kk & 1);
        t[k] = v[r];
    }
#pragma unroll
    for (int k = 0; k < RAD; ++k) v[k] = t[k];
}

// Shared-memory index with one pad element per 16: keeps the stride-16
// writes of the first pass and the unit-stride reads conflict-free.
__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + n / 16; }

template <int LOGN> struct Plan {
    static_assert(LOGN >= 4 && LOGN <= 12, "line length 16..4096");
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / 16;                 // threads per line
    static constexpr int P16 = LOGN / 4;             // radix-16 passes
    static constexpr int LASTLOG = LOGN % 4;         // log2 of the trailing radix (0: none)
    static constexpr int LASTR = 1 << LASTLOG;
};

// Twiddle exp(DIR * 2 pi i k / N) from the forward table tw[k] = exp(-2 pi i k / N).
template <int DIR, typename V>
__device__ __forceinline__ V twiddle(const V *__restrict__ tw, int k)
{
    V w = __ldg(tw + k);
    if (DIR > 0) w.y = -w.y;
    return w;
}

// One Stockham FFT of a line.  On entry v[s] = x[t + T s]; on exit
// v[s] = X[t + T s], X[k] = sum_j x[j] exp(DIR 2 pi i jk / N) (unnormalised).
// S(i) returns a reference to shared element i of this line (already padded
// by the caller's accessor); sync() is a barrier over every thread that
// shares the shared buffer.  Each exchange is barrier, write, barrier, read.
template <int LOGN, int DIR, typename V, typename SmemF, typename SyncF>
__device__ __forceinline__ void fft_line(V (&v)[16], int t, SmemF S, const V *__restrict__ tw, SyncF sync)
{
    using P = Plan<LOGN>;
    constexpr int N = P::N, T = P::T;
    // pass 0: radix 16, Ns = 1 (no twiddles)
    dft<16, DIR>(v);
    int Ns = 1;
#pragma unroll
    for (int p = 1; p < P::P16; ++p) {
        const int idxD = (t / Ns) * Ns * 16 + (t % Ns);
        sync();
#pragma unroll
        for (int r = 0; r < 16; ++r) S(idxD + r * Ns) = v[r];
        sync();
        Ns *= 16;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = S(t + r * T);
        const int e = (t % Ns) * (N / (16 * Ns));
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], twiddle<DIR>(tw, r * e));
        dft<16, DIR>(v);
    }
    if constexpr (P::LASTLOG > 0) {
        constexpr int RL = P::LASTR, NB = 16 / RL, NsL = N / RL;
        {
            const int idxD = (t / Ns) * Ns * 16 + (t % Ns);
            sync();
#pragma unroll
            for (int r = 0; r < 16; ++r) S(idxD + r * Ns) = v[r];
            sync();
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int j = t + i * T;
            V u[RL];
#pragma unroll
            for (int r = 0; r < RL; ++r) u[r] = S(j + r * NsL);
#pragma unroll
            for (int r = 1; r < RL; ++r) u[r] = cmul(u[r], twiddle<DIR>(tw, r * j));
            dft<RL, DIR>(u);
#pragma unroll
            for (int r = 0; r < RL; ++r) v[i + r * NB] = u[r];
        }
    }
}

}  // namespace rtk
