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
//
// Twiddles come from a pass-major table (see Plan::tw_size): for the pass
// with span Ns and radix R, entry [(r-1)*Ns + j] = exp(-2 pi i r j / (Ns R)),
// so the R-1 loads of a thread are each coalesced across the threads of a
// warp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// 1: bounds-checked build.  Every shared-memory access of the line FFT and
// the sweeps' row, column and item indices are checked; a violation stores
// RT_EBOUNDS (-7) in the kernel's error word and the access is skipped.
#ifndef RTK_CHECKED
#define RTK_CHECKED 0
#endif

namespace rtk {

constexpr int ERR_BOUNDS = -7;

// Checked builds: record a violation in *err (first writer wins) and report it.
__device__ __forceinline__ bool check_index(bool ok, int *err)
{
#if RTK_CHECKED
    if (!ok && err) atomicCAS(err, 0, ERR_BOUNDS);
    return ok;
#else
    (void)err;
    return true;
#endif
}

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
#ifndef RTK_PACKED_ADD
#define RTK_PACKED_ADD 1
#endif
#if RTK_PACKED_ADD
// FP32 complex add/subtract as one packed two-lane instruction each
// (sm_100 family); same IEEE round-to-nearest results as two scalar ops.
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b)
{
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
#endif
template <typename V> __device__ __forceinline__ V cmul(V a, V b)
{
    return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * b with every rounding spelled out: the same bits wherever it is
// inlined (no context-dependent contraction into fused multiply-adds).
__device__ __forceinline__ float2 cmul_rn(float2 a, float2 b)
{
    return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ double2 cmul_rn(double2 a, double2 b)
{
    return make_double2(__fma_rn(a.x, b.x, -__dmul_rn(a.y, b.y)), __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x)));
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b)
{
    return cmk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
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
__host__ __device__ constexpr int padi(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + n / 16; }

template <int LOGN> struct Plan {
    static_assert(LOGN >= 5 && LOGN <= 12, "line length 32..4096");
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / 16;                 // threads per line
    static constexpr int P16 = LOGN / 4;             // radix-16 passes
    static constexpr int LASTLOG = LOGN % 4;         // log2 of the trailing radix (0: none)
    static constexpr int LASTR = 1 << LASTLOG;
    // entries of the pass-major twiddle table
    static constexpr int tw_size()
    {
        int s = 0, Ns = 16;
        for (int p = 1; p < P16; ++p, Ns *= 16) s += 15 * Ns;
        if (LASTLOG) s += (LASTR - 1) * Ns;
        return s;
    }
};

// 1: a pass's twiddles are loaded before its exchange, so their latency
// overlaps the barrier and the shared-memory traffic.
#ifndef RTK_TW_PREFETCH
#define RTK_TW_PREFETCH 1
#endif

// Twiddle from the forward table (exp(-...)), conjugated for the inverse.
// TWS: the table is in shared memory (plain load) rather than global memory
// (read-only cache load).
template <int DIR, bool TWS = false, typename V>
__device__ __forceinline__ V twmul(V a, const V *__restrict__ tw, int k)
{
    const V w = TWS ? tw[k] : __ldg(tw + k);
    return DIR > 0 ? cmulc(a, w) : cmul(a, w);
}

// Element i of a padded line with element stride CS (1 for a row buffer; C
// for the [row][column] tile of the column sweep).
template <int CS, typename V> __device__ __forceinline__ V &sm_at(V *line, int i) { return line[padi(i) * CS]; }

// Exchange buffers of a line FFT.  With one buffer every exchange is
// barrier, write, barrier, read.  With two (ping-pong) an exchange is write,
// barrier, read into the buffer not used by the previous exchange: a thread
// can only write a buffer again after passing the barrier of the exchange in
// between, by which time every thread has finished reading it, so one
// barrier per exchange suffices.  `next` selects the buffer of the next
// exchange and carries across calls (forward then inverse transform).
template <typename V, bool PP> struct LineBufs {
    V *buf[2];
    int next;
    int *chk;  // error word of bounds-checked builds (may be null)
    __device__ __forceinline__ V *take()
    {
        V *b = buf[PP ? next : 0];
        if (PP) next ^= 1;
        return b;
    }
};

// A shared access at p is element padi(i) * CS of the line at base, 0 <= i < N
// (checked builds; always true otherwise).
template <int LOGN, int CS, typename V>
__device__ __forceinline__ bool sm_in(const V *base, const V *p, int *chk)
{
#if RTK_CHECKED
    const long long off = (long long)(p - base);
    return check_index(off >= 0 && off % CS == 0 && off / CS <= padi((1 << LOGN) - 1), chk);
#else
    (void)base, (void)p, (void)chk;
    return true;
#endif
}

// One Stockham FFT of a line.  On entry v[s] = x[t + T s]; on exit
// v[s] = X[t + T s], X[k] = sum_j x[j] exp(DIR 2 pi i jk / N) (unnormalised).
// `lb` holds this line's padded shared buffer(s) (element stride CS); sync()
// is a barrier over every thread that shares them.  Shared addresses are a
// per-thread base plus compile-time offsets: spans and T are multiples of 16
// wherever the pad arithmetic allows it.
// POST: multiply the result by post[k] (element k of the output line); the
// factors are loaded ahead of the last exchange when there is a trailing pass.
template <int LOGN, int DIR, int CS, bool PP, bool TWS = false, bool POST = false, typename V, typename SyncF>
__device__ __forceinline__ void fft_line(V (&v)[16], const int t, LineBufs<V, PP> &lb, const V *__restrict__ tw,
                                         SyncF sync, const V *__restrict__ post = nullptr)
{
    using P = Plan<LOGN>;
    constexpr int N = P::N, T = P::T;
    constexpr bool T16 = (T % 16) == 0;
    dft<16, DIR>(v);
    int off = 0;
#pragma unroll
    for (int p = 1; p < P::P16; ++p) {
        const int NsPrev = 1 << (4 * (p - 1));
        const int Ns = NsPrev * 16;
        V *line = lb.take();
        V *rd_base = line + padi(t) * CS;
        const V *twp = tw + off + (t & (Ns - 1));
        V wpre[RTK_TW_PREFETCH ? 15 : 1];
        if constexpr (RTK_TW_PREFETCH) {
#pragma unroll
            for (int r = 1; r < 16; ++r) wpre[r - 1] = TWS ? twp[(r - 1) * Ns] : __ldg(twp + (r - 1) * Ns);
        }
        if (!PP) sync();
        if (NsPrev == 1) {
            V *w = line + 17 * t * CS;
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (sm_in<LOGN, CS>(line, &w[r * CS], lb.chk)) w[r * CS] = v[r];
        } else {
            const int idxD = (t / NsPrev) * NsPrev * 16 + (t % NsPrev);
            V *w = line + padi(idxD) * CS;
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (sm_in<LOGN, CS>(line, &w[r * (17 * NsPrev / 16) * CS], lb.chk))
                    w[r * (17 * NsPrev / 16) * CS] = v[r];
        }
        sync();
        if constexpr (T16) {
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (sm_in<LOGN, CS>(line, &rd_base[r * (17 * T / 16) * CS], lb.chk))
                    v[r] = rd_base[r * (17 * T / 16) * CS];
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (sm_in<LOGN, CS>(line, &sm_at<CS>(line, t + r * T), lb.chk)) v[r] = sm_at<CS>(line, t + r * T);
        }
#pragma unroll
        for (int r = 1; r < 16; ++r) {
            if constexpr (RTK_TW_PREFETCH) v[r] = DIR > 0 ? cmulc(v[r], wpre[r - 1]) : cmul(v[r], wpre[r - 1]);
            else v[r] = twmul<DIR, TWS>(v[r], twp, (r - 1) * Ns);
        }
        off += 15 * Ns;
        dft<16, DIR>(v);
    }
    if constexpr (P::LASTLOG > 0) {
        constexpr int RL = P::LASTR, NB = 16 / RL, NsL = N / RL;
        constexpr int NsPrev = NsL / 16;
        V *line = lb.take();
        V *rd_base = line + padi(t) * CS;
        V pl[POST ? 16 : 1];
        if constexpr (POST) {
#pragma unroll
            for (int s = 0; s < 16; ++s) pl[s] = __ldg(post + t + s * T);
        }
        V wl[RTK_TW_PREFETCH ? NB * (RL - 1) : 1];
        if constexpr (RTK_TW_PREFETCH) {
#pragma unroll
            for (int i = 0; i < NB; ++i)
#pragma unroll
                for (int r = 1; r < RL; ++r) {
                    const V *q = tw + off + t + i * T + (r - 1) * NsL;
                    wl[i * (RL - 1) + r - 1] = TWS ? *q : __ldg(q);
                }
        }
        if (!PP) sync();
        if constexpr (NsPrev == 1) {
            V *w = line + 17 * t * CS;
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (sm_in<LOGN, CS>(line, &w[r * CS], lb.chk)) w[r * CS] = v[r];
        } else {
            const int idxD = (t / NsPrev) * NsPrev * 16 + (t % NsPrev);
            V *w = line + padi(idxD) * CS;
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (sm_in<LOGN, CS>(line, &w[r * (17 * NsPrev / 16) * CS], lb.chk))
                    w[r * (17 * NsPrev / 16) * CS] = v[r];
        }
        sync();
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int j = t + i * T;
            V *rb = T16 ? rd_base + i * (17 * T / 16) * CS : line + padi(j) * CS;
            V u[RL];
#pragma unroll
            for (int r = 0; r < RL; ++r)
                u[r] = sm_in<LOGN, CS>(line, &rb[r * (17 * NsL / 16) * CS], lb.chk) ? rb[r * (17 * NsL / 16) * CS]
                                                                                   : v[i];
            const V *twp = tw + off + j;
#pragma unroll
            for (int r = 1; r < RL; ++r) {
                if constexpr (RTK_TW_PREFETCH) {
                    const V w = wl[i * (RL - 1) + r - 1];
                    u[r] = DIR > 0 ? cmulc(u[r], w) : cmul(u[r], w);
                } else {
                    u[r] = twmul<DIR, TWS>(u[r], twp, (r - 1) * NsL);
                }
            }
            dft<RL, DIR>(u);
#pragma unroll
            for (int r = 0; r < RL; ++r) {
                if constexpr (POST) v[i + r * NB] = cmul_rn(u[r], pl[i + r * NB]);
                else v[i + r * NB] = u[r];
            }
        }
    } else if constexpr (POST) {
#pragma unroll
        for (int s = 0; s < 16; ++s) v[s] = cmul_rn(v[s], __ldg(post + t + s * T));
    }
}

}  // namespace rtk
