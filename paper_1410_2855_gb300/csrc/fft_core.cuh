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

// a * (DIR i)^q: quarter turns are swaps and negations only.
template <int DIR, typename V> __device__ __forceinline__ V quarter(V a, int q)
{
    q &= 3;
    if (q == 0) return a;
    if (q == 2) return cmk<V>(-a.x, -a.y);
    return (q == 1) == (DIR > 0) ? cmk<V>(-a.y, a.x) : cmk<V>(a.y, -a.x);
}

#ifndef RTK_ROT_SMALL
#define RTK_ROT_SMALL 1
#endif

// Rotation by a small angle theta in the form a + a * ((cos theta - 1) + i sin theta).
// cos theta - 1 is far smaller than cos theta, so its rounded value carries
// about three more bits of cos theta; with it the rounded pair lies within
// about 1e-8 of the unit circle, where the rounded (cos, sin) pair of pi/8
// or pi/4 falls 3-6e-8 inside it.  Every pass of every transform applied
// that shortfall to the same paths, so an FP32 round trip lost about 2.5e-7
// of its power to it; in this form the loss drops to rounding noise.
// RTK_ROT_SMALL=0 builds the rounded (cos, sin) form for comparison.
template <typename R> struct Rot16Const;
template <> struct Rot16Const<float> {
    // cos - 1 and sin of pi/8 rounded to nearest; of pi/4, cos - 1 is the
    // float one ulp above the nearest, which puts the pair 8e-9 outside the
    // circle instead of 3.4e-8 inside it (found by exact search over
    // neighbouring floats).
    static constexpr float cm8 = -0.0761204659938812255859375f, s8 = 0.3826834261417388916015625f;
    static constexpr float cm4 = -0.2928932011127471923828125f, s4 = 0.707106769084930419921875f;
};
template <> struct Rot16Const<double> {
    static constexpr double cm8 = -0.07612046748871324387, s8 = 0.38268343236508977173;
    static constexpr double cm4 = -0.29289321881345247560, s4 = 0.70710678118654752440;
};

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// g * Re(a w) and g * Im(a w) for w = (1 + cm) + i s and a sign g = +-1
// known at compile time, each rounding explicit.  The sign rides on the FMA
// operands (rounding to nearest is symmetric under negation), so a quarter
// turn after the rotation costs no instruction.
template <typename V, typename R> __device__ __forceinline__ R rot_re(V a, R cm, R s, R g)
{
    return fma_rn(g * a.x, cm, fma_rn(-g * a.y, s, g * a.x));
}
template <typename V, typename R> __device__ __forceinline__ R rot_im(V a, R cm, R s, R g)
{
    return fma_rn(g * a.y, cm, fma_rn(g * a.x, s, g * a.y));
}

#if RTK_ROT_SMALL
// exp(DIR * 2 pi i k / 16), k a constant after unrolling.  k = 4q + j with
// j in {-1, 0, 1, 2}: a rotation by j pi/8, then q quarter turns.
template <int DIR, typename V>
__device__ __forceinline__ V rot16(V a, int k)
{
    using R = typename real_of<V>::type;
    using K = Rot16Const<R>;
    k &= 15;
    const int j = (k & 3) == 3 ? -1 : (k & 3);
    if (j == 0) return quarter<DIR>(a, k >> 2);
    const int q = ((k - j) >> 2) & 3;
    const R cm = j == 2 ? K::cm4 : K::cm8;
    const R s = (j < 0) == (DIR > 0) ? -(j == 2 ? K::s4 : K::s8) : (j == 2 ? K::s4 : K::s8);
    // (DIR i)^q (P + i Q): q = 0: (P, Q); 2: (-P, -Q); DIR i: (-Q, P); -DIR i: (Q, -P).
    if (q == 0) return cmk<V>(rot_re(a, cm, s, R(1)), rot_im(a, cm, s, R(1)));
    if (q == 2) return cmk<V>(rot_re(a, cm, s, R(-1)), rot_im(a, cm, s, R(-1)));
    if ((q == 1) == (DIR > 0)) return cmk<V>(rot_im(a, cm, s, R(-1)), rot_re(a, cm, s, R(1)));
    return cmk<V>(rot_im(a, cm, s, R(1)), rot_re(a, cm, s, R(-1)));
}
#else
// exp(DIR * 2 pi i k / 16) from the rounded (cos, sin) pairs.
template <int DIR, typename V>
__device__ __forceinline__ V rot16(V a, int k)
{
    using R = typename real_of<V>::type;
    k &= 15;
    if ((k & 3) == 0) return quarter<DIR>(a, k >> 2);
    const R c8 = R(0.92387953251128675613), s8 = R(0.38268343236508977173), r2 = R(0.70710678118654752440);
    const R C[16] = {R(1), c8, r2, s8, R(0), -s8, -r2, -c8, R(-1), -c8, -r2, -s8, R(0), s8, r2, c8};
    const R S[16] = {R(0), s8, r2, c8, R(1), c8, r2, s8, R(0), -s8, -r2, -c8, R(-1), -c8, -r2, -s8};
    const R c = C[k], s = DIR > 0 ? S[k] : -S[k];
    return cmk<V>(a.x * c - a.y * s, a.x * s + a.y * c);
}
#endif

#ifndef RTK_DFT44
#define RTK_DFT44 1
#endif

// In-place radix-4 DFT, outputs in natural order: y_k = sum_j a_j (DIR i)^(jk).
template <int DIR, typename V> __device__ __forceinline__ void dft4(V &a0, V &a1, V &a2, V &a3)
{
    const V t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
    const V t3 = DIR > 0 ? cmk<V>(-d.y, d.x) : cmk<V>(d.y, -d.x);  // DIR i (a1 - a3)
    a0 = cadd(t0, t2);
    a1 = cadd(t1, t3);
    a2 = csub(t0, t2);
    a3 = csub(t1, t3);
}

template <int RAD, int DIR, typename V> __device__ __forceinline__ void dft_dif(V (&v)[RAD]);

// In-register DFT of size RAD (2, 4, 8, 16): X[k] = sum_j x[j] exp(DIR 2 pi i jk/RAD).
// Size 16 is split 4 x 4 (j = 4 j1 + j2, k = k1 + 4 k2): radix-4 DFTs over
// j1, the factors exp(DIR 2 pi i j2 k1 / 16), radix-4 DFTs over j2; eight
// non-trivial rotations where four radix-2 stages need ten.  The other sizes
// are radix-2 decimation in frequency.  Both end with a compile-time
// reordering (register renaming) back to natural order.
template <int RAD, int DIR, typename V>
__device__ __forceinline__ void dft(V (&v)[RAD])
{
#if RTK_DFT44
    if constexpr (RAD == 16) {
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) dft4<DIR>(v[j2], v[4 + j2], v[8 + j2], v[12 + j2]);
#pragma unroll
        for (int j2 = 1; j2 < 4; ++j2)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) v[j2 + 4 * k1] = rot16<DIR>(v[j2 + 4 * k1], j2 * k1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) dft4<DIR>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
        V t[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = t[k];
    } else
#endif
    {
        dft_dif<RAD, DIR>(v);
    }
}

// Radix-2 decimation in frequency of size RAD, then the bit-reversal
// reordering (register renaming) back to natural order.
template <int RAD, int DIR, typename V>
__device__ __forceinline__ void dft_dif(V (&v)[RAD])
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

// Twiddle multiply of a pass, every rounding spelled out (the same bits in
// every kernel that runs the line FFT): a * w for the forward transform
// (DIR < 0; the table holds exp(-...)), a * conj(w) for the inverse.
template <int DIR> __device__ __forceinline__ float2 twm(float2 a, float2 w)
{
    return DIR > 0 ? make_float2(__fmaf_rn(a.x, w.x, __fmul_rn(a.y, w.y)), __fmaf_rn(a.y, w.x, -__fmul_rn(a.x, w.y)))
                   : cmul_rn(a, w);
}
template <int DIR> __device__ __forceinline__ double2 twm(double2 a, double2 w)
{
    return DIR > 0 ? make_double2(__fma_rn(a.x, w.x, __dmul_rn(a.y, w.y)), __fma_rn(a.y, w.x, -__dmul_rn(a.x, w.y)))
                   : cmul_rn(a, w);
}

// ---- two lines at once ----------------------------------------------------
// A thread of the column-pair sweep carries the same element of two adjacent
// columns.  They share every twiddle and propagator factor, and the pair
// moves through shared and global memory as one 16-byte access.  Each half
// goes through exactly the operations of a single line, so the results are
// bit-identical to transforming the columns one at a time.
struct __align__(16) cpair {
    float2 a, b;
};
__device__ __forceinline__ cpair cadd(cpair x, cpair y) { return {cadd(x.a, y.a), cadd(x.b, y.b)}; }
__device__ __forceinline__ cpair csub(cpair x, cpair y) { return {csub(x.a, y.a), csub(x.b, y.b)}; }
template <int DIR> __device__ __forceinline__ cpair rot16(cpair x, int k)
{
    return {rot16<DIR>(x.a, k), rot16<DIR>(x.b, k)};
}
template <int DIR> __device__ __forceinline__ void dft4(cpair &a0, cpair &a1, cpair &a2, cpair &a3)
{
    dft4<DIR>(a0.a, a1.a, a2.a, a3.a);
    dft4<DIR>(a0.b, a1.b, a2.b, a3.b);
}
template <int DIR> __device__ __forceinline__ cpair twm(cpair x, float2 w) { return {twm<DIR>(x.a, w), twm<DIR>(x.b, w)}; }
__device__ __forceinline__ cpair cmul_rn(cpair x, float2 w) { return {cmul_rn(x.a, w), cmul_rn(x.b, w)}; }

template <typename V> struct table_of { using type = V; };
template <> struct table_of<cpair> { using type = float2; };

// ---- radix sequences --------------------------------------------------------
// A line of 2^LOGN points is transformed in P16 = floor(LOGN/4) passes of
// radix 16 and, when 4 does not divide LOGN, one pass of radix 2^(LOGN mod 4).
// ORDER places that small pass: 0 last, 1 first, 2 second (after one radix-16
// pass).  Pass p has radix R_p and span Ns_p = R_0 ... R_(p-1); its butterfly
// j (0 <= j < N/R_p) combines x[j + k N/R_p], k < R_p, after multiplying
// input k by exp(-2 pi i (j mod Ns_p) k / (Ns_p R_p)), and writes output r to
// position (j / Ns_p) Ns_p R_p + (j mod Ns_p) + r Ns_p (Stockham autosort):
// after the last pass the line is in natural order.  A thread holds 16
// values and runs 16 / R_p butterflies j = t + i T of each pass.
template <int LOGN, int ORDER = 0> struct Seq {
    static constexpr int N = 1 << LOGN;
    static constexpr int P16 = LOGN / 4, LASTLOG = LOGN % 4;
    static constexpr int NP = P16 + (LASTLOG ? 1 : 0);  // passes
    static constexpr int SMALL = LASTLOG == 0 ? -1 : (ORDER == 1 ? 0 : (ORDER == 2 && P16 >= 2 ? 1 : P16));
    static constexpr int logr(int p) { return p == SMALL ? LASTLOG : 4; }
    static constexpr int radix(int p) { return 1 << logr(p); }
    static constexpr int span(int p)
    {
        int s = 1;
        for (int q = 0; q < p; ++q) s *= radix(q);
        return s;
    }
    // pass-major twiddle table: pass p >= 1 owns (R_p - 1) Ns_p entries,
    // entry (k - 1) Ns_p + j' = exp(-2 pi i j' k / (Ns_p R_p)); N - R_0 in all
    static constexpr int tw_off(int p)
    {
        int o = 0;
        for (int q = 1; q < p; ++q) o += (radix(q) - 1) * span(q);
        return o;
    }
    static constexpr int tw_size() { return tw_off(NP); }
};

// Radix orders a line of 2^logn points can use (ORDER < orders); one when
// every pass has radix 16 or there is a single radix-16 pass to move.
__host__ __device__ constexpr int radix_orders(int logn) { return logn % 4 == 0 ? 1 : (logn / 4 >= 2 ? 3 : 2); }

// ---- table sources of the line FFT -------------------------------------------
// A line FFT needs, per thread, the twiddles of every pass after the first
// (16 / R_p butterflies x (R_p - 1) of them, at most 15) and (POST) the 16
// factors of its output elements.  TabGlobal loads them from global memory
// (read-only cache) where they are used; TabRegs holds them in registers for
// the life of a kernel, loaded once.
// SHARED: the tables were staged in shared memory (plain loads there).
template <int LOGN, typename W, int ORDER = 0, bool SHARED = false> struct TabMem {
    // loads from shared memory are short: taken where they are used, after
    // the exchange, so they are not live across it beside the line's values
    static constexpr bool late = SHARED;
    const W *__restrict__ tw;
    const W *__restrict__ post;
    __device__ __forceinline__ W at(const W *q) const { return SHARED ? *q : __ldg(q); }
    // twiddle (k - 1) + i (R_p - 1) of pass p: input k of butterfly t + i T
    __device__ __forceinline__ void pass(int p, int t, W (&w)[15]) const
    {
        using S = Seq<LOGN, ORDER>;
        constexpr int T = Plan<LOGN>::T;
        const int R = S::radix(p), Ns = S::span(p), NB = 16 / R;
        const W *q = tw + S::tw_off(p);
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int k = 1; k < R; ++k) w[i * (R - 1) + k - 1] = at(q + (k - 1) * Ns + ((t + i * T) & (Ns - 1)));
    }
    __device__ __forceinline__ void postv(int t, W (&w)[16]) const
    {
#pragma unroll
        for (int s = 0; s < 16; ++s) w[s] = at(post + t + s * Plan<LOGN>::T);
    }
};
template <int LOGN, typename W, int ORDER = 0> using TabGlobal = TabMem<LOGN, W, ORDER, false>;

template <int LOGN, typename W, int ORDER = 0> struct TabRegs {
    static constexpr bool late = false;
    static constexpr int NP = Seq<LOGN, ORDER>::NP;
    W pw[NP > 1 ? NP - 1 : 1][15];
    W h[16];
    __device__ __forceinline__ void load_tw(const W *__restrict__ tw, int t)
    {
        const TabGlobal<LOGN, W, ORDER> g{tw, nullptr};
#pragma unroll
        for (int p = 1; p < NP; ++p) g.pass(p, t, pw[p - 1]);
    }
    __device__ __forceinline__ void load_post(const W *__restrict__ post, int t)
    {
        const TabGlobal<LOGN, W, ORDER> g{nullptr, post};
        g.postv(t, h);
    }
    __device__ __forceinline__ void pass(int p, int t, W (&w)[15]) const
    {
#pragma unroll
        for (int r = 0; r < 15; ++r) w[r] = pw[p - 1][r];
    }
    __device__ __forceinline__ void postv(int t, W (&w)[16]) const
    {
#pragma unroll
        for (int s = 0; s < 16; ++s) w[s] = h[s];
    }
};

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

// One Stockham FFT of a line, passes in the radix order ORDER (Seq).  On
// entry v[s] = x[t + T s]; on exit v[s] = X[t + T s],
// X[k] = sum_j x[j] exp(DIR 2 pi i jk / N) (unnormalised).  `lb` holds this
// line's padded shared buffer(s) (element stride CS); sync() is a barrier
// over every thread that shares them.  Between passes the outputs go to
// shared memory at their Stockham positions and every thread reads back the
// 16 elements t + T s: the inputs of its butterflies of the next pass.
// Shared addresses are a per-thread base plus compile-time offsets wherever
// the spans are multiples of 16.  A pass's twiddles are fetched before its
// exchange, so their latency overlaps the barrier.  POST: multiply the result
// by factor k of `tab` (element k of the output line), fetched ahead of the
// last exchange.  read_done() runs once this thread has issued every read of
// the last exchange: a caller can release the buffer there.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// The butterflies of pass p in registers: butterfly i of the thread takes
// slots i + k NB (k < R), optionally twiddled, and returns its outputs there.
template <int DIR, int R, typename V, typename W>
__device__ __forceinline__ void pass_butterflies(V (&v)[16], const W (&w)[15], bool twiddled)
{
    constexpr int NB = 16 / R;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        V u[R];
#pragma unroll
        for (int k = 0; k < R; ++k) u[k] = v[i + k * NB];
        if (twiddled) {
#pragma unroll
            for (int k = 1; k < R; ++k) u[k] = twm<DIR>(u[k], w[i * (R - 1) + k - 1]);
        }
        dft<R, DIR>(u);
#pragma unroll
        for (int k = 0; k < R; ++k) v[i + k * NB] = u[k];
    }
}

template <int LOGN, int DIR, int CS, bool PP, bool POST, int ORDER = 0, typename V, typename Tab, typename SyncF,
          typename Hook = NoHook>
__device__ __forceinline__ void fft_line_t(V (&v)[16], const int t, LineBufs<V, PP> &lb, const Tab &tab, SyncF sync,
                                           Hook read_done = Hook{})
{
    using S = Seq<LOGN, ORDER>;
    using W = typename table_of<V>::type;
    constexpr int T = Plan<LOGN>::T;
    constexpr bool T16 = (T % 16) == 0;
    constexpr bool LATE = Tab::late;
    W none[15];
    pass_butterflies<DIR, S::radix(0)>(v, none, false);
#pragma unroll
    for (int p = 1; p < S::NP; ++p) {
        const int R = S::radix(p);
        const int Rp = S::radix(p - 1), Nsp = S::span(p - 1), NBp = 16 / Rp;
        V *line = lb.take();
        V *rd_base = line + padi(t) * CS;
        W w[15];
        W pl[16];
        if constexpr (!LATE) {
            tab.pass(p, t, w);
            if constexpr (POST) {
                if (p == S::NP - 1) tab.postv(t, pl);
            }
        }
        if (!PP) sync();
        // outputs of pass p - 1: butterfly t + i T, output r at (j / Ns) Ns R + (j mod Ns) + r Ns
        if (Nsp == 1 && Rp == 16) {
            V *wr = line + 17 * t * CS;
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (sm_in<LOGN, CS>(line, &wr[r * CS], lb.chk)) wr[r * CS] = v[r];
        } else if (Nsp % 16 == 0 && Rp == 16) {
            const int idxD = (t / Nsp) * Nsp * 16 + (t % Nsp);
            V *wr = line + padi(idxD) * CS;
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (sm_in<LOGN, CS>(line, &wr[r * (17 * Nsp / 16) * CS], lb.chk)) wr[r * (17 * Nsp / 16) * CS] = v[r];
        } else {
#pragma unroll
            for (int i = 0; i < NBp; ++i) {
                const int j = t + i * T;
                const int base = (j / Nsp) * Nsp * Rp + (j % Nsp);
#pragma unroll
                for (int r = 0; r < Rp; ++r) {
                    V *q = &sm_at<CS>(line, base + r * Nsp);
                    if (sm_in<LOGN, CS>(line, q, lb.chk)) *q = v[i + r * NBp];
                }
            }
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
        if (p == S::NP - 1) read_done();
        if constexpr (LATE) tab.pass(p, t, w);
        if (R == 16) pass_butterflies<DIR, 16>(v, w, true);
        else if (R == 8) pass_butterflies<DIR, 8>(v, w, true);
        else if (R == 4) pass_butterflies<DIR, 4>(v, w, true);
        else pass_butterflies<DIR, 2>(v, w, true);
        if constexpr (POST) {
            if (p == S::NP - 1) {
                if constexpr (LATE) tab.postv(t, pl);
#pragma unroll
                for (int s2 = 0; s2 < 16; ++s2) v[s2] = cmul_rn(v[s2], pl[s2]);
            }
        }
    }
    if constexpr (POST && S::NP == 1) {
        W pl[16];
        tab.postv(t, pl);
#pragma unroll
        for (int s2 = 0; s2 < 16; ++s2) v[s2] = cmul_rn(v[s2], pl[s2]);
    }
}

// The line FFT with its tables read from global memory where they are used.
template <int LOGN, int DIR, int CS, bool PP = false, bool POST = false, typename V, typename SyncF>
__device__ __forceinline__ void fft_line(V (&v)[16], const int t, LineBufs<V, PP> &lb, const V *__restrict__ tw,
                                         SyncF sync, const V *__restrict__ post = nullptr)
{
    const TabGlobal<LOGN, V> tab{tw, post};
    fft_line_t<LOGN, DIR, CS, PP, POST>(v, t, lb, tab, sync);
}

}  // namespace rtk
