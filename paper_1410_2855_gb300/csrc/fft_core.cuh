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
        return;
    }
#endif
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

// Offset of pass p's block in the pass-major twiddle table (passes p >= 1;
// p = P16 is the trailing pass).
template <int LOGN> __host__ __device__ constexpr int tw_pass_off(int p)
{
    int s = 0, Ns = 16;
    for (int q = 1; q < p; ++q, Ns *= 16) s += 15 * Ns;
    return s;
}

// ---- table sources of the line FFT -------------------------------------------
// A line FFT needs, per thread, 15 twiddles for each radix-16 pass after the
// first, NB (RL - 1) for the trailing radix-RL pass, and (POST) the 16
// factors of its output elements.  TabGlobal loads them from global memory
// (read-only cache) where they are used; TabRegs holds them in registers for
// the life of a kernel, loaded once.
template <int LOGN, typename W> struct TabShape {
    using P = Plan<LOGN>;
    static constexpr int NP = P::P16 - 1;                                          // radix-16 passes with twiddles
    static constexpr int NL = P::LASTLOG ? (16 / P::LASTR) * (P::LASTR - 1) : 0;  // trailing-pass twiddles
};

template <int LOGN, typename W> struct TabGlobal {
    const W *__restrict__ tw;
    const W *__restrict__ post;
    __device__ __forceinline__ void pass(int p, int t, W (&w)[15]) const
    {
        const int Ns = 1 << (4 * p);
        const W *q = tw + tw_pass_off<LOGN>(p) + (t & (Ns - 1));
#pragma unroll
        for (int r = 1; r < 16; ++r) w[r - 1] = __ldg(q + (r - 1) * Ns);
    }
    template <int NL> __device__ __forceinline__ void last(int t, W (&w)[NL]) const
    {
        using P = Plan<LOGN>;
        constexpr int RL = P::LASTR, NB = 16 / RL, NsL = P::N / RL, T = P::T;
        const W *q = tw + tw_pass_off<LOGN>(P::P16) + t;
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int r = 1; r < RL; ++r) w[i * (RL - 1) + r - 1] = __ldg(q + i * T + (r - 1) * NsL);
    }
    __device__ __forceinline__ void postv(int t, W (&w)[16]) const
    {
#pragma unroll
        for (int s = 0; s < 16; ++s) w[s] = __ldg(post + t + s * Plan<LOGN>::T);
    }
};

template <int LOGN, typename W> struct TabRegs {
    using S = TabShape<LOGN, W>;
    W pw[S::NP > 0 ? S::NP : 1][15];
    W lw[S::NL > 0 ? S::NL : 1];
    W h[16];
    __device__ __forceinline__ void load_tw(const W *__restrict__ tw, int t)
    {
        const TabGlobal<LOGN, W> g{tw, nullptr};
#pragma unroll
        for (int p = 1; p <= S::NP; ++p) g.pass(p, t, pw[p - 1]);
        if constexpr (S::NL > 0) g.last(t, lw);
    }
    __device__ __forceinline__ void load_post(const W *__restrict__ post, int t)
    {
        const TabGlobal<LOGN, W> g{nullptr, post};
        g.postv(t, h);
    }
    __device__ __forceinline__ void pass(int p, int t, W (&w)[15]) const
    {
#pragma unroll
        for (int r = 0; r < 15; ++r) w[r] = pw[p - 1][r];
    }
    template <int NL> __device__ __forceinline__ void last(int t, W (&w)[NL]) const
    {
#pragma unroll
        for (int i = 0; i < NL; ++i) w[i] = lw[i];
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

// One Stockham FFT of a line.  On entry v[s] = x[t + T s]; on exit
// v[s] = X[t + T s], X[k] = sum_j x[j] exp(DIR 2 pi i jk / N) (unnormalised).
// `lb` holds this line's padded shared buffer(s) (element stride CS); sync()
// is a barrier over every thread that shares them.  Shared addresses are a
// per-thread base plus compile-time offsets: spans and T are multiples of 16
// wherever the pad arithmetic allows it.  A pass's twiddles are fetched
// before its exchange, so their latency overlaps the barrier.
// POST: multiply the result by factor k of `tab` (element k of the output
// line); the factors are fetched ahead of the last exchange when there is a
// trailing pass.  read_done() runs once every read of the last exchange is
// issued (by this thread): a caller can release the buffer there.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};
template <int LOGN, int DIR, int CS, bool PP, bool POST, typename V, typename Tab, typename SyncF,
          typename Hook = NoHook>
__device__ __forceinline__ void fft_line_t(V (&v)[16], const int t, LineBufs<V, PP> &lb, const Tab &tab, SyncF sync,
                                           Hook read_done = Hook{})
{
    using P = Plan<LOGN>;
    using W = typename table_of<V>::type;
    constexpr int N = P::N, T = P::T;
    constexpr bool T16 = (T % 16) == 0;
    dft<16, DIR>(v);
#pragma unroll
    for (int p = 1; p < P::P16; ++p) {
        const int NsPrev = 1 << (4 * (p - 1));
        V *line = lb.take();
        V *rd_base = line + padi(t) * CS;
        W wpre[15];
        tab.pass(p, t, wpre);
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
        if (P::LASTLOG == 0 && p == P::P16 - 1) read_done();
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = twm<DIR>(v[r], wpre[r - 1]);
        dft<16, DIR>(v);
    }
    if constexpr (P::LASTLOG > 0) {
        constexpr int RL = P::LASTR, NB = 16 / RL, NsL = N / RL;
        constexpr int NsPrev = NsL / 16;
        V *line = lb.take();
        V *rd_base = line + padi(t) * CS;
        W pl[POST ? 16 : 1];
        if constexpr (POST) tab.postv(t, pl);
        W wl[NB * (RL - 1)];
        tab.last(t, wl);
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
        // every read of the exchange first (the values' old copies in v are
        // dead once written), then the passes
        V ua[16];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int j = t + i * T;
            V *rb = T16 ? rd_base + i * (17 * T / 16) * CS : line + padi(j) * CS;
#pragma unroll
            for (int r = 0; r < RL; ++r)
                ua[i * RL + r] = sm_in<LOGN, CS>(line, &rb[r * (17 * NsL / 16) * CS], lb.chk)
                                     ? rb[r * (17 * NsL / 16) * CS]
                                     : v[i];
        }
        read_done();
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            V u[RL];
#pragma unroll
            for (int r = 0; r < RL; ++r) u[r] = ua[i * RL + r];
#pragma unroll
            for (int r = 1; r < RL; ++r) u[r] = twm<DIR>(u[r], wl[i * (RL - 1) + r - 1]);
            dft<RL, DIR>(u);
#pragma unroll
            for (int r = 0; r < RL; ++r) {
                if constexpr (POST) v[i + r * NB] = cmul_rn(u[r], pl[i + r * NB]);
                else v[i + r * NB] = u[r];
            }
        }
    } else if constexpr (POST) {
        W pl[16];
        tab.postv(t, pl);
#pragma unroll
        for (int s = 0; s < 16; ++s) v[s] = cmul_rn(v[s], pl[s]);
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
