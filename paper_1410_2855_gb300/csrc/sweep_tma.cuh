// Persistent, copy-engine-fed sweeps of the fused FP32 bounce.
//
// Each block loops over work items: a group of rows (row sweep) or a tile of
// adjacent columns (column sweep).  While it transforms item i, the copy
// engine (TMA) is already loading item i + gridDim.x into the other of two
// shared-memory stages, so global-memory latency is hidden behind the FFT
// arithmetic.  A stage uses the line FFT's padded stride: the copy engine
// fills the first n elements of each line densely, the first pass reads
// them, and from then on the same bytes serve as that line's exchange
// buffer.  Results leave registers straight to global memory.
//
// Batched forms take an array of per-resonator descriptors and spread the
// items of every resonator of one grid size over one persistent launch, so
// the last wave of a launch is a small fraction of its work.
//
// Every barrier wait is bounded in time; a timeout sets RT_ETIMEOUT in the
// error word, drains the copy still in flight and ends the block.
#pragma once

#include "sweep.cuh"
#include "tma.cuh"

namespace rtk {

constexpr int ERR_TIMEOUT = -5;

// Ping-pong exchange buffers in the persistent sweeps (one barrier per
// exchange instead of two, for one more padded line buffer per line).
#ifndef RTK_ROW_PP
#define RTK_ROW_PP 0
#endif
#ifndef RTK_COL_PP
#define RTK_COL_PP 1
#endif

// TAB: the stage also carries the rows' N0 (pump table) values.
template <int LOGN, int LPC, bool PP, bool TAB = false> struct RowStage {
    static constexpr int N = 1 << LOGN;
    static constexpr size_t e_bytes = round128((size_t)LPC * padded_len(N) * sizeof(float2));
    static constexpr size_t n_bytes = round128((size_t)LPC * N * sizeof(float));
    static constexpr size_t t_bytes = TAB ? n_bytes : 0;
    static constexpr size_t stage = e_bytes + n_bytes + t_bytes;
    static constexpr size_t extra = PP ? e_bytes : 0;          // second exchange buffer
    static constexpr size_t total = 128 + 2 * stage + extra;   // two mbarriers, two stages, extra buffer
};
template <int LOGN, int LPC> using RowPlan = RowStage<LOGN, LPC, RTK_ROW_PP>;

template <int LOGN, int C, bool PP> struct ColStage {
    static constexpr int N = 1 << LOGN;
    static constexpr int BR = N < 256 ? N : 256;  // rows per tensor-map box (box dims are <= 256)
    static constexpr int NBOX = N / BR;
    static constexpr size_t stage = round128((size_t)C * padded_len(N) * sizeof(float2));
    static constexpr size_t total = 128 + (PP ? 3 : 2) * stage;
};
template <int LOGN, int C> using ColPlan = ColStage<LOGN, C, RTK_COL_PP>;

// Blocks per SM that the shared-memory plan allows (at most 8).
constexpr int smem_blocks(size_t bytes)
{
    return (int)((228 * 1024) / (bytes + 1024)) > 8 ? 8
           : ((int)((228 * 1024) / (bytes + 1024)) > 0 ? (int)((228 * 1024) / (bytes + 1024)) : 1);
}

// Resident blocks asked of the compiler for the column sweep: what shared
// memory allows, but never fewer than RTK_COL_REGS registers per thread (the
// column FFT spills below ~96).
#ifndef RTK_COL_REGS
#define RTK_COL_REGS 128
#endif
constexpr int col_min_blocks(int threads, size_t bytes)
{
    return smem_blocks(bytes) < 65536 / (threads * RTK_COL_REGS)
               ? smem_blocks(bytes)
               : (65536 / (threads * RTK_COL_REGS) > 0 ? 65536 / (threads * RTK_COL_REGS) : 1);
}

// A batched resonator still has bounces to do.  Its counter only changes at
// the end of a row sweep, after every item of that resonator in the launch
// has been processed, so all items of a launch see the same answer.
__device__ __forceinline__ bool res_active(const BatchRes &R)
{
    return __ldcg(R.st.bounce) < R.target;
}

// First item >= i on this block's stride (items congruent to blockIdx.x
// modulo gridDim.x) that belongs to an active resonator; a finished
// resonator is skipped in one step.  `per` items per resonator.
__device__ __forceinline__ int next_active_item(const BatchRes *__restrict__ res, int per, int nitems, int i)
{
    const int grid = gridDim.x, b = blockIdx.x;
    while (i < nitems) {
        const int r = i / per;
        if (res_active(res[r])) return i;
        const int first = (r + 1) * per;
        i = first + (int)((((long long)b - first) % grid + grid) % grid);
    }
    return nitems;
}

// Contiguous share of a launch's items for this block: block b runs items
// [lo, end), q or q + 1 of them for q = nitems / grid (a persistent grid
// never exceeds its items, so q >= 1), and block_of(i) is the block that runs
// item i.  A row sweep over many resonators uses it so that a block keeps one
// running mean-intensity sum per resonator over many items and files it once.
struct BlockRange {
    int q, rem, lo, end;
    __device__ __forceinline__ explicit BlockRange(int nitems)
    {
        const int grid = (int)gridDim.x, b = (int)blockIdx.x;
        q = nitems / grid;
        rem = nitems % grid;
        lo = b * q + (b < rem ? b : rem);
        end = lo + q + (b < rem ? 1 : 0);
    }
    __device__ __forceinline__ int block_of(int i) const
    {
        const int cut = rem * (q + 1);
        return i < cut ? i / (q + 1) : rem + (i - cut) / q;
    }
};

// ---- shared pieces ----------------------------------------------------------

// Bounded wait on a stage barrier; on a timeout the block drains the copy
// still in flight, records RT_ETIMEOUT and reports true (leave the loop).
__device__ __forceinline__ bool stage_wait_or_abort(uint64_t *bar, int it, bool next_in_flight, int *err)
{
    const bool late = !mbar_wait(&bar[it & 1], (uint32_t)((it >> 1) & 1));
    if (__syncthreads_or(late)) {
        if (threadIdx.x == 0) {
            atomicExch(err, ERR_TIMEOUT);
            if (next_in_flight) mbar_wait(&bar[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1));
        }
        return true;
    }
    return false;
}

__device__ __forceinline__ void init_stage_barriers(uint64_t *bar)
{
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
}

// Order-10 super-Gaussian pump g0 exp(-q^5), q = (x^2 + y^2) / r_p^2, with
// yq = y^2 / r_p^2 precomputed per row; roundings spelled out as above (the
// general forms; the plain form leaves contraction to the compiler, which
// is the faster code and is only ever compared with itself).
__device__ __forceinline__ float sg10_pump(float g0, float xc, float yq, float inv_rp2)
{
    const float q = __fmaf_rn(__fmul_rn(xc, xc), inv_rp2, yq);
    const float q2 = __fmul_rn(q, q);
    return __fmul_rn(g0, fexp(-__fmul_rn(__fmul_rn(q2, q2), q)));
}

// Local map of one row held in registers (slot s = column t + T s):
// gain against the frozen inversion, mirror, absorbing edge, inversion
// relaxation.  The general forms also apply the complex aperture D (smooth
// taper, curved mirror, roughness) from g.phase when set, else from the
// separable g.lens (one of them must be set): FEAT_TABLE with the Euler
// inversion step, FEAT_TABLE_EXACT with the exact one.  PE_RUNTIME takes the
// pump evaluation from pe_rt.  Returns sum |E_new|^2 over the thread's 16
// elements.
template <int LOGN, int PE, bool STAGED_N0 = false, int FEAT = FEAT_PLAIN>
__device__ __forceinline__ float row_local_map(float2 (&v)[16], int t, int row, const float *nrow, float2 *erow,
                                               float *ngl, const GainParams<float> &g, const float *n0row = nullptr,
                                               int pe_rt = PE_SG10)
{
    constexpr int N = 1 << LOGN, T = Plan<LOGN>::T;
    const float step = 2.0f / (float)N;
    const float xc0 = (float)(t - N / 2) * step;
    const float yc = (float)(row - N / 2) * step;
    const float yq = FEAT != FEAT_PLAIN ? __fmul_rn(__fmul_rn(yc, yc), g.inv_rp2) : yc * yc * g.inv_rp2;
    const bool row_in = row >= g.edge && row < N - g.edge;
    // Aperture factor of element x: drow * dtab[x] (sqrtR folded into drow).
    const float2 *dtab = nullptr;
    float2 drow = make_float2(g.sqrtR, 0.0f);
    if constexpr (FEAT != FEAT_PLAIN) {
        if (g.phase) {
            dtab = g.phase + (size_t)row * N + t;
        } else {
            dtab = g.lens + t;
            drow = cscale(__ldg(g.lens + row), g.sqrtR);
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int si = 0; si < 16; ++si) {
        const int x = t + si * T;
        const float nn = nrow[si * T];
        float2 e = v[si];
        const float inten = FEAT != FEAT_PLAIN ? __fmaf_rn(e.x, e.x, __fmul_rn(e.y, e.y)) : e.x * e.x + e.y * e.y;
        const bool inside = row_in && x >= g.edge && x < N - g.edge;
        if constexpr (FEAT != FEAT_PLAIN) {
            const float gain = inside ? fexp(__fmul_rn(0.5f, nn)) : 0.0f;
            e = cmul_rn(e, cmul_rn(drow, __ldg(dtab + si * T)));
            e = make_float2(__fmul_rn(e.x, gain), __fmul_rn(e.y, gain));
        } else {
            e = cscale(e, inside ? g.sqrtR * fexp(0.5f * nn) : 0.0f);
        }
        float n0;
        if constexpr (PE == PE_RUNTIME) {
            if (pe_rt == PE_UNIFORM) {
                n0 = g.g0;
            } else if (pe_rt == PE_TABLE) {
                n0 = __ldg(g.pump_tab + (size_t)row * N + x);
            } else {
                n0 = sg10_pump(g.g0, __fmaf_rn((float)(si * T), step, xc0), yq, g.inv_rp2);
            }
        } else if constexpr (PE == PE_UNIFORM) {
            n0 = g.g0;
        } else if constexpr (PE == PE_TABLE && STAGED_N0) {
            n0 = n0row[si * T];
        } else if constexpr (PE == PE_TABLE) {
            n0 = __ldg(g.pump_tab + (size_t)row * N + x);
        } else if constexpr (FEAT != FEAT_PLAIN) {
            n0 = sg10_pump(g.g0, __fmaf_rn((float)(si * T), step, xc0), yq, g.inv_rp2);
        } else {
            const float xc = xc0 + (float)(si * T) * step;
            const float q = xc * xc * g.inv_rp2 + yq;
            const float q2 = q * q;
            n0 = g.g0 * fexp(-(q2 * q2 * q));
        }
        if constexpr (FEAT == FEAT_TABLE_EXACT) {
            const float a = __fmaf_rn(inten, g.invIsat, 1.0f);
            const float nss = __fdiv_rn(n0, a);
            ngl[si * T] = __fmaf_rn(__fsub_rn(nn, nss), fexp(-__fmul_rn(a, g.invT1)), nss);
        } else if constexpr (FEAT == FEAT_TABLE) {
            const float a = __fmaf_rn(inten, g.invIsat, 1.0f);
            ngl[si * T] = __fmaf_rn(__fmaf_rn(-nn, a, n0), g.invT1, nn);
        } else {
            ngl[si * T] = nn + (n0 - nn * (1.0f + inten * g.invIsat)) * g.invT1;
        }
        erow[si * T] = e;
        if constexpr (FEAT != FEAT_PLAIN) acc = __fmaf_rn(e.x, e.x, __fmaf_rn(e.y, e.y, acc));
        else acc += e.x * e.x + e.y * e.y;
    }
    return acc;
}

// Forward FFT, x h, inverse FFT of the line held in v (exchanges in lb).
// The propagator factors are fetched ahead of the forward transform's last
// exchange and applied as its outputs come out.
template <int LOGN, int CS, bool PP, typename SyncF>
__device__ __forceinline__ void diffract_line(float2 (&v)[16], int t, LineBufs<float2, PP> &lb,
                                              const float2 *__restrict__ tw, const float2 *__restrict__ h,
                                              SyncF sync)
{
    fft_line<LOGN, -1, CS, PP, true>(v, t, lb, tw, sync, h);
    fft_line<LOGN, +1, CS>(v, t, lb, tw, sync);
}

// The same with the tables in registers (TabRegs: twiddles, and the
// propagator factors in tab.h).
template <int LOGN, int CS, bool PP, typename V, typename SyncF>
__device__ __forceinline__ void diffract_line_regs(V (&v)[16], int t, LineBufs<V, PP> &lb,
                                                   const TabRegs<LOGN, float2> &tab, SyncF sync)
{
    fft_line_t<LOGN, -1, CS, PP, true>(v, t, lb, tab, sync);
    fft_line_t<LOGN, +1, CS, PP, false>(v, t, lb, tab, sync);
}

// Per-resonator mean intensity of a batched row sweep.  A block keeps one
// running sum per resonator while it works through that resonator's items
// and, when it moves on, stores the block sum in slot k of the resonator's
// partials; the last of the `arrivals` blocks to do so adds the partials up
// in slot order and records the mean (deterministic for a given grid).
template <int NT>
__device__ __forceinline__ void res_finish(double v, const StatParams &st, int k, int arrivals, double inv_points)
{
    static_assert(NT % 32 == 0, "whole warps");
    __shared__ double red[NT / 32];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red[w];
        st.part[k] = s;
        __threadfence();
        is_last = (atomicAdd(st.count, 1u) == (unsigned)arrivals - 1u);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < arrivals; i += NT) s += __ldcg(st.part + i);
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

// ---- single resonator -------------------------------------------------------

// Row sweep: LPC rows per group, T = n/16 threads per row.  With a pump
// table (PE_TABLE) the rows' N0 values are staged by the copy engine too.
template <int LOGN, int LPC, int PE, int FEAT = FEAT_PLAIN, bool PP = RTK_ROW_PP>
__global__ void __launch_bounds__(LPC * Plan<LOGN>::T, smem_blocks(RowStage<LOGN, LPC, PP, PE == PE_TABLE>::total))
k_row_tma(float2 *E, float *Nv, const float2 *__restrict__ tw, const float2 *__restrict__ h, GainParams<float> g,
          StatParams st, int ngroups)
{
    using P = Plan<LOGN>;
    constexpr bool TAB = PE == PE_TABLE;
    using L = RowStage<LOGN, LPC, PP, TAB>;
    constexpr int N = P::N, T = P::T, NT = LPC * T, LS = padded_len(N);
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const int lig = threadIdx.x / T, t = threadIdx.x % T;
    auto stage_e = [](int s) { return reinterpret_cast<float2 *>(sm + 128 + s * L::stage); };
    auto stage_n = [](int s) { return reinterpret_cast<float *>(sm + 128 + s * L::stage + L::e_bytes); };
    auto stage_t = [](int s) {
        return reinterpret_cast<float *>(sm + 128 + s * L::stage + L::e_bytes + L::n_bytes);
    };
    auto sync = []() { __syncthreads(); };
    auto issue = [&](int s, int grp) {
        mbar_arrive_expect_tx(&bar[s], (uint32_t)(LPC * N * (sizeof(float2) + (TAB ? 2 : 1) * sizeof(float))));
        for (int l = 0; l < LPC; ++l) {
            const size_t row = (size_t)grp * LPC + l;
            bulk_g2s(stage_e(s) + l * LS, E + row * N, N * sizeof(float2), &bar[s]);
            bulk_g2s(stage_n(s) + l * N, Nv + row * N, N * sizeof(float), &bar[s]);
            if constexpr (TAB) bulk_g2s(stage_t(s) + l * N, g.pump_tab + row * N, N * sizeof(float), &bar[s]);
        }
    };

    init_stage_barriers(bar);
    int grp = blockIdx.x;
    if (threadIdx.x == 0 && grp < ngroups) issue(0, grp);
    double dacc = 0.0;
    for (int it = 0; grp < ngroups; ++it, grp += gridDim.x) {
        const int s = it & 1;
        const int nxt = grp + (int)gridDim.x;
        if (threadIdx.x == 0 && nxt < ngroups) {
            fence_proxy_async_smem();
            issue(s ^ 1, nxt);
        }
        if (stage_wait_or_abort(bar, it, nxt < ngroups, st.err)) break;
        const int row = grp * LPC + lig;
        float2 *line = stage_e(s) + lig * LS;
        float2 v[16];
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = line[t + si * T];
        // With ping-pong the first exchange goes to the extra buffer, so the
        // dense stage is only overwritten after every thread has read it.
        float2 *extra = reinterpret_cast<float2 *>(sm + 128 + 2 * L::stage) + lig * LS;
        LineBufs<float2, PP> lb{{PP ? extra : line, line}, 0, st.err};
        diffract_line<LOGN, 1>(v, t, lb, tw, h, sync);
        dacc += (double)row_local_map<LOGN, PE, TAB, FEAT>(v, t, row, stage_n(s) + lig * N + t, E + (size_t)row * N + t,
                                                     Nv + (size_t)row * N + t, g, stage_t(s) + lig * N + t);
        __syncthreads();  // stage s fully consumed before it is refilled
    }
    finish_mean<NT>(dacc, st, 1.0 / ((double)N * (double)N));
}

// Column sweep: tiles of C adjacent columns, loaded as NBOX tensor-map boxes
// of BR rows x C complex columns.  Thread (c, t), c fastest.
template <int LOGN, int C, bool PP = RTK_COL_PP>
__global__ void __launch_bounds__(C * Plan<LOGN>::T,
                                  col_min_blocks(C * Plan<LOGN>::T, ColStage<LOGN, C, PP>::total))
k_col_tma(float2 *E, const float2 *__restrict__ tw, const float2 *__restrict__ h,
          const __grid_constant__ CUtensorMap tmap, int ntiles, int *err)
{
    using P = Plan<LOGN>;
    using L = ColStage<LOGN, C, PP>;
    constexpr int N = P::N, T = P::T;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const int c = threadIdx.x % C, t = threadIdx.x / C;
    auto stage = [](int s) { return reinterpret_cast<float2 *>(sm + 128 + s * L::stage); };
    auto sync = []() { __syncthreads(); };
    auto issue = [&](int s, int tile) {
        mbar_arrive_expect_tx(&bar[s], (uint32_t)(N * C * sizeof(float2)));
        for (int b = 0; b < L::NBOX; ++b)
            tma_load_2d(stage(s) + b * L::BR * C, &tmap, 2 * tile * C, b * L::BR, &bar[s]);
    };

    init_stage_barriers(bar);
    int tile = blockIdx.x;
    if (threadIdx.x == 0 && tile < ntiles) issue(0, tile);
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const int s = it & 1;
        const int nxt = tile + (int)gridDim.x;
        if (threadIdx.x == 0 && nxt < ntiles) {
            fence_proxy_async_smem();
            issue(s ^ 1, nxt);
        }
        if (stage_wait_or_abort(bar, it, nxt < ntiles, err)) break;
        float2 *base = stage(s);
        float2 v[16];
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = base[(t + si * T) * C + c];
        LineBufs<float2, PP> lb{{PP ? stage(2) + c : base + c, base + c}, 0, err};
        diffract_line<LOGN, C>(v, t, lb, tw, h, sync);
        float2 *col = E + (size_t)t * N + tile * C + c;
#pragma unroll
        for (int si = 0; si < 16; ++si) col[(size_t)si * T * N] = v[si];
        __syncthreads();  // stage s fully consumed before it is refilled
    }
}

// Column-pair sweep: the column sweep with each thread carrying two adjacent
// columns of the tile (C/2 pairs per row, thread (c2, t), c2 fastest) and
// every table in registers.  The twiddles are loaded once per block and the
// propagator factors once per resonator, so no table load remains inside the
// tile loop; the pairs move through shared and global memory as 16-byte
// accesses, half the instructions of one column at a time.  The arithmetic
// of each column is exactly that of k_col_tma (bit-identical fields).
#ifndef RTK_PAIR_REGS
#define RTK_PAIR_REGS 192
#endif
constexpr int pair_min_blocks(int threads, size_t bytes)
{
    return smem_blocks(bytes) < 65536 / (threads * RTK_PAIR_REGS)
               ? smem_blocks(bytes)
               : (65536 / (threads * RTK_PAIR_REGS) > 0 ? 65536 / (threads * RTK_PAIR_REGS) : 1);
}

template <int LOGN, int C, bool PP = RTK_COL_PP>
__global__ void __launch_bounds__((C / 2) * Plan<LOGN>::T,
                                  pair_min_blocks((C / 2) * Plan<LOGN>::T, ColStage<LOGN, C, PP>::total))
k_col_pair(float2 *E, const float2 *__restrict__ tw, const float2 *__restrict__ h,
           const __grid_constant__ CUtensorMap tmap, int ntiles, int *err)
{
    static_assert(C >= 2 && C % 2 == 0, "whole column pairs");
    using P = Plan<LOGN>;
    using L = ColStage<LOGN, C, PP>;
    constexpr int N = P::N, T = P::T, CP = C / 2;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const int c2 = threadIdx.x % CP, t = threadIdx.x / CP;
    auto stage = [](int s) { return reinterpret_cast<cpair *>(sm + 128 + s * L::stage); };
    auto sync = []() { __syncthreads(); };
    auto issue = [&](int s, int tile) {
        mbar_arrive_expect_tx(&bar[s], (uint32_t)(N * C * sizeof(float2)));
        for (int b = 0; b < L::NBOX; ++b)
            tma_load_2d(stage(s) + b * L::BR * CP, &tmap, 2 * tile * C, b * L::BR, &bar[s]);
    };

    init_stage_barriers(bar);
    int tile = blockIdx.x;
    if (threadIdx.x == 0 && tile < ntiles) issue(0, tile);
    TabRegs<LOGN, float2> tab;
    tab.load_tw(tw, t);
    tab.load_post(h, t);
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const int s = it & 1;
        const int nxt = tile + (int)gridDim.x;
        if (threadIdx.x == 0 && nxt < ntiles) {
            fence_proxy_async_smem();
            issue(s ^ 1, nxt);
        }
        if (stage_wait_or_abort(bar, it, nxt < ntiles, err)) break;
        cpair *base = stage(s);
        cpair v[16];
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = base[(t + si * T) * CP + c2];
        LineBufs<cpair, PP> lb{{PP ? stage(2) + c2 : base + c2, base + c2}, 0, err};
        diffract_line_regs<LOGN, CP>(v, t, lb, tab, sync);
        cpair *col = reinterpret_cast<cpair *>(E + (size_t)t * N + tile * C) + c2;
#pragma unroll
        for (int si = 0; si < 16; ++si) col[(size_t)si * T * (N / 2)] = v[si];
        __syncthreads();  // stage s fully consumed before it is refilled
    }
}

// One-stage column-pair sweep: one shared stage per block that serves as the
// copy engine's destination and then, in place, as the exchange buffer (two
// barriers per exchange), and the tables read from global memory where they
// are used.  That keeps a block within ~70 KB of shared memory and 128
// registers per thread, so two or more blocks share an SM: one block's
// exchanges overlap another's arithmetic, and each block's next copy is
// issued as soon as its last exchange has been read (before the inverse
// transform's last pass and the store).  Bit-identical to k_col_pair.
// 1: the handle's one-stage column sweep stages its twiddle and propagator
// tables in shared memory at n >= 2048 where two blocks still fit an SM with
// them, instead of the L1 cache, where one table load in three missed (ncu,
// two blocks per SM).  Measured on GB300 (graph-timed sweep): 2048^2
// with 4-column tiles 24.7 against 25.6 us, 2-column tiles 29.7 against 33.7;
// at 1024^2 and below, where a block runs about one tile, the copy costs more
// than it saves (7.6 against 7.1 us).
#ifndef RTK_COL_TABS
#define RTK_COL_TABS 1
#endif
template <int LOGN, int C> struct ColStage1 {
    static constexpr int N = 1 << LOGN;
    static constexpr int BR = N < 256 ? N : 256;
    static constexpr int NBOX = N / BR;
    static constexpr size_t stage = round128((size_t)C * padded_len(N) * sizeof(float2));
    static constexpr size_t total = 128 + stage;
    // tables: twiddles of any order (at most N entries) and the N propagator factors
    static constexpr size_t tabs = round128((size_t)2 * N * sizeof(float2));
    static constexpr bool tabs_fit = RTK_COL_TABS && LOGN >= 11 && 2 * (total + tabs + 1024) <= 228 * 1024;
    static constexpr size_t total_tabs = tabs_fit ? total + tabs : total;
};
#ifndef RTK_PAIR1_REGS
#define RTK_PAIR1_REGS 128
#endif
constexpr int pair1_min_blocks(int threads, size_t bytes)
{
    return smem_blocks(bytes) < 65536 / (threads * RTK_PAIR1_REGS)
               ? smem_blocks(bytes)
               : (65536 / (threads * RTK_PAIR1_REGS) > 0 ? 65536 / (threads * RTK_PAIR1_REGS) : 1);
}

// Issue the copy of the next item into the (single) stage once every thread
// has read its last exchange: a barrier, then thread 0 orders the shared
// writes before the copy engine's (proxy fence) and starts the copy.
template <typename IssueF> struct IssueAfterReads {
    IssueF issue;
    int next;
    bool valid;
    __device__ __forceinline__ void operator()() const
    {
        __syncthreads();
        if (threadIdx.x == 0 && valid) {
            fence_proxy_async_smem();
            issue(next);
        }
    }
};

// ORDER: radix order of the column transforms (Seq); tw is that order's table.
// When they fit (ColStage1::tabs_fit) the tables are staged in shared memory
// behind the stage once per block.
template <int LOGN, int C, int ORDER = 0>
__global__ void __launch_bounds__((C / 2) * Plan<LOGN>::T,
                                  pair1_min_blocks((C / 2) * Plan<LOGN>::T, ColStage1<LOGN, C>::total_tabs))
k_col_pair1(float2 *E, const float2 *__restrict__ tw, const float2 *__restrict__ h,
            const __grid_constant__ CUtensorMap tmap, int ntiles, int *err)
{
    static_assert(C >= 2 && C % 2 == 0, "whole column pairs");
    using P = Plan<LOGN>;
    using L = ColStage1<LOGN, C>;
    constexpr int N = P::N, T = P::T, CP = C / 2;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    cpair *base = reinterpret_cast<cpair *>(sm + 128);
    const int c2 = threadIdx.x % CP, t = threadIdx.x / CP;
    auto sync = []() { __syncthreads(); };
    auto issue = [&](int tile) {
        mbar_arrive_expect_tx(&bar[0], (uint32_t)(N * C * sizeof(float2)));
        for (int b = 0; b < L::NBOX; ++b) tma_load_2d(base + b * L::BR * CP, &tmap, 2 * tile * C, b * L::BR, &bar[0]);
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        fence_barrier_init();
    }
    __syncthreads();
    int tile = blockIdx.x;
    if (threadIdx.x == 0 && tile < ntiles) issue(tile);
    constexpr bool TABS = L::tabs_fit;
    const float2 *stw = tw, *sh = h;
    if constexpr (TABS) {
        float2 *t2 = reinterpret_cast<float2 *>(sm + L::total);
        constexpr int NTW = Seq<LOGN, ORDER>::tw_size();
        for (int i = threadIdx.x; i < NTW; i += blockDim.x) t2[i] = __ldg(tw + i);
        for (int i = threadIdx.x; i < N; i += blockDim.x) t2[N + i] = __ldg(h + i);
        __syncthreads();
        stw = t2;
        sh = t2 + N;
    }
    const TabMem<LOGN, float2, ORDER, TABS> tab{stw, sh};
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const int nxt = tile + (int)gridDim.x;
        const bool late = !mbar_wait(&bar[0], (uint32_t)(it & 1));
        if (__syncthreads_or(late)) {  // the copy in flight is this one: nothing else to drain
            if (threadIdx.x == 0) atomicExch(err, ERR_TIMEOUT);
            break;
        }
        cpair v[16];
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = base[(t + si * T) * CP + c2];
        LineBufs<cpair, false> lb{{base + c2, base + c2}, 0, err};
        fft_line_t<LOGN, -1, CP, false, true, ORDER>(v, t, lb, tab, sync);
        const IssueAfterReads<decltype(issue)> next{issue, nxt, nxt < ntiles};
        fft_line_t<LOGN, +1, CP, false, false, ORDER>(v, t, lb, tab, sync, next);
        cpair *col = reinterpret_cast<cpair *>(E + (size_t)t * N + tile * C) + c2;
#pragma unroll
        for (int si = 0; si < 16; ++si) col[(size_t)si * T * (N / 2)] = v[si];
    }
}

// ---- batches of resonators of one grid size -----------------------------------

// Row sweep over nres resonators: item i is row group i % G of resonator
// i / G, G = n / LPC.  The pump evaluation and the aperture phase are chosen
// per resonator.
template <int LOGN, int LPC, bool PP = RTK_ROW_PP>
__global__ void __launch_bounds__(LPC * Plan<LOGN>::T, smem_blocks(RowStage<LOGN, LPC, PP>::total))
k_row_tma_batch(const BatchRes *__restrict__ res, int nres, const float2 *__restrict__ tw, int *err)
{
    using P = Plan<LOGN>;
    using L = RowStage<LOGN, LPC, PP>;
    constexpr int N = P::N, T = P::T, NT = LPC * T, LS = padded_len(N), G = N / LPC;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const int lig = threadIdx.x / T, t = threadIdx.x % T;
    const int nitems = nres * G;
    auto stage_e = [](int s) { return reinterpret_cast<float2 *>(sm + 128 + s * L::stage); };
    auto stage_n = [](int s) { return reinterpret_cast<float *>(sm + 128 + s * L::stage + L::e_bytes); };
    auto sync = []() { __syncthreads(); };
    // Items of resonators that are done are skipped: no copy is issued for
    // them and no barrier phase is consumed, so the stage parity follows the
    // count of issued copies (`used`), not the item index.
    auto issue = [&](int s, int item) {
        const BatchRes &R = res[item / G];
        const int grp = item % G;
        mbar_arrive_expect_tx(&bar[s], (uint32_t)(LPC * N * (sizeof(float2) + sizeof(float))));
        for (int l = 0; l < LPC; ++l) {
            const size_t row = (size_t)grp * LPC + l;
            bulk_g2s(stage_e(s) + l * LS, R.E + row * N, N * sizeof(float2), &bar[s]);
            bulk_g2s(stage_n(s) + l * N, R.N + row * N, N * sizeof(float), &bar[s]);
        }
    };
    // Block b runs the contiguous items [lo, end) (BlockRange), so it stays
    // with one resonator for many items and files one partial per resonator
    // it touches: the blocks that touch resonator r are block_of(rG) ..
    // block_of(rG + G - 1), and block b files under slot b - block_of(rG).
    // A finished resonator is skipped in one step.
    const BlockRange br(nitems);
    const int end = br.end;
    auto next_active = [&](int i) {
        while (i < end) {
            const int r = i / G;
            if (res_active(res[r])) return i;
            i = (r + 1) * G;
        }
        return end;
    };
    int item = next_active(br.lo);

    init_stage_barriers(bar);
    if (threadIdx.x == 0 && item < end) issue(0, item);
    double dacc = 0.0;
    for (int it = 0; item < end; ++it) {
        const int s = it & 1;
        const int nxt = next_active(item + 1);
        if (threadIdx.x == 0 && nxt < end) {
            fence_proxy_async_smem();
            issue(s ^ 1, nxt);
        }
        if (stage_wait_or_abort(bar, it, nxt < end, err)) break;
        const int r = item / G;
        const BatchRes &R = res[r];
        const int grp = item % G;
        const int row = grp * LPC + lig;
        float2 *line = stage_e(s) + lig * LS;
        float2 v[16];
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = line[t + si * T];
        float2 *extra = reinterpret_cast<float2 *>(sm + 128 + 2 * L::stage) + lig * LS;
        LineBufs<float2, PP> lb{{PP ? extra : line, line}, 0, err};
        diffract_line<LOGN, 1>(v, t, lb, tw, R.h, sync);
        const GainParams<float> g = R.g;
        const float *nrow = stage_n(s) + lig * N + t;
        float2 *erow = R.E + (size_t)row * N + t;
        float *ngl = R.N + (size_t)row * N + t;
        float acc;
        const int feat = feature_form(g);
        if (feat == FEAT_TABLE_EXACT) {
            acc = row_local_map<LOGN, PE_RUNTIME, false, FEAT_TABLE_EXACT>(v, t, row, nrow, erow, ngl, g, nullptr, R.pe);
        } else if (feat == FEAT_TABLE) {
            acc = row_local_map<LOGN, PE_RUNTIME, false, FEAT_TABLE>(v, t, row, nrow, erow, ngl, g, nullptr, R.pe);
        } else {
            if (R.pe == PE_UNIFORM) acc = row_local_map<LOGN, PE_UNIFORM>(v, t, row, nrow, erow, ngl, g);
            else if (R.pe == PE_TABLE) acc = row_local_map<LOGN, PE_TABLE>(v, t, row, nrow, erow, ngl, g);
            else acc = row_local_map<LOGN, PE_SG10>(v, t, row, nrow, erow, ngl, g);
        }
        dacc += (double)acc;
        __syncthreads();  // stage s fully consumed before it is refilled
        if (nxt >= end || nxt / G != r) {
            const int first = br.block_of(r * G);
            const int k = (int)blockIdx.x - first, arrivals = br.block_of(r * G + G - 1) - first + 1;
            res_finish<NT>(dacc, R.st, k, arrivals, 1.0 / ((double)N * (double)N));
            dacc = 0.0;
        }
        item = nxt;
    }
}

// Column sweep over nres resonators: item i is tile i % (n/C) of resonator
// i / (n/C), loaded through that resonator's tensor map.
template <int LOGN, int C, bool PP = RTK_COL_PP>
__global__ void __launch_bounds__(C * Plan<LOGN>::T,
                                  col_min_blocks(C * Plan<LOGN>::T, ColStage<LOGN, C, PP>::total))
k_col_tma_batch(const BatchRes *__restrict__ res, int nres, const float2 *__restrict__ tw, int *err)
{
    using P = Plan<LOGN>;
    using L = ColStage<LOGN, C, PP>;
    constexpr int N = P::N, T = P::T, TILES = N / C;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const int c = threadIdx.x % C, t = threadIdx.x / C;
    const int nitems = nres * TILES;
    auto stage = [](int s) { return reinterpret_cast<float2 *>(sm + 128 + s * L::stage); };
    auto sync = []() { __syncthreads(); };
    auto issue = [&](int s, int item) {
        const CUtensorMap *map = res[item / TILES].tmap;
        const int tile = item % TILES;
        mbar_arrive_expect_tx(&bar[s], (uint32_t)(N * C * sizeof(float2)));
        for (int b = 0; b < L::NBOX; ++b)
            tma_load_2d(stage(s) + b * L::BR * C, map, 2 * tile * C, b * L::BR, &bar[s]);
    };

    auto next_active = [&](int i) { return next_active_item(res, TILES, nitems, i); };

    init_stage_barriers(bar);
    int item = next_active(blockIdx.x);
    if (threadIdx.x == 0 && item < nitems) issue(0, item);
    for (int it = 0; item < nitems; ++it) {
        const int s = it & 1;
        const int nxt = next_active(item + (int)gridDim.x);
        if (threadIdx.x == 0 && nxt < nitems) {
            fence_proxy_async_smem();
            issue(s ^ 1, nxt);
        }
        if (stage_wait_or_abort(bar, it, nxt < nitems, err)) break;
        const BatchRes &R = res[item / TILES];
        const int tile = item % TILES;
        float2 *base = stage(s);
        float2 v[16];
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = base[(t + si * T) * C + c];
        LineBufs<float2, PP> lb{{PP ? stage(2) + c : base + c, base + c}, 0, err};
        diffract_line<LOGN, C>(v, t, lb, tw, R.h, sync);
        float2 *col = R.E + (size_t)t * N + tile * C + c;
#pragma unroll
        for (int si = 0; si < 16; ++si) col[(size_t)si * T * N] = v[si];
        __syncthreads();  // stage s fully consumed before it is refilled
        item = nxt;
    }
}

// Column-pair sweep over nres resonators of one grid size (as
// k_col_tma_batch; twiddles in registers for the whole launch, propagator
// factors reloaded whenever the block moves to another resonator).
template <int LOGN, int C, bool PP = RTK_COL_PP>
__global__ void __launch_bounds__((C / 2) * Plan<LOGN>::T,
                                  pair_min_blocks((C / 2) * Plan<LOGN>::T, ColStage<LOGN, C, PP>::total))
k_col_pair_batch(const BatchRes *__restrict__ res, int nres, const float2 *__restrict__ tw, int *err)
{
    static_assert(C >= 2 && C % 2 == 0, "whole column pairs");
    using P = Plan<LOGN>;
    using L = ColStage<LOGN, C, PP>;
    constexpr int N = P::N, T = P::T, CP = C / 2, TILES = N / C;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const int c2 = threadIdx.x % CP, t = threadIdx.x / CP;
    const int nitems = nres * TILES;
    auto stage = [](int s) { return reinterpret_cast<cpair *>(sm + 128 + s * L::stage); };
    auto sync = []() { __syncthreads(); };
    auto issue = [&](int s, int item) {
        const CUtensorMap *map = res[item / TILES].tmap;
        const int tile = item % TILES;
        mbar_arrive_expect_tx(&bar[s], (uint32_t)(N * C * sizeof(float2)));
        for (int b = 0; b < L::NBOX; ++b)
            tma_load_2d(stage(s) + b * L::BR * CP, map, 2 * tile * C, b * L::BR, &bar[s]);
    };
    auto next_active = [&](int i) { return next_active_item(res, TILES, nitems, i); };

    init_stage_barriers(bar);
    int item = next_active(blockIdx.x);
    if (threadIdx.x == 0 && item < nitems) issue(0, item);
    TabRegs<LOGN, float2> tab;
    tab.load_tw(tw, t);
    int cur = -1;  // resonator whose propagator factors are in tab.h
    for (int it = 0; item < nitems; ++it) {
        const int s = it & 1;
        const int nxt = next_active(item + (int)gridDim.x);
        if (threadIdx.x == 0 && nxt < nitems) {
            fence_proxy_async_smem();
            issue(s ^ 1, nxt);
        }
        const int r = item / TILES;
        const BatchRes &R = res[r];
        if (r != cur) {
            tab.load_post(R.h, t);
            cur = r;
        }
        if (stage_wait_or_abort(bar, it, nxt < nitems, err)) break;
        const int tile = item % TILES;
        cpair *base = stage(s);
        cpair v[16];
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = base[(t + si * T) * CP + c2];
        LineBufs<cpair, PP> lb{{PP ? stage(2) + c2 : base + c2, base + c2}, 0, err};
        diffract_line_regs<LOGN, CP>(v, t, lb, tab, sync);
        cpair *col = reinterpret_cast<cpair *>(R.E + (size_t)t * N + tile * C) + c2;
#pragma unroll
        for (int si = 0; si < 16; ++si) col[(size_t)si * T * (N / 2)] = v[si];
        __syncthreads();  // stage s fully consumed before it is refilled
        item = nxt;
    }
}

// One-stage column-pair sweep over nres resonators of one grid size.
template <int LOGN, int C, int ORDER = 0>
__global__ void __launch_bounds__((C / 2) * Plan<LOGN>::T,
                                  pair1_min_blocks((C / 2) * Plan<LOGN>::T, ColStage1<LOGN, C>::total))
k_col_pair1_batch(const BatchRes *__restrict__ res, int nres, const float2 *__restrict__ tw, int *err)
{
    static_assert(C >= 2 && C % 2 == 0, "whole column pairs");
    using P = Plan<LOGN>;
    using L = ColStage1<LOGN, C>;
    constexpr int N = P::N, T = P::T, CP = C / 2, TILES = N / C;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    cpair *base = reinterpret_cast<cpair *>(sm + 128);
    const int c2 = threadIdx.x % CP, t = threadIdx.x / CP;
    const int nitems = nres * TILES;
    auto sync = []() { __syncthreads(); };
    auto issue = [&](int item) {
        const CUtensorMap *map = res[item / TILES].tmap;
        const int tile = item % TILES;
        mbar_arrive_expect_tx(&bar[0], (uint32_t)(N * C * sizeof(float2)));
        for (int b = 0; b < L::NBOX; ++b) tma_load_2d(base + b * L::BR * CP, map, 2 * tile * C, b * L::BR, &bar[0]);
    };
    auto next_active = [&](int i) { return next_active_item(res, TILES, nitems, i); };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        fence_barrier_init();
    }
    __syncthreads();
    int item = next_active(blockIdx.x);
    if (threadIdx.x == 0 && item < nitems) issue(item);
    for (int it = 0; item < nitems; ++it) {
        const int nxt = next_active(item + (int)gridDim.x);
        const BatchRes &R = res[item / TILES];
        const int tile = item % TILES;
        const bool late = !mbar_wait(&bar[0], (uint32_t)(it & 1));
        if (__syncthreads_or(late)) {
            if (threadIdx.x == 0) atomicExch(err, ERR_TIMEOUT);
            break;
        }
        const TabGlobal<LOGN, float2, ORDER> tab{tw, R.h};
        cpair v[16];
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = base[(t + si * T) * CP + c2];
        LineBufs<cpair, false> lb{{base + c2, base + c2}, 0, err};
        fft_line_t<LOGN, -1, CP, false, true, ORDER>(v, t, lb, tab, sync);
        const IssueAfterReads<decltype(issue)> next{issue, nxt, nxt < nitems};
        fft_line_t<LOGN, +1, CP, false, false, ORDER>(v, t, lb, tab, sync, next);
        cpair *col = reinterpret_cast<cpair *>(R.E + (size_t)t * N + tile * C) + c2;
#pragma unroll
        for (int si = 0; si < 16; ++si) col[(size_t)si * T * (N / 2)] = v[si];
        item = nxt;
    }
}

}  // namespace rtk
