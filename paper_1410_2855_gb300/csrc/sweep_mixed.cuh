// One persistent launch per sweep for resonators of uneven grid sizes.
//
// Every work item holds the same number of points whatever the resonator's
// side n: a column item is a tile of C(n) = 8192/n adjacent columns (8192
// points, 256 threads carrying column pairs), a row item is a group of
// LPC(n) = 2048/n rows (2048 points, 128 threads).  The items of all size
// classes form one index space, class after class; a block walks it with the
// grid stride and, per item, dispatches on log2 n into the device function of
// that size, so one class's tail is filled by the items of the others.  The
// per-item arithmetic is that of the per-class batched kernels (same bits).
#pragma once

#include "sweep_tma.cuh"

namespace rtk {

constexpr int kMixColPoints = 8192;  // points of a column item
constexpr int kMixRowPoints = 2048;  // points of a row item
constexpr int kMixColThreads = 256;
constexpr int kMixRowThreads = 128;
constexpr int kMixMinLog = 7, kMixMaxLog = 11;  // sides 128 .. 2048
constexpr int kMixMaxClasses = kMixMaxLog - kMixMinLog + 1;

__host__ __device__ constexpr int mix_col_width(int logn) { return kMixColPoints >> logn; }
__host__ __device__ constexpr int mix_row_lines(int logn) { return kMixRowPoints >> logn; }

// Column-item stage: C(n) columns of n padded rows, the same bytes for every n.
constexpr size_t kMixColStage = round128((size_t)kMixColPoints / 16 * 17 * sizeof(float2));
constexpr size_t kMixColSmem = 128 + kMixColStage;
// Row-item stage: LPC(n) padded rows of the field and LPC(n) rows of the inversion.
constexpr size_t kMixRowE = round128((size_t)kMixRowPoints / 16 * 17 * sizeof(float2));
constexpr size_t kMixRowN = round128((size_t)kMixRowPoints * sizeof(float));
constexpr size_t kMixRowStage = kMixRowE + kMixRowN;
constexpr size_t kMixRowSmem = 128 + 2 * kMixRowStage;

struct MixClass {
    const BatchRes *res;  // descriptors of the class's resonators
    const float2 *tw;     // the class's twiddle table
    int nres;
    int logn;
    int item0;            // first item of the class in this launch
    int per;              // items per resonator
};

struct MixPlan {
    MixClass c[kMixMaxClasses];
    int ncls;
    int nitems;
};

// Class of item i (classes are few and in item order).
__device__ __forceinline__ int mix_class(const MixPlan &p, int i)
{
    int k = 0;
    while (k + 1 < p.ncls && i >= p.c[k + 1].item0) ++k;
    return k;
}

// First item >= i on this block's grid stride whose resonator still has
// bounces to do; a finished resonator is skipped in one step.
__device__ __forceinline__ int mix_next_active(const MixPlan &p, int i)
{
    const int grid = gridDim.x, b = blockIdx.x;
    while (i < p.nitems) {
        const MixClass &c = p.c[mix_class(p, i)];
        const int r = (i - c.item0) / c.per;
        if (res_active(c.res[r])) return i;
        const int first = c.item0 + (r + 1) * c.per;
        i = first + (int)((((long long)b - first) % grid + grid) % grid);
    }
    return p.nitems;
}

// ---- column items -------------------------------------------------------------

// Start the copy of column item `item` into the stage.
__device__ __forceinline__ void mix_col_issue(const MixPlan &p, int item, cpair *stage, uint64_t *bar)
{
    const MixClass &c = p.c[mix_class(p, item)];
    const int local = item - c.item0, r = local / c.per, tile = local % c.per;
    const int n = 1 << c.logn, C = mix_col_width(c.logn), BR = n < 256 ? n : 256;
    mbar_arrive_expect_tx(bar, (uint32_t)(n * C * sizeof(float2)));
    for (int b = 0; b < n / BR; ++b)
        tma_load_2d(stage + b * BR * (C / 2), c.res[r].tmap, 2 * tile * C, b * BR, bar);
}

template <typename F> struct MixIssueAfterReads {
    F issue;
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

// Diffract the C(n) columns of one item held in the stage (forward FFT,
// x h(my), inverse FFT) and store them; the next item's copy starts once the
// stage's last exchange has been read.
template <int LOGN, typename Hook>
__device__ __forceinline__ void mix_col_item(cpair *stage, const BatchRes &R, const float2 *__restrict__ tw, int tile,
                                             int *err, Hook next)
{
    constexpr int N = 1 << LOGN, T = Plan<LOGN>::T, C = mix_col_width(LOGN), CP = C / 2;
    static_assert(CP * T == kMixColThreads, "one column pair per thread");
    const int c2 = threadIdx.x % CP, t = threadIdx.x / CP;
    auto sync = []() { __syncthreads(); };
    const TabGlobal<LOGN, float2> tab{tw, R.h};
    cpair v[16];
#pragma unroll
    for (int si = 0; si < 16; ++si) v[si] = stage[(t + si * T) * CP + c2];
    LineBufs<cpair, false> lb{{stage + c2, stage + c2}, 0, err};
    fft_line_t<LOGN, -1, CP, false, true>(v, t, lb, tab, sync);
    fft_line_t<LOGN, +1, CP, false, false>(v, t, lb, tab, sync, next);
    cpair *col = reinterpret_cast<cpair *>(R.E + (size_t)t * N + tile * C) + c2;
#pragma unroll
    for (int si = 0; si < 16; ++si) col[(size_t)si * T * (N / 2)] = v[si];
}

__global__ void __launch_bounds__(kMixColThreads, 2) k_col_mixed(const __grid_constant__ MixPlan p, int *err)
{
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    cpair *stage = reinterpret_cast<cpair *>(sm + 128);
    auto issue = [&](int item) { mix_col_issue(p, item, stage, &bar[0]); };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        fence_barrier_init();
    }
    __syncthreads();
    int item = mix_next_active(p, blockIdx.x);
    if (threadIdx.x == 0 && item < p.nitems) issue(item);
    for (int it = 0; item < p.nitems; ++it) {
        const int nxt = mix_next_active(p, item + (int)gridDim.x);
        const MixClass &c = p.c[mix_class(p, item)];
        const int local = item - c.item0;
        const BatchRes &R = c.res[local / c.per];
        const int tile = local % c.per;
        const bool late = !mbar_wait(&bar[0], (uint32_t)(it & 1));
        if (__syncthreads_or(late)) {
            if (threadIdx.x == 0) atomicExch(err, ERR_TIMEOUT);
            break;
        }
        const MixIssueAfterReads<decltype(issue)> next{issue, nxt, nxt < p.nitems};
        switch (c.logn) {
        case 7: mix_col_item<7>(stage, R, c.tw, tile, err, next); break;
        case 8: mix_col_item<8>(stage, R, c.tw, tile, err, next); break;
        case 9: mix_col_item<9>(stage, R, c.tw, tile, err, next); break;
        case 10: mix_col_item<10>(stage, R, c.tw, tile, err, next); break;
        default: mix_col_item<11>(stage, R, c.tw, tile, err, next); break;
        }
        item = nxt;
    }
}

// ---- row items ------------------------------------------------------------------

__device__ __forceinline__ void mix_row_issue(const MixPlan &p, int item, unsigned char *stage, uint64_t *bar)
{
    const MixClass &c = p.c[mix_class(p, item)];
    const int local = item - c.item0, r = local / c.per, grp = local % c.per;
    const int n = 1 << c.logn, lpc = mix_row_lines(c.logn), ls = n / 16 * 17;
    const BatchRes &R = c.res[r];
    float2 *se = reinterpret_cast<float2 *>(stage);
    float *sn = reinterpret_cast<float *>(stage + kMixRowE);
    mbar_arrive_expect_tx(bar, (uint32_t)(lpc * n * (sizeof(float2) + sizeof(float))));
    for (int l = 0; l < lpc; ++l) {
        const size_t row = (size_t)grp * lpc + l;
        bulk_g2s(se + l * ls, R.E + row * n, n * sizeof(float2), bar);
        bulk_g2s(sn + l * n, R.N + row * n, n * sizeof(float), bar);
    }
}

// One row item: forward FFT, x h(mx), inverse FFT and the local map of its
// LPC(n) rows; returns the block's sum of |E_new|^2 over them (every thread
// gets it from the caller's reduction, here only the thread's share).
template <int LOGN>
__device__ __forceinline__ float mix_row_item(unsigned char *stage, const BatchRes &R, const float2 *__restrict__ tw,
                                              int grp, int *err)
{
    constexpr int N = 1 << LOGN, T = Plan<LOGN>::T, LPC = mix_row_lines(LOGN), LS = padded_len(N);
    static_assert(LPC * T == kMixRowThreads, "one row thread group per line");
    const int lig = threadIdx.x / T, t = threadIdx.x % T;
    auto sync = []() { __syncthreads(); };
    float2 *line = reinterpret_cast<float2 *>(stage) + lig * LS;
    const float *nrow = reinterpret_cast<const float *>(stage + kMixRowE) + lig * N + t;
    float2 v[16];
#pragma unroll
    for (int si = 0; si < 16; ++si) v[si] = line[t + si * T];
    LineBufs<float2, false> lb{{line, line}, 0, err};
    diffract_line<LOGN, 1>(v, t, lb, tw, R.h, sync);
    const int row = grp * LPC + lig;
    const GainParams<float> g = R.g;
    float2 *erow = R.E + (size_t)row * N + t;
    float *ngl = R.N + (size_t)row * N + t;
    const int feat = feature_form(g);
    if (feat == FEAT_TABLE_EXACT)
        return row_local_map<LOGN, PE_RUNTIME, false, FEAT_TABLE_EXACT>(v, t, row, nrow, erow, ngl, g, nullptr, R.pe);
    if (feat == FEAT_TABLE)
        return row_local_map<LOGN, PE_RUNTIME, false, FEAT_TABLE>(v, t, row, nrow, erow, ngl, g, nullptr, R.pe);
    if (R.pe == PE_UNIFORM) return row_local_map<LOGN, PE_UNIFORM>(v, t, row, nrow, erow, ngl, g);
    if (R.pe == PE_TABLE) return row_local_map<LOGN, PE_TABLE>(v, t, row, nrow, erow, ngl, g);
    return row_local_map<LOGN, PE_SG10>(v, t, row, nrow, erow, ngl, g);
}

__global__ void __launch_bounds__(kMixRowThreads, 4) k_row_mixed(const __grid_constant__ MixPlan p, int *err)
{
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    auto stage = [](int s) { return sm + 128 + s * kMixRowStage; };
    auto issue = [&](int s, int item) { mix_row_issue(p, item, stage(s), &bar[s]); };
    // A block runs a contiguous share of the items (BlockRange) and keeps one
    // running sum per resonator while it works through that resonator's
    // items, filing it when it moves on: the blocks that touch resonator r,
    // items [f, f + G), are block_of(f) .. block_of(f + G - 1), and block b
    // files under slot b - block_of(f).  A finished resonator is skipped in
    // one step.
    const BlockRange br(p.nitems);
    auto next_active = [&](int i) {
        while (i < br.end) {
            const MixClass &c = p.c[mix_class(p, i)];
            const int r = (i - c.item0) / c.per;
            if (res_active(c.res[r])) return i;
            i = c.item0 + (r + 1) * c.per;
        }
        return br.end;
    };
    init_stage_barriers(bar);
    int item = next_active(br.lo);
    if (threadIdx.x == 0 && item < br.end) issue(0, item);
    double dacc = 0.0;
    for (int it = 0; item < br.end; ++it) {
        const int s = it & 1;
        const int nxt = next_active(item + 1);
        if (threadIdx.x == 0 && nxt < br.end) {
            fence_proxy_async_smem();
            issue(s ^ 1, nxt);
        }
        if (stage_wait_or_abort(bar, it, nxt < br.end, err)) break;
        const int ci = mix_class(p, item);
        const MixClass &c = p.c[ci];
        const int local = item - c.item0, r = local / c.per, grp = local % c.per;
        const BatchRes &R = c.res[r];
        float acc;
        switch (c.logn) {
        case 7: acc = mix_row_item<7>(stage(s), R, c.tw, grp, err); break;
        case 8: acc = mix_row_item<8>(stage(s), R, c.tw, grp, err); break;
        case 9: acc = mix_row_item<9>(stage(s), R, c.tw, grp, err); break;
        case 10: acc = mix_row_item<10>(stage(s), R, c.tw, grp, err); break;
        default: acc = mix_row_item<11>(stage(s), R, c.tw, grp, err); break;
        }
        dacc += (double)acc;
        __syncthreads();  // stage s fully consumed before it is refilled
        const int first = c.item0 + r * c.per;
        if (nxt >= br.end || nxt < first || nxt >= first + c.per) {
            const int b0 = br.block_of(first);
            const int k = (int)blockIdx.x - b0, arrivals = br.block_of(first + c.per - 1) - b0 + 1;
            const int n = 1 << c.logn;
            res_finish<kMixRowThreads>(dacc, R.st, k, arrivals, 1.0 / ((double)n * (double)n));
            dacc = 0.0;
        }
        item = nxt;
    }
}

}  // namespace rtk
