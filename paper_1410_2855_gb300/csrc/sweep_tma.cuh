// Persistent, copy-engine-fed sweeps of the fused FP32 bounce.
//
// Each block loops over its share of lines (rows) or tiles (column strips).
// While it transforms line group g, the copy engine (TMA) is already
// loading group g + gridDim.x into the other of two shared-memory stages,
// so global-memory latency is hidden behind the FFT arithmetic instead of
// being paid by every block at its start.  A stage is laid out with the
// line FFT's padded stride: the copy engine fills the first n elements of
// each line densely, the first pass reads them, and from then on the same
// bytes serve as that line's exchange buffer.  Results leave registers
// straight to global memory.
//
// Every barrier wait is bounded in time; a timeout sets RT_ETIMEOUT in the
// handle's error word, drains the copy still in flight and ends the block.
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

template <int LOGN, int LPC, bool PP> struct RowStage {
    static constexpr int N = 1 << LOGN;
    static constexpr size_t e_bytes = round128((size_t)LPC * padded_len(N) * sizeof(float2));
    static constexpr size_t n_bytes = round128((size_t)LPC * N * sizeof(float));
    static constexpr size_t stage = e_bytes + n_bytes;
    static constexpr size_t extra = PP ? e_bytes : 0;   // second exchange buffer
    static constexpr size_t total = 128 + 2 * stage + extra;  // two mbarriers, two stages, extra buffer
};

template <int LOGN, int C, bool PP> struct ColStage {
    static constexpr int N = 1 << LOGN;
    static constexpr int BR = N < 256 ? N : 256;  // rows per tensor-map box (box dims are <= 256)
    static constexpr int NBOX = N / BR;
    static constexpr size_t stage = round128((size_t)C * padded_len(N) * sizeof(float2));
    static constexpr size_t total = 128 + (PP ? 3 : 2) * stage;
};

// Blocks per SM that the shared-memory plan allows (at most 8).
constexpr int smem_blocks(size_t bytes)
{
    return (int)((228 * 1024) / (bytes + 1024)) > 8 ? 8 : ((int)((228 * 1024) / (bytes + 1024)) > 0 ? (int)((228 * 1024) / (bytes + 1024)) : 1);
}

// Resident blocks asked of the compiler for the column sweep: what shared
// memory allows, but never fewer than RTK_COL_REGS registers per thread (the
// column FFT spills below ~96).
#ifndef RTK_COL_REGS
#define RTK_COL_REGS 128
#endif
constexpr int col_min_blocks(int threads, size_t bytes)
{
    return smem_blocks(bytes) < 65536 / (threads * RTK_COL_REGS) ? smem_blocks(bytes)
                                                                   : (65536 / (threads * RTK_COL_REGS) > 0 ? 65536 / (threads * RTK_COL_REGS) : 1);
}

// Row sweep: LPC rows per group, T = n/16 threads per row.
template <int LOGN, int LPC, int PE, bool PP = RTK_ROW_PP>
__global__ void __launch_bounds__(LPC * Plan<LOGN>::T, smem_blocks(RowStage<LOGN, LPC, PP>::total))
k_row_tma(float2 *E, float *Nv, const float2 *__restrict__ tw, const float2 *__restrict__ h, GainParams<float> g,
          StatParams st, int ngroups)
{
    using P = Plan<LOGN>;
    using L = RowStage<LOGN, LPC, PP>;
    constexpr int N = P::N, T = P::T, NT = LPC * T, LS = padded_len(N);
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const int lig = threadIdx.x / T, t = threadIdx.x % T;
    auto stage_e = [](int s) { return reinterpret_cast<float2 *>(sm + 128 + s * L::stage); };
    auto stage_n = [](int s) { return reinterpret_cast<float *>(sm + 128 + s * L::stage + L::e_bytes); };
    auto sync = []() { __syncthreads(); };
    auto issue = [&](int s, int grp) {
        mbar_arrive_expect_tx(&bar[s], (uint32_t)(LPC * N * (sizeof(float2) + sizeof(float))));
        for (int l = 0; l < LPC; ++l) {
            const size_t row = (size_t)grp * LPC + l;
            bulk_g2s(stage_e(s) + l * LS, E + row * N, N * sizeof(float2), &bar[s]);
            bulk_g2s(stage_n(s) + l * N, Nv + row * N, N * sizeof(float), &bar[s]);
        }
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
    int grp = blockIdx.x;
    if (threadIdx.x == 0 && grp < ngroups) issue(0, grp);

    const float step = 2.0f / (float)N;
    const float xc0 = (float)(t - N / 2) * step;
    double dacc = 0.0;
    for (int it = 0; grp < ngroups; ++it, grp += gridDim.x) {
        const int s = it & 1;
        const int nxt = grp + (int)gridDim.x;
        if (threadIdx.x == 0 && nxt < ngroups) {
            fence_proxy_async_smem();
            issue(s ^ 1, nxt);
        }
        const bool late = !mbar_wait(&bar[s], (uint32_t)((it >> 1) & 1));
        if (__syncthreads_or(late)) {
            if (threadIdx.x == 0) {
                atomicExch(st.err, ERR_TIMEOUT);
                if (nxt < ngroups) mbar_wait(&bar[s ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            break;
        }
        const int row = grp * LPC + lig;
        float2 *line = stage_e(s) + lig * LS;
        const float *nrow = stage_n(s) + lig * N + t;
        float2 v[16];
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = line[t + si * T];
        // With ping-pong the first exchange goes to the extra buffer, so the
        // dense stage is only overwritten after every thread has read it.
        float2 *extra = reinterpret_cast<float2 *>(sm + 128 + 2 * L::stage) + lig * LS;
        LineBufs<float2, PP> lb{{PP ? extra : line, line}, 0};
        fft_line<LOGN, -1, 1>(v, t, lb, tw, sync);
        const float2 *hp = h + t;
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = cmul(v[si], __ldg(hp + si * T));
        fft_line<LOGN, +1, 1>(v, t, lb, tw, sync);

        const float yc = (float)(row - N / 2) * step;
        const float yq = yc * yc * g.inv_rp2;
        const bool row_in = row >= g.edge && row < N - g.edge;
        float2 *erow = E + (size_t)row * N + t;
        float *ngl = Nv + (size_t)row * N + t;
        float acc = 0.0f;
#pragma unroll
        for (int si = 0; si < 16; ++si) {
            const int x = t + si * T;
            const float nn = nrow[si * T];
            float2 e = v[si];
            const float inten = e.x * e.x + e.y * e.y;
            const bool inside = row_in && x >= g.edge && x < N - g.edge;
            e = cscale(e, inside ? g.sqrtR * fexp(0.5f * nn) : 0.0f);
            float n0;
            if constexpr (PE == PE_UNIFORM) {
                n0 = g.g0;
            } else if constexpr (PE == PE_TABLE) {
                n0 = __ldg(g.pump_tab + (size_t)row * N + x);
            } else {
                const float xc = xc0 + (float)(si * T) * step;
                const float q = xc * xc * g.inv_rp2 + yq;
                const float q2 = q * q;
                n0 = g.g0 * fexp(-(q2 * q2 * q));
            }
            ngl[si * T] = nn + (n0 - nn * (1.0f + inten * g.invIsat)) * g.invT1;
            erow[si * T] = e;
            acc += e.x * e.x + e.y * e.y;
        }
        dacc += (double)acc;
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

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
    int tile = blockIdx.x;
    if (threadIdx.x == 0 && tile < ntiles) issue(0, tile);
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const int s = it & 1;
        const int nxt = tile + (int)gridDim.x;
        if (threadIdx.x == 0 && nxt < ntiles) {
            fence_proxy_async_smem();
            issue(s ^ 1, nxt);
        }
        const bool late = !mbar_wait(&bar[s], (uint32_t)((it >> 1) & 1));
        if (__syncthreads_or(late)) {
            if (threadIdx.x == 0) {
                atomicExch(err, ERR_TIMEOUT);
                if (nxt < ntiles) mbar_wait(&bar[s ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            break;
        }
        float2 *base = stage(s);
        float2 v[16];
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = base[(t + si * T) * C + c];
        float2 *extra = stage(2);
        LineBufs<float2, PP> lb{{PP ? extra + c : base + c, base + c}, 0};
        fft_line<LOGN, -1, C>(v, t, lb, tw, sync);
        const float2 *hp = h + t;
#pragma unroll
        for (int si = 0; si < 16; ++si) v[si] = cmul(v[si], __ldg(hp + si * T));
        fft_line<LOGN, +1, C>(v, t, lb, tw, sync);
        float2 *col = E + (size_t)t * N + tile * C + c;
#pragma unroll
        for (int si = 0; si < 16; ++si) col[(size_t)si * T * N] = v[si];
        __syncthreads();  // stage s fully consumed before it is refilled
    }
}

}  // namespace rtk
