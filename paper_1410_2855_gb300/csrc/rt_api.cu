// C ABI of the bounce-map library (include/rt.h): resonator handles,
// stepping with captured CUDA graphs, checkpoint reads/writes, statistics and
// spectrum readout.  Every entry point returns an rt_status and never aborts.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>

#include "rt.h"
#include "rt_internal.h"
#include "trace.h"

// 1: FP32 handles with the order-10 super-Gaussian pump read N0 from a table
// staged with each row (4 more bytes per point, no exp per point).
#ifndef RTK_ROW_PUMP_TABLE
#define RTK_ROW_PUMP_TABLE 0
#endif

using namespace rtk;

namespace {

// Device-side control block of a handle (one small allocation).
struct Ctl {
    unsigned int count;       // arrival counter of the mean-intensity reduction
    unsigned int peak_count;  // arrival counter of the spectrum-peak reduction
    int err;                  // sticky device error (0 or RT_ENUMERIC)
    int pad;
    long long bounce;         // bounces completed on the device
    double last_mean;         // mean intensity after the last bounce
    PeakResult peak;
};

constexpr int kMaxPart = 4096;  // block partials of any reduction (>= every launch's grid)

rt_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return RT_OK;
    if (e == cudaErrorMemoryAllocation) return RT_ENOMEM;
    return RT_ECUDA;
}

#define RT_TRY(expr)                              \
    do {                                          \
        cudaError_t e_ = (expr);                  \
        if (e_ != cudaSuccess) return from_cuda(e_); \
    } while (0)

int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// Keeps the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1, want;
    explicit DeviceGuard(int dev) : want(dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != want) cudaSetDevice(want);
    }
    ~DeviceGuard()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

}  // namespace

struct rt_handle {
    int n = 0, logn = 0, precision = RT_FP32, device = 0;
    double fresnel = 0, alpha = 0, g0 = 0, T1 = 1, R = 1;
    rt_opts opts{};
    rt_pump pump{};
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    void *E = nullptr, *N = nullptr, *tw = nullptr, *h = nullptr;
    void *pump_tab = nullptr;     // N0 table (array pump, FP32 path)
    void *lens = nullptr;         // per-axis curved-mirror factors (no roughness)
    void *phase = nullptr;        // n*n aperture factors (roughness, with the lens folded in)
    void *ones = nullptr;         // n unit factors: the slices before the last under the exact inversion update
    double *profile = nullptr;    // device copy of the array pump profile
    void *X = nullptr, *S = nullptr;  // spectrum scratch (lazily allocated)
    void *hz = nullptr;               // propagator of the last intracavity readout distance (lazily allocated)
    double *part = nullptr;
    double *peak_val = nullptr;
    long long *peak_idx = nullptr;
    double *hist = nullptr;
    Ctl *ctl = nullptr;
    Ctl *slice_ctl = nullptr;     // reduction counters of the slices before the last (m > 1)
    int slices = 1;
    long long bounces = 0;
    int colC = 4;
    int col_order = 0;            // radix order of the FP32 column transforms (0: built-in)
    void *tw_col = nullptr;       // that order's twiddles (only when col_order != 0; else tw serves)
    int pe = 0;                   // pump evaluation of the FP32 row sweep (PumpEval)
    alignas(64) unsigned char tmap[128] = {};  // tensor map of E for the column sweep's tile loads
    std::map<long long, cudaGraphExec_t> graphs;
    size_t esz() const { return precision == RT_FP64 ? 16 : 8; }
    size_t rsz() const { return precision == RT_FP64 ? 8 : 4; }
    size_t points() const { return (size_t)n * n; }
    size_t inv_points() const { return points() * (size_t)slices; }
};

namespace {

// Statistics of a bounce (the last slice); the slices before it reduce into
// their own counters and leave the bounce count and history alone.
StatParams stat_params(rt_handle *h, bool last = true)
{
    StatParams st{};
    Ctl *c = last ? h->ctl : h->slice_ctl;
    st.part = h->part;
    st.count = &c->count;
    st.hist = last ? h->hist : nullptr;
    st.hist_cap = last ? h->opts.history_cap : 0;
    st.bounce = &c->bounce;
    st.last_mean = &c->last_mean;
    st.err = &h->ctl->err;
    return st;
}

// Local-map parameters of one slice: the pump is N0/m in every slice; the
// mirror (sqrt R, edge, aperture phase) acts only in the last.
template <typename R>
GainParams<R> gain_params(rt_handle *h, bool last = true)
{
    GainParams<R> g{};
    g.sqrtR = last ? (R)std::sqrt(h->R) : R(1);
    g.invT1 = (R)(1.0 / h->T1);
    g.invIsat = (R)(1.0 / h->opts.Isat);
    g.g0 = (R)(h->g0 / h->slices);
    const double r = h->pump.radius;
    g.inv_rp2 = (R)(1.0 / (r * r));
    const double half = 0.5 * h->pump.order;
    g.half_order = (R)half;
    g.int_half_order = (h->pump.kind == RT_PUMP_SUPERGAUSS && half == 5.0) ? 5 : 0;
    g.edge = last ? h->opts.edge_px : 0;
    g.pump_kind = h->pump.kind;
    g.pump_tab = reinterpret_cast<const R *>(h->pump_tab);
    using C = typename cplx_of<R>::type;
    g.relax_exact = h->opts.relax == RT_RELAX_EXACT;
    g.lens = last ? static_cast<const C *>(h->lens) : (g.relax_exact ? static_cast<const C *>(h->ones) : nullptr);
    g.phase = last ? static_cast<const C *>(h->phase) : nullptr;
    return g;
}

// One bounce: per slice (one unless the gain medium is sliced) the
// diffraction over z/m and the slice's local map on its own inversion.
const float2 *col_twiddles(const rt_handle *h)
{
    return static_cast<const float2 *>(h->col_order ? h->tw_col : h->tw);
}

cudaError_t enqueue_bounce(rt_handle *h, cudaStream_t s)
{
    const size_t P = h->points();
    cudaError_t e;
    for (int k = 0; k < h->slices; ++k) {
        const bool last = k == h->slices - 1;
        const StatParams st = stat_params(h, last);
        if (h->precision == RT_FP32) {
            float2 *E = static_cast<float2 *>(h->E);
            const float2 *tw = static_cast<const float2 *>(h->tw), *hh = static_cast<const float2 *>(h->h);
            if ((e = launch_col_diffract32(h->logn, h->colC, E, col_twiddles(h), hh, h->tmap, &h->ctl->err, s,
                                           h->col_order)) != cudaSuccess)
                return e;
            e = launch_row_diffract_gain32(h->logn, h->pe, E, static_cast<float *>(h->N) + k * P, tw, hh,
                                           gain_params<float>(h, last), st, s);
        } else {
            double2 *E = static_cast<double2 *>(h->E);
            const double2 *tw = static_cast<const double2 *>(h->tw), *hh = static_cast<const double2 *>(h->h);
            if ((e = launch_row_fft64(h->logn, E, E, tw, -1, s)) != cudaSuccess) return e;
            if ((e = launch_col_fft64(h->logn, E, tw, -1, s)) != cudaSuccess) return e;
            if ((e = launch_mul_h64(h->n, E, hh, s)) != cudaSuccess) return e;
            if ((e = launch_col_fft64(h->logn, E, tw, +1, s)) != cudaSuccess) return e;
            if ((e = launch_row_fft64(h->logn, E, E, tw, +1, s)) != cudaSuccess) return e;
            e = launch_gain64(h->n, E, static_cast<double *>(h->N) + k * P, gain_params<double>(h, last), st, s);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t get_graph(rt_handle *h, long long k, cudaGraphExec_t *out)
{
    auto it = h->graphs.find(k);
    if (it != h->graphs.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaError_t e = h->precision == RT_FP32
                        ? prepare_bounce32(h->logn, h->colC, h->pe, feature_form(gain_params<float>(h, true)))
                        : prepare_bounce64(h->logn);
    if (e == cudaSuccess && h->precision == RT_FP32 && h->slices > 1)
        e = prepare_row32(h->logn, h->pe, feature_form(gain_params<float>(h, false)));
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t launch_err = cudaSuccess;
    for (long long i = 0; i < k && launch_err == cudaSuccess; ++i) launch_err = enqueue_bounce(h, h->capture_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->capture_stream, &g);
    if (launch_err != cudaSuccess) e = launch_err;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    h->graphs[k] = ge;
    *out = ge;
    return cudaSuccess;
}

rt_status check_device_error(rt_handle *h)
{
    int err = 0;
    RT_TRY(cudaMemcpyAsync(&err, &h->ctl->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    RT_TRY(cudaStreamSynchronize(h->stream));
    return err ? (rt_status)err : RT_OK;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

void release(rt_handle *h)
{
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    void *bufs[] = {h->E, h->N, h->tw, h->tw_col, h->h, h->pump_tab, h->lens, h->phase, h->ones, h->profile, h->X, h->S, h->hz,
                    h->part, h->peak_val, h->peak_idx, h->hist, h->ctl, h->slice_ctl};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
}

rt_status ensure_spectrum_scratch(rt_handle *h)
{
    if (!h->X) RT_TRY(dev_alloc(&h->X, h->points() * h->esz()));
    if (!h->S) RT_TRY(dev_alloc(&h->S, h->points() * h->rsz()));
    if (!h->peak_val) RT_TRY(dev_alloc(&h->peak_val, sizeof(double) * kMaxPart));
    if (!h->peak_idx) RT_TRY(dev_alloc(&h->peak_idx, sizeof(long long) * kMaxPart));
    return RT_OK;
}

// S = |DFT2(E)|^2 into h->S.
rt_status compute_spectrum(rt_handle *h)
{
    rt_status st = ensure_spectrum_scratch(h);
    if (st != RT_OK) return st;
    if (h->precision == RT_FP32) {
        const float2 *tw = static_cast<const float2 *>(h->tw);
        float2 *X = static_cast<float2 *>(h->X);
        RT_TRY(launch_row_fft32(h->logn, static_cast<const float2 *>(h->E), X, tw, -1, h->stream));
        RT_TRY(launch_col_fft32(h->logn, X, tw, -1, h->stream));
        RT_TRY(launch_power32(h->n, X, static_cast<float *>(h->S), h->stream));
    } else {
        const double2 *tw = static_cast<const double2 *>(h->tw);
        double2 *X = static_cast<double2 *>(h->X);
        RT_TRY(launch_row_fft64(h->logn, static_cast<const double2 *>(h->E), X, tw, -1, h->stream));
        RT_TRY(launch_col_fft64(h->logn, X, tw, -1, h->stream));
        RT_TRY(launch_power64(h->n, X, static_cast<double *>(h->S), h->stream));
    }
    return RT_OK;
}

}  // namespace

extern "C" {

int rt_version(void) { return 100; }

const char *rt_status_string(rt_status s)
{
    switch (s) {
    case RT_OK: return "ok";
    case RT_EINVAL: return "invalid argument";
    case RT_ENOMEM: return "out of memory";
    case RT_ECUDA: return "CUDA error";
    case RT_ENUMERIC: return "non-finite field intensity";
    case RT_ETIMEOUT: return "bounded wait timed out";
    case RT_EBUSY: return "busy";
    case RT_EBOUNDS: return "index out of bounds (checked build)";
    case RT_ECANCELED: return "request cancelled";
    default: return "unknown status";
    }
}

rt_status rt_opts_default(rt_opts *o)
{
    if (!o) return RT_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->Isat = 1.0;
    o->edge_px = 8;
    o->precision = RT_FP32;
    o->seed = 14102855ull;
    o->noise_amp = 1e-6;
    o->pump_diam_over_window = 0.8;
    o->cuda_stream = nullptr;
    o->history_cap = 65536;
    o->chunk = 500;
    return RT_OK;
}

rt_status rt_create(int n, double fresnel, const rt_pump *pump, double g0, double T1, double R, const rt_opts *opts,
                    rt_handle **out)
{
    if (!out) return RT_EINVAL;
    *out = nullptr;
    rt_opts o;
    if (opts) o = *opts;
    else rt_opts_default(&o);
    rt_pump p{RT_PUMP_SUPERGAUSS, 10.0, 0.8, nullptr};
    if (pump) p = *pump;
    if (!is_pow2(n) || n < 32 || n > 4096) return RT_EINVAL;
    if (!finite_pos(fresnel) || !std::isfinite(g0) || g0 < 0.0 || !std::isfinite(T1) || T1 < 1.0) return RT_EINVAL;
    if (!std::isfinite(R) || R <= 0.0 || R > 1.0) return RT_EINVAL;
    if (!finite_pos(o.Isat) || o.edge_px < 0 || o.edge_px > n / 2) return RT_EINVAL;
    if (o.precision != RT_FP32 && o.precision != RT_FP64) return RT_EINVAL;
    if (!std::isfinite(o.noise_amp) || o.noise_amp < 0.0 || !finite_pos(o.pump_diam_over_window)) return RT_EINVAL;
    if (!std::isfinite(o.z_over_F) || o.slices < 0 || o.slices > 64) return RT_EINVAL;
    if (o.taper_px < 0 || o.taper_px > n / 2 || (o.relax != RT_RELAX_EULER && o.relax != RT_RELAX_EXACT))
        return RT_EINVAL;
    if (o.history_cap < 0 || o.chunk < 0) return RT_EINVAL;
    if (o.col_tile != 0 && (o.precision != RT_FP32 || !col_tile_ok32(ilog2(n), o.col_tile))) return RT_EINVAL;
    if (p.kind == RT_PUMP_SUPERGAUSS && (!finite_pos(p.order) || !finite_pos(p.radius))) return RT_EINVAL;
    if (p.kind == RT_PUMP_ARRAY && !p.profile) return RT_EINVAL;
    if (p.kind < RT_PUMP_SUPERGAUSS || p.kind > RT_PUMP_ARRAY) return RT_EINVAL;

    TraceRange tr("rt_create");
    rt_handle *h = new (std::nothrow) rt_handle();
    if (!h) return RT_ENOMEM;
    h->n = n;
    h->logn = ilog2(n);
    h->precision = o.precision;
    h->fresnel = fresnel;
    h->alpha = o.pump_diam_over_window * o.pump_diam_over_window / fresnel;
    h->g0 = g0;
    h->T1 = T1;
    h->R = R;
    h->opts = o;
    h->pump = p;
    h->pump.profile = nullptr;
    h->opts.roughness = nullptr;
    h->slices = o.slices > 1 ? o.slices : 1;
    h->stream = static_cast<cudaStream_t>(o.cuda_stream);
    h->colC = o.col_tile ? o.col_tile : default_col_tile32(h->logn);
    // the tuned radix order goes with the tuned tile width
    if (h->precision == RT_FP32 && o.col_tile == 0) {
        const int ord = tuned_col_order32(h->logn);
        h->col_order = ord < col_orders32(h->logn, h->colC) ? ord : 0;
    }
    // N0 on the fly for the order-10 super-Gaussian and the uniform pump, else from a table
    h->pe = p.kind == RT_PUMP_UNIFORM ? 1 : ((p.kind == RT_PUMP_SUPERGAUSS && p.order == 10.0) ? 0 : 2);
#if RTK_ROW_PUMP_TABLE
    // FP32 handles read N0 from a table staged with the rows instead of evaluating it.
    if (h->precision == RT_FP32 && h->pe == 0) h->pe = 2;
#endif
    cudaGetDevice(&h->device);

    auto fail = [&](rt_status s) {
        release(h);
        delete h;
        return s;
    };
#define RT_CREATE_TRY(expr)                       \
    do {                                          \
        cudaError_t e_ = (expr);                  \
        if (e_ != cudaSuccess) return fail(from_cuda(e_)); \
    } while (0)

    const size_t P = h->points();
    RT_CREATE_TRY(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    RT_CREATE_TRY(dev_alloc(&h->E, P * h->esz()));
    RT_CREATE_TRY(dev_alloc(&h->N, h->inv_points() * h->rsz()));
    RT_CREATE_TRY(dev_alloc(&h->tw, (size_t)(twiddle_entries(h->logn) + 1) * h->esz()));
    RT_CREATE_TRY(dev_alloc(&h->h, (size_t)n * h->esz()));
    RT_CREATE_TRY(dev_alloc(&h->part, sizeof(double) * kMaxPart));
    RT_CREATE_TRY(dev_alloc(reinterpret_cast<void **>(&h->ctl), sizeof(Ctl)));
    RT_CREATE_TRY(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->stream));
    if (h->slices > 1) {
        RT_CREATE_TRY(dev_alloc(reinterpret_cast<void **>(&h->slice_ctl), sizeof(Ctl)));
        RT_CREATE_TRY(cudaMemsetAsync(h->slice_ctl, 0, sizeof(Ctl), h->stream));
    }
    if (o.history_cap > 0) RT_CREATE_TRY(dev_alloc(&h->hist, sizeof(double) * (size_t)o.history_cap));
    if (p.kind == RT_PUMP_ARRAY) {
        RT_CREATE_TRY(dev_alloc(&h->profile, sizeof(double) * P));
        RT_CREATE_TRY(cudaMemcpyAsync(h->profile, p.profile, sizeof(double) * P, cudaMemcpyDefault, h->stream));
    }
    // Complex aperture beyond the hard edge: a full table when the mirror is
    // rough (lens and taper folded in), else per-axis factors when it is
    // curved or the edge tapered or the general local map is needed anyway
    // (exact inversion update), else nothing.
    const double c = lens_curvature(h->alpha, o.z_over_F);
    const double g0s = g0 / h->slices;   // pump of one slice: N0/m
    double *psi = nullptr;
    if (o.roughness) {
        RT_CREATE_TRY(dev_alloc(&h->phase, P * h->esz()));
        RT_CREATE_TRY(dev_alloc(&psi, sizeof(double) * P));
        cudaError_t e = cudaMemcpyAsync(psi, o.roughness, sizeof(double) * P, cudaMemcpyDefault, h->stream);
        if (e == cudaSuccess)
            e = h->precision == RT_FP32
                    ? launch_phase32(n, c, o.edge_px, o.taper_px, psi, static_cast<float2 *>(h->phase), h->stream)
                    : launch_phase64(n, c, o.edge_px, o.taper_px, psi, static_cast<double2 *>(h->phase), h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        cudaFree(psi);
        RT_CREATE_TRY(e);
    } else if (o.z_over_F != 0.0 || o.taper_px > 0 || o.relax == RT_RELAX_EXACT) {
        RT_CREATE_TRY(dev_alloc(&h->lens, (size_t)n * h->esz()));
        RT_CREATE_TRY(h->precision == RT_FP32
                          ? launch_lens32(n, c, o.edge_px, o.taper_px, static_cast<float2 *>(h->lens), h->stream)
                          : launch_lens64(n, c, o.edge_px, o.taper_px, static_cast<double2 *>(h->lens), h->stream));
    }

    if (h->precision == RT_FP32) {
        RT_CREATE_TRY(launch_tables32(n, h->alpha / h->slices, static_cast<float2 *>(h->tw), static_cast<float2 *>(h->h),
                                      h->stream));
        if (h->col_order) {
            RT_CREATE_TRY(dev_alloc(&h->tw_col, (size_t)(twiddle_entries(h->logn) + 1) * sizeof(float2)));
            RT_CREATE_TRY(launch_twiddles32(n, h->col_order, static_cast<float2 *>(h->tw_col), h->stream));
        }
        RT_CREATE_TRY(make_col_tensor_map(h->tmap, static_cast<float2 *>(h->E), n, h->colC));
        RT_CREATE_TRY(launch_noise32(n, o.seed, o.noise_amp, static_cast<float2 *>(h->E), h->stream));
        RT_CREATE_TRY(launch_pump32(n, p.kind, g0s, p.order, p.radius, h->profile, static_cast<float *>(h->N), h->stream));
        if (h->pe == 2) {
            RT_CREATE_TRY(dev_alloc(&h->pump_tab, sizeof(float) * P));
            RT_CREATE_TRY(cudaMemcpyAsync(h->pump_tab, h->N, sizeof(float) * P, cudaMemcpyDeviceToDevice, h->stream));
        }
    } else {
        RT_CREATE_TRY(launch_tables64(n, h->alpha / h->slices, static_cast<double2 *>(h->tw),
                                      static_cast<double2 *>(h->h), h->stream));
        RT_CREATE_TRY(launch_noise64(n, o.seed, o.noise_amp, static_cast<double2 *>(h->E), h->stream));
        RT_CREATE_TRY(launch_pump64(n, p.kind, g0s, p.order, p.radius, h->profile, static_cast<double *>(h->N), h->stream));
        if (h->pe == 2) {
            RT_CREATE_TRY(dev_alloc(&h->pump_tab, sizeof(double) * P));
            RT_CREATE_TRY(cudaMemcpyAsync(h->pump_tab, h->N, sizeof(double) * P, cudaMemcpyDeviceToDevice, h->stream));
        }
    }
    if (h->slices > 1 && o.relax == RT_RELAX_EXACT) {
        RT_CREATE_TRY(dev_alloc(&h->ones, (size_t)n * h->esz()));
        RT_CREATE_TRY(h->precision == RT_FP32 ? launch_lens32(n, 0.0, 0, 0, static_cast<float2 *>(h->ones), h->stream)
                                              : launch_lens64(n, 0.0, 0, 0, static_cast<double2 *>(h->ones), h->stream));
    }
    // every slice starts fully pumped: N0/m
    for (int k = 1; k < h->slices; ++k)
        RT_CREATE_TRY(cudaMemcpyAsync(static_cast<char *>(h->N) + k * P * h->rsz(), h->N, P * h->rsz(),
                                      cudaMemcpyDeviceToDevice, h->stream));
    RT_CREATE_TRY(cudaStreamSynchronize(h->stream));
#undef RT_CREATE_TRY
    *out = h;
    return RT_OK;
}

rt_status rt_step(rt_handle *h, long long nb)
{
    if (!h || nb < 0) return RT_EINVAL;
    if (nb == 0) return RT_OK;
    TraceRange tr("rt_step");
    DeviceGuard dg(h->device);
    const long long K = h->opts.chunk;
    long long left = nb;
    if (K > 0 && left >= K) {
        cudaGraphExec_t ge;
        RT_TRY(get_graph(h, K, &ge));
        for (; left >= K; left -= K) RT_TRY(cudaGraphLaunch(ge, h->stream));
    }
    for (; left > 0; --left) RT_TRY(enqueue_bounce(h, h->stream));
    h->bounces += nb;
    return RT_OK;
}

rt_status rt_sweep(rt_handle *h, int which)
{
    if (!h || h->precision != RT_FP32 || h->slices > 1 || (which != RT_SWEEP_COLUMNS && which != RT_SWEEP_ROWS))
        return RT_EINVAL;
    TraceRange tr(which == RT_SWEEP_COLUMNS ? "rt_sweep columns" : "rt_sweep rows");
    DeviceGuard dg(h->device);
    float2 *E = static_cast<float2 *>(h->E);
    const float2 *tw = static_cast<const float2 *>(h->tw), *hh = static_cast<const float2 *>(h->h);
    if (which == RT_SWEEP_COLUMNS) {
        RT_TRY(launch_col_diffract32(h->logn, h->colC, E, col_twiddles(h), hh, h->tmap, &h->ctl->err, h->stream,
                                     h->col_order));
    } else {
        RT_TRY(launch_row_diffract_gain32(h->logn, h->pe, E, static_cast<float *>(h->N), tw, hh, gain_params<float>(h),
                                          stat_params(h), h->stream));
        h->bounces += 1;
    }
    return RT_OK;
}

rt_status rt_sync(rt_handle *h)
{
    if (!h) return RT_EINVAL;
    DeviceGuard dg(h->device);
    return check_device_error(h);
}

static rt_status copy_out(rt_handle *h, void *dst, const void *src, size_t bytes, size_t want)
{
    if (!h || !dst) return RT_EINVAL;
    if (bytes != want) return RT_EINVAL;
    DeviceGuard dg(h->device);
    RT_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->stream));
    return check_device_error(h);
}

rt_status rt_read_field(rt_handle *h, void *dst, size_t bytes)
{
    if (!h) return RT_EINVAL;
    return copy_out(h, dst, h->E, bytes, h->points() * h->esz());
}

rt_status rt_read_inversion(rt_handle *h, void *dst, size_t bytes)
{
    if (!h) return RT_EINVAL;
    return copy_out(h, dst, h->N, bytes, h->inv_points() * h->rsz());
}

static rt_status copy_in(rt_handle *h, void *dst, const void *src, size_t bytes, size_t want)
{
    if (!h || !src) return RT_EINVAL;
    if (bytes != want) return RT_EINVAL;
    DeviceGuard dg(h->device);
    RT_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->stream));
    return RT_OK;
}

rt_status rt_write_field(rt_handle *h, const void *src, size_t bytes)
{
    if (!h) return RT_EINVAL;
    return copy_in(h, h->E, src, bytes, h->points() * h->esz());
}

rt_status rt_write_inversion(rt_handle *h, const void *src, size_t bytes)
{
    if (!h) return RT_EINVAL;
    return copy_in(h, h->N, src, bytes, h->inv_points() * h->rsz());
}

rt_status rt_set_bounces(rt_handle *h, long long bounces)
{
    if (!h || bounces < 0) return RT_EINVAL;
    DeviceGuard dg(h->device);
    RT_TRY(cudaStreamSynchronize(h->stream));
    RT_TRY(cudaMemcpy(&h->ctl->bounce, &bounces, sizeof(bounces), cudaMemcpyHostToDevice));
    h->bounces = bounces;
    return RT_OK;
}

rt_status rt_stats(rt_handle *h, rt_stats_t *out)
{
    if (!h || !out) return RT_EINVAL;
    DeviceGuard dg(h->device);
    Ctl c;
    RT_TRY(cudaMemcpyAsync(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    RT_TRY(cudaStreamSynchronize(h->stream));
    std::memset(out, 0, sizeof(*out));
    out->bounces = c.bounce;
    out->mean_intensity = c.last_mean;
    out->alpha = h->alpha;
    out->n = h->n;
    out->precision = h->precision;
    out->last_error = c.err;
    const long long cap = h->opts.history_cap;
    out->history_len = cap > 0 ? (c.bounce < cap ? c.bounce : cap) : 0;
    return RT_OK;
}

rt_status rt_read_history(rt_handle *h, double *dst, long long max, long long *got)
{
    if (!h || !got || max < 0 || (max > 0 && !dst)) return RT_EINVAL;
    *got = 0;
    rt_stats_t s;
    rt_status st = rt_stats(h, &s);
    if (st != RT_OK) return st;
    const long long cap = h->opts.history_cap;
    long long len = s.history_len < max ? s.history_len : max;
    if (len <= 0 || cap <= 0) return RT_OK;
    DeviceGuard dg(h->device);
    // the last `len` bounces: b = total-len .. total-1, slot b % cap
    const long long first = s.bounces - len;
    long long done = 0;
    while (done < len) {
        const long long slot = (first + done) % cap;
        long long run = cap - slot;
        if (run > len - done) run = len - done;
        RT_TRY(cudaMemcpy(dst + done, h->hist + slot, sizeof(double) * (size_t)run, cudaMemcpyDeviceToHost));
        done += run;
    }
    *got = len;
    return RT_OK;
}

rt_status rt_read_spectrum(rt_handle *h, void *dst, size_t bytes)
{
    if (!h || !dst) return RT_EINVAL;
    if (bytes != h->points() * h->rsz()) return RT_EINVAL;
    DeviceGuard dg(h->device);
    rt_status st = compute_spectrum(h);
    if (st != RT_OK) return st;
    RT_TRY(cudaMemcpyAsync(dst, h->S, bytes, cudaMemcpyDefault, h->stream));
    return check_device_error(h);
}

rt_status rt_set_field_pattern(rt_handle *h, const rt_pattern *pt)
{
    if (!h || !pt) return RT_EINVAL;
    if (pt->kind < RT_PATTERN_GAUSSIAN || pt->kind > RT_PATTERN_VORTEX_ARRAY) return RT_EINVAL;
    if (!finite_pos(pt->width) || !std::isfinite(pt->envelope) || pt->envelope < 0.0) return RT_EINVAL;
    if (!std::isfinite(pt->curvature) || !std::isfinite(pt->amplitude)) return RT_EINVAL;
    if (pt->kind != RT_PATTERN_GAUSSIAN &&
        (pt->periods < 1 || pt->periods > 4096 || (pt->out_of_phase && (pt->periods & 1))))
        return RT_EINVAL;
    DeviceGuard dg(h->device);
    const int q = pt->kind == RT_PATTERN_GAUSSIAN ? 1 : pt->periods, alt = pt->out_of_phase ? 1 : 0;
    if (h->precision == RT_FP32)
        RT_TRY(launch_pattern32(h->n, pt->kind, q, alt, pt->width, pt->envelope, pt->curvature, pt->amplitude,
                                static_cast<float2 *>(h->E), h->stream));
    else
        RT_TRY(launch_pattern64(h->n, pt->kind, q, alt, pt->width, pt->envelope, pt->curvature, pt->amplitude,
                                static_cast<double2 *>(h->E), h->stream));
    return RT_OK;
}

rt_status rt_read_field_at(rt_handle *h, double zeta, void *dst, size_t bytes)
{
    if (!h || !dst || !std::isfinite(zeta)) return RT_EINVAL;
    if (bytes != h->points() * h->esz()) return RT_EINVAL;
    DeviceGuard dg(h->device);
    rt_status st = ensure_spectrum_scratch(h);
    if (st != RT_OK) return st;
    if (!h->hz) RT_TRY(dev_alloc(&h->hz, (size_t)h->n * h->esz()));
    const double a = h->alpha * zeta;
    if (h->precision == RT_FP32) {
        const float2 *tw = static_cast<const float2 *>(h->tw);
        float2 *X = static_cast<float2 *>(h->X), *hz = static_cast<float2 *>(h->hz);
        RT_TRY(launch_prop32(h->n, a, hz, h->stream));
        RT_TRY(launch_row_diffract_plain32(h->logn, static_cast<const float2 *>(h->E), X, tw, hz, h->stream));
        RT_TRY(launch_col_diffract_plain32(h->logn, X, tw, hz, h->stream));
    } else {
        const double2 *tw = static_cast<const double2 *>(h->tw);
        double2 *X = static_cast<double2 *>(h->X), *hz = static_cast<double2 *>(h->hz);
        RT_TRY(launch_prop64(h->n, a, hz, h->stream));
        RT_TRY(launch_row_diffract_plain64(h->logn, static_cast<const double2 *>(h->E), X, tw, hz, h->stream));
        RT_TRY(launch_col_diffract_plain64(h->logn, X, tw, hz, h->stream));
    }
    RT_TRY(cudaMemcpyAsync(dst, h->X, bytes, cudaMemcpyDefault, h->stream));
    return check_device_error(h);
}

rt_status rt_spectrum_peak(rt_handle *h, int ring, int *mx, int *my, double *power)
{
    if (!h || !mx || !my || !power || ring < 0) return RT_EINVAL;
    DeviceGuard dg(h->device);
    rt_status st = compute_spectrum(h);
    if (st != RT_OK) return st;
    PeakResult *d_out = &h->ctl->peak;
    unsigned int *cnt = &h->ctl->peak_count;
    if (h->precision == RT_FP32)
        RT_TRY(launch_peak32(h->n, ring, static_cast<const float *>(h->S), h->peak_val, h->peak_idx, cnt, d_out, h->stream));
    else
        RT_TRY(launch_peak64(h->n, ring, static_cast<const double *>(h->S), h->peak_val, h->peak_idx, cnt, d_out, h->stream));
    PeakResult r;
    RT_TRY(cudaMemcpyAsync(&r, d_out, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
    st = check_device_error(h);
    if (st != RT_OK) return st;
    if (r.value < 0.0) {
        *mx = 0;
        *my = 0;
        *power = 0.0;
        return RT_OK;
    }
    const int n = h->n;
    const int kx = (int)(r.index % n), ky = (int)(r.index / n);
    *mx = kx < n / 2 ? kx : kx - n;
    *my = ky < n / 2 ? ky : ky - n;
    *power = r.value;
    return RT_OK;
}

rt_status rt_destroy(rt_handle *h)
{
    if (!h) return RT_OK;
    DeviceGuard dg(h->device);
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
    return RT_OK;
}

}  // extern "C"
