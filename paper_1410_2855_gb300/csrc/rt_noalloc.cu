// rt_step_noalloc: the fused FP32 bounce on caller-owned field and inversion
// buffers, with every piece of scratch memory taken from one fixed-size
// device array declared in this file instead of being allocated.
//
// Scratch layout (g_noalloc_scratch, kScratchBytes per device):
//   [0, 256)                  control block: reduction arrival counter,
//                             sticky error word, bounce counter, last mean
//   [256, +kMaxN*8)           per-axis propagator table h (n complex64)
//   [.., +kTwMax*8)           pass-major twiddle table (complex64)
//   [.., +kPartMax*8)         block partial sums of the mean intensity
//   [.., +kMaxN*8)            per-axis curved-mirror factors (n complex64)
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "rt.h"
#include "rt_internal.h"

namespace {

constexpr int kMaxN = RT_NOALLOC_MAX_N;
constexpr size_t kCtlBytes = 256;
constexpr size_t kHBytes = (size_t)kMaxN * sizeof(float2);
constexpr size_t kTwMax = 4096;    // >= twiddle_entries(log2 n) for n <= 4096
constexpr size_t kPartMax = 4096;  // >= blocks of any row-sweep launch
constexpr size_t kTwBytes = kTwMax * sizeof(float2);
constexpr size_t kPartBytes = kPartMax * sizeof(double);
constexpr size_t kLensBytes = (size_t)kMaxN * sizeof(float2);
constexpr size_t kScratchBytes = kCtlBytes + kHBytes + kTwBytes + kPartBytes + kLensBytes;

// The counters come first and are cleared by every call; the sticky error
// word comes last and is cleared only once a synchronous call has reported it.
struct NoAllocCtl {
    unsigned int count;
    unsigned int pad;
    long long bounce;
    double last_mean;
    int err;
};
constexpr size_t kCountersBytes = offsetof(NoAllocCtl, err);
static_assert(sizeof(NoAllocCtl) <= kCtlBytes, "control block");

}  // namespace

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// Device address of the scratch array.  In host code the array's name only
// denotes a host-side stand-in, so kernels must be given the address that
// cudaGetSymbolAddress reports with the device current.  It is looked up once
// per CUDA context: a context created after cudaDeviceReset gets a new id
// (cuCtxGetId), and with it a fresh lookup instead of a stale address.
std::mutex g_addr_mutex;
struct ScratchAddr {
    unsigned long long ctx_id;
    void *ptr;
};
ScratchAddr g_addr[64] = {};

using PFN_ctx_current = CUresult (*)(CUcontext *);
using PFN_ctx_id = CUresult (*)(CUcontext, unsigned long long *);

// Id of the calling thread's current context (made current by the runtime).
rt_status current_context_id(int dev, unsigned long long *id)
{
    static PFN_ctx_current get_current = nullptr;
    static PFN_ctx_id get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || !f1)
            return RT_ECUDA;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess || !f2)
            return RT_ECUDA;
        get_current = reinterpret_cast<PFN_ctx_current>(f1);
        get_id = reinterpret_cast<PFN_ctx_id>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return RT_ECUDA;
    if (!ctx) {  // nothing current yet: the runtime makes the device's primary context current
        if (cudaSetDevice(dev) != cudaSuccess || get_current(&ctx) != CUDA_SUCCESS || !ctx) return RT_ECUDA;
    }
    return get_id(ctx, id) == CUDA_SUCCESS ? RT_OK : RT_ECUDA;
}

rt_status scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= 64) return RT_ECUDA;
    unsigned long long ctx = 0;
    rt_status st = current_context_id(dev, &ctx);
    if (st != RT_OK) return st;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev].ptr || g_addr[dev].ctx_id != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RT_ECUDA;
        g_addr[dev] = {ctx, p};
    }
    *out = static_cast<unsigned char *>(g_addr[dev].ptr);
    return RT_OK;
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
bool fpos(double v) { return std::isfinite(v) && v > 0.0; }

int log2i(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

}  // namespace

extern "C" rt_status rt_step_noalloc(int n, double fresnel, const rt_pump *pump, double g0, double T1, double R,
                                     const rt_opts *opts, void *field, void *inversion, long long n_bounces,
                                     double *mean_intensity)
{
    rt_opts o;
    if (opts) o = *opts;
    else rt_opts_default(&o);
    rt_pump p{RT_PUMP_SUPERGAUSS, 10.0, 0.8, nullptr};
    if (pump) p = *pump;
    if (!pow2(n) || n < 32 || n > kMaxN) return RT_EINVAL;
    if (!fpos(fresnel) || !std::isfinite(g0) || g0 < 0.0 || !std::isfinite(T1) || T1 < 1.0) return RT_EINVAL;
    if (!std::isfinite(R) || R <= 0.0 || R > 1.0 || n_bounces < 0) return RT_EINVAL;
    if (!fpos(o.Isat) || o.edge_px < 0 || o.edge_px > n / 2 || !fpos(o.pump_diam_over_window)) return RT_EINVAL;
    if (o.precision != RT_FP32 || !std::isfinite(o.z_over_F) || o.roughness || o.slices > 1) return RT_EINVAL;
    if (o.taper_px < 0 || o.taper_px > n / 2 || (o.relax != RT_RELAX_EULER && o.relax != RT_RELAX_EXACT))
        return RT_EINVAL;
    const bool sg10 = p.kind == RT_PUMP_SUPERGAUSS && p.order == 10.0 && fpos(p.radius);
    if (!sg10 && p.kind != RT_PUMP_UNIFORM) return RT_EINVAL;
    if (!field || !inversion) return RT_EINVAL;
    if ((reinterpret_cast<uintptr_t>(field) & 15) || (reinterpret_cast<uintptr_t>(inversion) & 15)) return RT_EINVAL;
    const int logn = log2i(n);
    const int colC = o.col_tile ? o.col_tile : rtk::default_col_tile32(logn);
    if (!rtk::col_tile_ok32(logn, colC)) return RT_EINVAL;
    // the same twiddle_entries + 1 slots as the handle, batch and serve paths
    if ((size_t)rtk::twiddle_entries(logn) + 1 > kTwMax || (size_t)rtk::row_blocks32(logn) > kPartMax) return RT_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RT_ECUDA;
    unsigned char *base = nullptr;
    rt_status st = scratch_address(dev, &base);
    if (st != RT_OK) return st;
    NoAllocCtl *ctl = reinterpret_cast<NoAllocCtl *>(base);
    float2 *h = reinterpret_cast<float2 *>(base + kCtlBytes);
    float2 *tw = reinterpret_cast<float2 *>(base + kCtlBytes + kHBytes);
    double *part = reinterpret_cast<double *>(base + kCtlBytes + kHBytes + kTwBytes);
    float2 *lens = reinterpret_cast<float2 *>(base + kCtlBytes + kHBytes + kTwBytes + kPartBytes);

    cudaStream_t s = static_cast<cudaStream_t>(o.cuda_stream);
    float2 *E = static_cast<float2 *>(field);
    float *N = static_cast<float *>(inversion);
    const double alpha = o.pump_diam_over_window * o.pump_diam_over_window / fresnel;
    alignas(64) unsigned char tmap[128];
    if (rtk::make_col_tensor_map(tmap, E, n, colC) != cudaSuccess) return RT_ECUDA;

    // The array keeps whatever the previous call left: the counters must
    // start at zero.  The error word is kept, so that an error of an
    // asynchronous call is still there for the next synchronous one.
    if (cudaMemsetAsync(ctl, 0, kCountersBytes, s) != cudaSuccess) return RT_ECUDA;
    if (rtk::launch_tables32(n, alpha, tw, h, s) != cudaSuccess) return RT_ECUDA;
    // per-axis aperture factors: curved mirror, taper, or the general local map (exact update)
    const bool curved = o.z_over_F != 0.0 || o.taper_px > 0 || o.relax == RT_RELAX_EXACT;
    if (curved &&
        rtk::launch_lens32(n, rtk::lens_curvature(alpha, o.z_over_F), o.edge_px, o.taper_px, lens, s) != cudaSuccess)
        return RT_ECUDA;

    rtk::GainParams<float> g{};
    g.sqrtR = (float)std::sqrt(R);
    g.invT1 = (float)(1.0 / T1);
    g.invIsat = (float)(1.0 / o.Isat);
    g.g0 = (float)g0;
    g.inv_rp2 = sg10 ? (float)(1.0 / (p.radius * p.radius)) : 0.0f;
    g.half_order = 5.0f;
    g.int_half_order = 5;
    g.edge = o.edge_px;
    g.pump_kind = p.kind;
    g.pump_tab = nullptr;
    g.lens = curved ? lens : nullptr;
    g.phase = nullptr;
    g.relax_exact = o.relax == RT_RELAX_EXACT;
    rtk::StatParams sp{};
    sp.part = part;
    sp.count = &ctl->count;
    sp.hist = nullptr;
    sp.hist_cap = 0;
    sp.bounce = &ctl->bounce;
    sp.last_mean = &ctl->last_mean;
    sp.err = &ctl->err;
    const int pe = sg10 ? 0 : 1;
    for (long long b = 0; b < n_bounces; ++b) {
        if (rtk::launch_col_diffract32(logn, colC, E, tw, h, tmap, &ctl->err, s) != cudaSuccess) return RT_ECUDA;
        if (rtk::launch_row_diffract_gain32(logn, pe, E, N, tw, h, g, sp, s) != cudaSuccess) return RT_ECUDA;
    }
    if (!mean_intensity) return RT_OK;
    NoAllocCtl c;
    if (cudaMemcpyAsync(&c, ctl, sizeof(c), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RT_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RT_ECUDA;
    if (c.err) {  // reported once: clear it for the calls that follow
        if (cudaMemsetAsync(&ctl->err, 0, sizeof(int), s) != cudaSuccess) return RT_ECUDA;
        return (rt_status)c.err;
    }
    *mean_intensity = n_bounces > 0 ? c.last_mean : 0.0;
    return RT_OK;
}
