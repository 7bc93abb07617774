// Batches of resonators (include/rt.h, rt_batch_*): slots grouped by grid
// size; each bounce is one batched column sweep and one batched row sweep per
// size class, captured as CUDA graphs of `chunk` bounces.  Each slot carries
// a stop-at-bounce target that the kernels honour, so slots with different
// remaining work (the serving loop) share the same launches and graphs.
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "rt.h"
#include "rt_internal.h"

using namespace rtk;

namespace {

// Per-slot device counters (one 64-byte line each).
struct SlotCtl {
    unsigned int count;  // arrival counter of the row-sweep reduction
    int err;             // sticky error (RT_ENUMERIC)
    long long bounce;    // bounces done since the slot's job started
    double last_mean;    // mean intensity after the last bounce
    long long pad[5];
};
static_assert(sizeof(SlotCtl) == 64, "slot control block is one line");

struct Slot {
    rt_job job{};
    int logn = 0, pe = 0, cls = -1, idx = -1;
    double alpha = 0.0;
    long long target = LLONG_MAX;
    unsigned char *mem = nullptr;  // one allocation holding the buffers below
    size_t bytes = 0;
    float2 *E = nullptr;
    float *N = nullptr;
    float2 *h = nullptr;
    double *part = nullptr;
    double *hist = nullptr;
    CUtensorMap *tmap = nullptr;
    float *pump_tab = nullptr;
};

struct SizeClass {
    int logn = 0, colC = 4;
    std::vector<int> slots;
    BatchRes *d_res = nullptr;
    float2 *tw = nullptr;
};

size_t al256(size_t b) { return (b + 255) / 256 * 256; }
bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
bool fpos(double v) { return std::isfinite(v) && v > 0.0; }

int log2i(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

rt_status cuda_status(cudaError_t e)
{
    return e == cudaSuccess ? RT_OK : (e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA);
}

#define BT_TRY(x)                                   \
    do {                                            \
        cudaError_t e_ = (x);                       \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

bool job_ok(const rt_job &j)
{
    if (!pow2(j.n) || j.n < 32 || j.n > 2048) return false;
    if (!fpos(j.fresnel) || !std::isfinite(j.g0) || j.g0 < 0.0 || !std::isfinite(j.T1) || j.T1 < 1.0) return false;
    if (!std::isfinite(j.R) || j.R <= 0.0 || j.R > 1.0) return false;
    if (!fpos(j.Isat) || j.edge_px < 0 || j.edge_px > j.n / 2 || !fpos(j.pump_diam_over_window)) return false;
    if (!std::isfinite(j.noise_amp) || j.noise_amp < 0.0) return false;
    if (j.pump.kind < RT_PUMP_SUPERGAUSS || j.pump.kind > RT_PUMP_ARRAY) return false;
    if (j.pump.kind == RT_PUMP_SUPERGAUSS && (!fpos(j.pump.order) || !fpos(j.pump.radius))) return false;
    if (j.pump.kind == RT_PUMP_ARRAY && !j.pump.profile) return false;
    return true;
}

int pump_eval(const rt_pump &p)
{
    return p.kind == RT_PUMP_UNIFORM ? PE_UNIFORM
                                     : ((p.kind == RT_PUMP_SUPERGAUSS && p.order == 10.0) ? PE_SG10 : PE_TABLE);
}

}  // namespace

struct rt_batch {
    int device = 0;
    rt_opts opts{};
    cudaStream_t stream = nullptr, capture = nullptr;
    std::vector<Slot> slots;
    std::vector<SizeClass> classes;
    SlotCtl *ctl = nullptr;  // one per slot
    int *err = nullptr;      // batch-wide error word (copy-engine timeouts)
    size_t shared_bytes = 0;
    std::map<long long, cudaGraphExec_t> graphs;
};

namespace {

// Carve the slot's buffers out of one allocation.
rt_status alloc_slot(rt_batch *b, Slot &s)
{
    const size_t n = (size_t)s.job.n, P = n * n;
    const size_t cap = b->opts.history_cap > 0 ? (size_t)b->opts.history_cap : 0;
    size_t off[8], sz[8];
    sz[0] = al256(P * sizeof(float2));                           // E
    sz[1] = al256(P * sizeof(float));                            // N
    sz[2] = al256(n * sizeof(float2));                           // h
    sz[3] = al256((size_t)row_groups32(s.logn) * sizeof(double));  // part
    sz[4] = al256(cap * sizeof(double));                         // hist
    sz[5] = al256(sizeof(CUtensorMap));                          // tensor map
    sz[6] = s.pe == PE_TABLE ? al256(P * sizeof(float)) : 0;     // N0 table
    size_t total = 0;
    for (int k = 0; k < 7; ++k) {
        off[k] = total;
        total += sz[k];
    }
    BT_TRY(cudaMalloc(&s.mem, total));
    s.bytes = total;
    s.E = reinterpret_cast<float2 *>(s.mem + off[0]);
    s.N = reinterpret_cast<float *>(s.mem + off[1]);
    s.h = reinterpret_cast<float2 *>(s.mem + off[2]);
    s.part = reinterpret_cast<double *>(s.mem + off[3]);
    s.hist = cap ? reinterpret_cast<double *>(s.mem + off[4]) : nullptr;
    s.tmap = reinterpret_cast<CUtensorMap *>(s.mem + off[5]);
    s.pump_tab = sz[6] ? reinterpret_cast<float *>(s.mem + off[6]) : nullptr;
    return RT_OK;
}

BatchRes descriptor(rt_batch *b, int i)
{
    const Slot &s = b->slots[i];
    BatchRes r{};
    r.E = s.E;
    r.N = s.N;
    r.h = s.h;
    r.tmap = s.tmap;
    GainParams<float> &g = r.g;
    g.sqrtR = (float)std::sqrt(s.job.R);
    g.invT1 = (float)(1.0 / s.job.T1);
    g.invIsat = (float)(1.0 / s.job.Isat);
    g.g0 = (float)s.job.g0;
    g.inv_rp2 = s.job.pump.kind == RT_PUMP_SUPERGAUSS ? (float)(1.0 / (s.job.pump.radius * s.job.pump.radius)) : 0.0f;
    g.half_order = (float)(0.5 * s.job.pump.order);
    g.int_half_order = s.pe == PE_SG10 ? 5 : 0;
    g.edge = s.job.edge_px;
    g.pump_kind = s.job.pump.kind;
    g.pump_tab = s.pump_tab;
    r.pe = s.pe;
    r.target = s.target;
    r.st.part = s.part;
    r.st.count = &b->ctl[i].count;
    r.st.hist = s.hist;
    r.st.hist_cap = s.hist ? b->opts.history_cap : 0;
    r.st.bounce = &b->ctl[i].bounce;
    r.st.last_mean = &b->ctl[i].last_mean;
    r.st.err = &b->ctl[i].err;
    return r;
}

// Initial state of slot i (as rt_create): tables, noise field, N = N0,
// tensor map, zeroed counters, descriptor.
rt_status init_slot(rt_batch *b, int i)
{
    Slot &s = b->slots[i];
    const int n = s.job.n;
    const size_t P = (size_t)n * n;
    cudaStream_t st = b->stream;
    SizeClass &c = b->classes[s.cls];
    BT_TRY(launch_tables32(n, s.alpha, c.tw, s.h, st));
    BT_TRY(launch_noise32(n, s.job.seed, s.job.noise_amp, s.E, st));
    double *profile = nullptr;
    if (s.job.pump.kind == RT_PUMP_ARRAY) {
        BT_TRY(cudaMallocAsync(reinterpret_cast<void **>(&profile), P * sizeof(double), st));
        BT_TRY(cudaMemcpyAsync(profile, s.job.pump.profile, P * sizeof(double), cudaMemcpyDefault, st));
    }
    BT_TRY(launch_pump32(n, s.job.pump.kind, s.job.g0, s.job.pump.order, s.job.pump.radius, profile, s.N, st));
    if (profile) BT_TRY(cudaFreeAsync(profile, st));
    if (s.pump_tab) BT_TRY(cudaMemcpyAsync(s.pump_tab, s.N, P * sizeof(float), cudaMemcpyDeviceToDevice, st));
    alignas(64) unsigned char map[128];
    BT_TRY(make_col_tensor_map(map, s.E, n, c.colC));
    BT_TRY(cudaMemcpyAsync(s.tmap, map, sizeof(map), cudaMemcpyHostToDevice, st));
    BT_TRY(cudaMemsetAsync(&b->ctl[i], 0, sizeof(SlotCtl), st));
    const BatchRes r = descriptor(b, i);
    BT_TRY(cudaMemcpyAsync(c.d_res + s.idx, &r, sizeof(r), cudaMemcpyHostToDevice, st));
    return RT_OK;
}

void release(rt_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    for (Slot &s : b->slots)
        if (s.mem) cudaFree(s.mem);
    for (SizeClass &c : b->classes) {
        if (c.d_res) cudaFree(c.d_res);
        if (c.tw) cudaFree(c.tw);
    }
    if (b->ctl) cudaFree(b->ctl);
    if (b->err) cudaFree(b->err);
    if (b->capture) cudaStreamDestroy(b->capture);
}

cudaError_t enqueue_batch_bounce(rt_batch *b, cudaStream_t st)
{
    cudaError_t e;
    for (SizeClass &c : b->classes)
        if ((e = launch_col_batch32(c.logn, c.colC, c.d_res, (int)c.slots.size(), c.tw, b->err, st)) != cudaSuccess)
            return e;
    for (SizeClass &c : b->classes)
        if ((e = launch_row_batch32(c.logn, c.d_res, (int)c.slots.size(), c.tw, b->err, st)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t batch_graph(rt_batch *b, long long k, cudaGraphExec_t *out)
{
    auto it = b->graphs.find(k);
    if (it != b->graphs.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaError_t e;
    for (SizeClass &c : b->classes)
        if ((e = prepare_batch32(c.logn, c.colC)) != cudaSuccess) return e;
    if ((e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (long long i = 0; i < k && le == cudaSuccess; ++i) le = enqueue_batch_bounce(b, b->capture);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->capture, &g);
    if (le != cudaSuccess) e = le;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    b->graphs[k] = ge;
    *out = ge;
    return cudaSuccess;
}

rt_status check_errors(rt_batch *b)
{
    std::vector<SlotCtl> c(b->slots.size());
    int err = 0;
    BT_TRY(cudaMemcpyAsync(&err, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    if (!c.empty()) BT_TRY(cudaMemcpyAsync(c.data(), b->ctl, c.size() * sizeof(SlotCtl), cudaMemcpyDeviceToHost, b->stream));
    BT_TRY(cudaStreamSynchronize(b->stream));
    if (err) return (rt_status)err;
    for (const SlotCtl &x : c)
        if (x.err) return (rt_status)x.err;
    return RT_OK;
}

struct Guard {
    int prev = -1, want;
    explicit Guard(int d) : want(d)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != want) cudaSetDevice(want);
    }
    ~Guard()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

rt_status rt_job_default(rt_job *job, int n)
{
    if (!job) return RT_EINVAL;
    std::memset(job, 0, sizeof(*job));
    rt_opts o;
    rt_opts_default(&o);
    job->n = n;
    job->fresnel = 100.0;
    job->g0 = 0.2;
    job->T1 = 1000.0;
    job->R = 0.95;
    job->pump.kind = RT_PUMP_SUPERGAUSS;
    job->pump.order = 10.0;
    job->pump.radius = 0.8;
    job->pump.profile = nullptr;
    job->Isat = o.Isat;
    job->edge_px = o.edge_px;
    job->seed = o.seed;
    job->noise_amp = o.noise_amp;
    job->pump_diam_over_window = o.pump_diam_over_window;
    return RT_OK;
}

rt_status rt_batch_create(const rt_job *jobs, int count, const rt_opts *opts, rt_batch **out)
{
    if (!out || !jobs || count <= 0) return RT_EINVAL;
    *out = nullptr;
    rt_opts o;
    if (opts) o = *opts;
    else rt_opts_default(&o);
    if (o.precision != RT_FP32 || o.history_cap < 0 || o.chunk < 0) return RT_EINVAL;
    for (int i = 0; i < count; ++i)
        if (!job_ok(jobs[i])) return RT_EINVAL;
    rt_batch *b = new (std::nothrow) rt_batch();
    if (!b) return RT_ENOMEM;
    b->opts = o;
    b->stream = static_cast<cudaStream_t>(o.cuda_stream);
    cudaGetDevice(&b->device);
    auto fail = [&](rt_status s) {
        release(b);
        delete b;
        return s;
    };
    b->slots.resize(count);
    std::map<int, int> class_of;  // logn -> class index
    for (int i = 0; i < count; ++i) {
        Slot &s = b->slots[i];
        s.job = jobs[i];
        s.job.pump.profile = jobs[i].pump.profile;
        s.logn = log2i(s.job.n);
        s.pe = pump_eval(s.job.pump);
        s.alpha = s.job.pump_diam_over_window * s.job.pump_diam_over_window / s.job.fresnel;
        auto it = class_of.find(s.logn);
        if (it == class_of.end()) {
            SizeClass c;
            c.logn = s.logn;
            c.colC = o.col_tile ? o.col_tile : default_col_tile32(s.logn);
            if (!col_tile_ok32(s.logn, c.colC)) return fail(RT_EINVAL);
            it = class_of.emplace(s.logn, (int)b->classes.size()).first;
            b->classes.push_back(c);
        }
        s.cls = it->second;
        s.idx = (int)b->classes[s.cls].slots.size();
        b->classes[s.cls].slots.push_back(i);
    }
    if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) return fail(RT_ECUDA);
    if (cudaMalloc(&b->ctl, sizeof(SlotCtl) * count) != cudaSuccess) return fail(RT_ENOMEM);
    if (cudaMalloc(&b->err, sizeof(int)) != cudaSuccess) return fail(RT_ENOMEM);
    if (cudaMemsetAsync(b->err, 0, sizeof(int), b->stream) != cudaSuccess) return fail(RT_ECUDA);
    b->shared_bytes = sizeof(SlotCtl) * count + sizeof(int);
    for (SizeClass &c : b->classes) {
        if (cudaMalloc(&c.d_res, sizeof(BatchRes) * c.slots.size()) != cudaSuccess) return fail(RT_ENOMEM);
        if (cudaMalloc(&c.tw, sizeof(float2) * (twiddle_entries(c.logn) + 1)) != cudaSuccess) return fail(RT_ENOMEM);
        b->shared_bytes += sizeof(BatchRes) * c.slots.size() + sizeof(float2) * (twiddle_entries(c.logn) + 1);
    }
    for (int i = 0; i < count; ++i) {
        rt_status st = alloc_slot(b, b->slots[i]);
        if (st != RT_OK) return fail(st);
        if ((st = init_slot(b, i)) != RT_OK) return fail(st);
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(RT_ECUDA);
    *out = b;
    return RT_OK;
}

rt_status rt_batch_step(rt_batch *b, long long nb)
{
    if (!b || nb < 0) return RT_EINVAL;
    if (nb == 0) return RT_OK;
    Guard g(b->device);
    const long long K = b->opts.chunk;
    long long left = nb;
    if (K > 0 && left >= K) {
        cudaGraphExec_t ge;
        BT_TRY(batch_graph(b, K, &ge));
        for (; left >= K; left -= K) BT_TRY(cudaGraphLaunch(ge, b->stream));
    }
    for (; left > 0; --left) BT_TRY(enqueue_batch_bounce(b, b->stream));
    return RT_OK;
}

rt_status rt_batch_sweep(rt_batch *b, int which)
{
    if (!b || (which != RT_SWEEP_COLUMNS && which != RT_SWEEP_ROWS)) return RT_EINVAL;
    Guard g(b->device);
    for (SizeClass &c : b->classes) {
        if (which == RT_SWEEP_COLUMNS)
            BT_TRY(launch_col_batch32(c.logn, c.colC, c.d_res, (int)c.slots.size(), c.tw, b->err, b->stream));
        else
            BT_TRY(launch_row_batch32(c.logn, c.d_res, (int)c.slots.size(), c.tw, b->err, b->stream));
    }
    return RT_OK;
}

rt_status rt_batch_set_job(rt_batch *b, int i, const rt_job *job, long long n_bounces)
{
    if (!b || !job || i < 0 || i >= (int)b->slots.size() || !job_ok(*job)) return RT_EINVAL;
    Slot &s = b->slots[i];
    if (job->n != s.job.n || pump_eval(job->pump) == PE_TABLE) {
        // A different size needs another slot; a table pump needs a table sized at creation.
        if (job->n != s.job.n || !s.pump_tab) return RT_EINVAL;
    }
    Guard g(b->device);
    s.job = *job;
    s.pe = pump_eval(job->pump);
    s.alpha = job->pump_diam_over_window * job->pump_diam_over_window / job->fresnel;
    s.target = n_bounces < 0 ? LLONG_MAX : n_bounces;
    return init_slot(b, i);
}

rt_status rt_batch_sync(rt_batch *b)
{
    if (!b) return RT_EINVAL;
    Guard g(b->device);
    return check_errors(b);
}

static rt_status batch_copy(rt_batch *b, int i, void *dst, const void *src, size_t bytes, size_t want, bool out)
{
    if (!b || i < 0 || i >= (int)b->slots.size() || !dst || !src || bytes != want) return RT_EINVAL;
    Guard g(b->device);
    BT_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, b->stream));
    return out ? check_errors(b) : RT_OK;
}

rt_status rt_batch_read_field(rt_batch *b, int i, void *dst, size_t bytes)
{
    if (!b || i < 0 || i >= (int)b->slots.size()) return RT_EINVAL;
    const size_t P = (size_t)b->slots[i].job.n * b->slots[i].job.n;
    return batch_copy(b, i, dst, b->slots[i].E, bytes, P * sizeof(float2), true);
}

rt_status rt_batch_read_inversion(rt_batch *b, int i, void *dst, size_t bytes)
{
    if (!b || i < 0 || i >= (int)b->slots.size()) return RT_EINVAL;
    const size_t P = (size_t)b->slots[i].job.n * b->slots[i].job.n;
    return batch_copy(b, i, dst, b->slots[i].N, bytes, P * sizeof(float), true);
}

rt_status rt_batch_write_field(rt_batch *b, int i, const void *src, size_t bytes)
{
    if (!b || i < 0 || i >= (int)b->slots.size()) return RT_EINVAL;
    const size_t P = (size_t)b->slots[i].job.n * b->slots[i].job.n;
    return batch_copy(b, i, b->slots[i].E, src, bytes, P * sizeof(float2), false);
}

rt_status rt_batch_write_inversion(rt_batch *b, int i, const void *src, size_t bytes)
{
    if (!b || i < 0 || i >= (int)b->slots.size()) return RT_EINVAL;
    const size_t P = (size_t)b->slots[i].job.n * b->slots[i].job.n;
    return batch_copy(b, i, b->slots[i].N, src, bytes, P * sizeof(float), false);
}

rt_status rt_batch_stats(rt_batch *b, int i, rt_stats_t *out)
{
    if (!b || !out || i < 0 || i >= (int)b->slots.size()) return RT_EINVAL;
    Guard g(b->device);
    SlotCtl c;
    BT_TRY(cudaMemcpyAsync(&c, &b->ctl[i], sizeof(c), cudaMemcpyDeviceToHost, b->stream));
    BT_TRY(cudaStreamSynchronize(b->stream));
    const Slot &s = b->slots[i];
    std::memset(out, 0, sizeof(*out));
    out->bounces = c.bounce;
    out->mean_intensity = c.last_mean;
    out->alpha = s.alpha;
    out->n = s.job.n;
    out->precision = RT_FP32;
    out->last_error = c.err;
    const long long cap = s.hist ? b->opts.history_cap : 0;
    out->history_len = cap > 0 ? (c.bounce < cap ? c.bounce : cap) : 0;
    return RT_OK;
}

rt_status rt_batch_read_history(rt_batch *b, int i, double *dst, long long max, long long *got)
{
    if (!b || !got || max < 0 || (max > 0 && !dst) || i < 0 || i >= (int)b->slots.size()) return RT_EINVAL;
    *got = 0;
    rt_stats_t s;
    rt_status st = rt_batch_stats(b, i, &s);
    if (st != RT_OK) return st;
    const long long cap = b->opts.history_cap;
    const long long len = s.history_len < max ? s.history_len : max;
    if (len <= 0 || cap <= 0) return RT_OK;
    Guard g(b->device);
    const long long first = s.bounces - len;
    long long done = 0;
    while (done < len) {
        const long long slot = (first + done) % cap;
        long long run = cap - slot;
        if (run > len - done) run = len - done;
        BT_TRY(cudaMemcpy(dst + done, b->slots[i].hist + slot, sizeof(double) * (size_t)run, cudaMemcpyDeviceToHost));
        done += run;
    }
    *got = len;
    return RT_OK;
}

rt_status rt_batch_bounces(rt_batch *b, long long *counts)
{
    if (!b || !counts) return RT_EINVAL;
    Guard g(b->device);
    std::vector<SlotCtl> c(b->slots.size());
    BT_TRY(cudaMemcpyAsync(c.data(), b->ctl, c.size() * sizeof(SlotCtl), cudaMemcpyDeviceToHost, b->stream));
    BT_TRY(cudaStreamSynchronize(b->stream));
    for (size_t k = 0; k < c.size(); ++k) counts[k] = c[k].bounce;
    return RT_OK;
}

rt_status rt_batch_footprint(rt_batch *b, size_t *bytes)
{
    if (!b || !bytes) return RT_EINVAL;
    size_t t = b->shared_bytes;
    for (const Slot &s : b->slots) t += s.bytes;
    *bytes = t;
    return RT_OK;
}

rt_status rt_batch_destroy(rt_batch *b)
{
    if (!b) return RT_OK;
    Guard g(b->device);
    cudaStreamSynchronize(b->stream);
    release(b);
    delete b;
    return RT_OK;
}

}  // extern "C"
