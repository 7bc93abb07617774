// Batches of resonators (include/rt.h, rt_batch_*): slots grouped by grid
// size; each bounce is one batched column sweep and one batched row sweep per
// size class, captured as CUDA graphs of `chunk` bounces with one or more
// chains per size class on graph branches (batch_split; their launches
// overlap).  Each slot carries
// a stop-at-bounce target that the kernels honour, so slots with different
// remaining work share the same launches and graphs.
#include <climits>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "engine.h"
#include "trace.h"

using namespace rtk;

namespace {

struct Slot {
    rt_job job{};
    int cls = -1, idx = -1;
    long long target = LLONG_MAX;
    SlotBufs buf;
};

struct SizeClass {
    int logn = 0, colC = 4;
    bool mixed = false;  // runs in the launches shared across sizes
    int order = 0;       // radix order of the column transforms
    float2 *tw_col = nullptr;  // that order's twiddles (order != 0)
    std::vector<int> slots;
    BatchRes *d_res = nullptr;
    float2 *tw = nullptr;
};

#define BT_TRY(x)                                         \
    do {                                                  \
        cudaError_t e_ = (x);                             \
        if (e_ != cudaSuccess) return cuda_to_status(e_); \
    } while (0)

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
    Branches branches;       // one graph branch per size class
};

namespace {

long long hist_cap(const rt_batch *b) { return b->opts.history_cap > 0 ? b->opts.history_cap : 0; }

cudaError_t start_slot(rt_batch *b, int i)
{
    Slot &s = b->slots[i];
    SizeClass &c = b->classes[s.cls];
    return slot_start(s.job, s.buf, c.colC, c.tw, &b->ctl[i], c.d_res + s.idx, hist_cap(b), s.target, b->stream);
}

std::vector<ClassLaunch> launches(rt_batch *b)
{
    std::vector<ClassLaunch> v;
    for (SizeClass &c : b->classes)
        v.push_back({c.logn, c.colC, c.d_res, (int)c.slots.size(), c.tw, c.mixed, c.order, c.tw_col});
    return v;
}

void release(rt_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    for (Slot &s : b->slots) slot_free(&s.buf);
    for (SizeClass &c : b->classes) {
        if (c.d_res) cudaFree(c.d_res);
        if (c.tw) cudaFree(c.tw);
        if (c.tw_col) cudaFree(c.tw_col);
    }
    if (b->ctl) cudaFree(b->ctl);
    if (b->err) cudaFree(b->err);
    if (b->capture) cudaStreamDestroy(b->capture);
    branches_free(b->branches);
}

cudaError_t batch_graph(rt_batch *b, long long k, cudaGraphExec_t *out)
{
    auto it = b->graphs.find(k);
    if (it != b->graphs.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaError_t e;
    const std::vector<ClassLaunch> cl = launches(b);
    if ((e = prepare_classes(cl)) != cudaSuccess) return e;
    const int split = batch_split(cl);
    if ((e = branches_prepare(b->branches, cl, split)) != cudaSuccess) return e;
    if ((e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    const cudaError_t le = capture_class_bounces(cl, b->err, k, b->capture, b->branches, split);
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
    if (!c.empty())
        BT_TRY(cudaMemcpyAsync(c.data(), b->ctl, c.size() * sizeof(SlotCtl), cudaMemcpyDeviceToHost, b->stream));
    BT_TRY(cudaStreamSynchronize(b->stream));
    if (err) return (rt_status)err;
    for (const SlotCtl &x : c)
        if (x.err) return (rt_status)x.err;
    return RT_OK;
}

bool valid_slot(const rt_batch *b, int i) { return b && i >= 0 && i < (int)b->slots.size(); }

size_t field_bytes(const rt_batch *b, int i)
{
    return (size_t)b->slots[i].job.n * b->slots[i].job.n * sizeof(float2);
}

size_t inv_bytes(const rt_batch *b, int i) { return (size_t)b->slots[i].job.n * b->slots[i].job.n * sizeof(float); }

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
    if (o.precision != RT_FP32 || o.history_cap < 0 || o.chunk < 0 || o.slices > 1) return RT_EINVAL;
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
    std::map<int, int> class_of;  // log2 n -> class index
    for (int i = 0; i < count; ++i) {
        Slot &s = b->slots[i];
        s.job = jobs[i];
        const int logn = log2_of(s.job.n);
        auto it = class_of.find(logn);
        if (it == class_of.end()) {
            SizeClass c;
            c.logn = logn;
            c.colC = class_col_tile(logn, o.col_tile, &c.mixed);
            if (!c.mixed && !col_tile_ok32(logn, c.colC)) return fail(RT_EINVAL);
            c.order = class_col_order(logn, c.colC, o.col_tile, c.mixed);
            it = class_of.emplace(logn, (int)b->classes.size()).first;
            b->classes.push_back(c);
        }
        s.cls = it->second;
        s.idx = (int)b->classes[s.cls].slots.size();
        b->classes[s.cls].slots.push_back(i);
    }
    if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) return fail(RT_ECUDA);
    if (dev_alloc(&b->ctl, sizeof(SlotCtl) * count) != cudaSuccess) return fail(RT_ENOMEM);
    if (dev_alloc(&b->err, sizeof(int)) != cudaSuccess) return fail(RT_ENOMEM);
    if (cudaMemsetAsync(b->err, 0, sizeof(int), b->stream) != cudaSuccess) return fail(RT_ECUDA);
    b->shared_bytes = sizeof(SlotCtl) * count + sizeof(int);
    for (SizeClass &c : b->classes) {
        const size_t twb = sizeof(float2) * (twiddle_entries(c.logn) + 1);
        if (dev_alloc(&c.d_res, sizeof(BatchRes) * c.slots.size()) != cudaSuccess) return fail(RT_ENOMEM);
        if (dev_alloc(&c.tw, twb) != cudaSuccess) return fail(RT_ENOMEM);
        b->shared_bytes += sizeof(BatchRes) * c.slots.size() + twb;
        if (c.order) {
            if (dev_alloc(&c.tw_col, twb) != cudaSuccess) return fail(RT_ENOMEM);
            if (launch_twiddles32(1 << c.logn, c.order, c.tw_col, b->stream) != cudaSuccess) return fail(RT_ECUDA);
            b->shared_bytes += twb;
        }
    }
    for (int i = 0; i < count; ++i) {
        Slot &s = b->slots[i];
        cudaError_t e = slot_alloc(s.job.n, hist_cap(b), pump_eval(s.job.pump) == PE_TABLE, job_rough(s.job), &s.buf);
        if (e != cudaSuccess) return fail(cuda_to_status(e));
        if ((e = start_slot(b, i)) != cudaSuccess) return fail(cuda_to_status(e));
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(RT_ECUDA);
    *out = b;
    return RT_OK;
}

rt_status rt_batch_step(rt_batch *b, long long nb)
{
    if (!b || nb < 0) return RT_EINVAL;
    if (nb == 0) return RT_OK;
    TraceRange tr("rt_batch_step");
    DeviceGuard g(b->device);
    const long long K = b->opts.chunk;
    long long left = nb;
    if (K > 0 && left >= K) {
        cudaGraphExec_t ge;
        BT_TRY(batch_graph(b, K, &ge));
        for (; left >= K; left -= K) BT_TRY(cudaGraphLaunch(ge, b->stream));
    }
    const std::vector<ClassLaunch> cl = launches(b);
    for (; left > 0; --left) BT_TRY(enqueue_classes_bounce(cl, b->err, b->stream));
    return RT_OK;
}

rt_status rt_batch_sweep(rt_batch *b, int which)
{
    if (!b || (which != RT_SWEEP_COLUMNS && which != RT_SWEEP_ROWS)) return RT_EINVAL;
    DeviceGuard g(b->device);
    BT_TRY(enqueue_sweep(launches(b), which, b->err, b->stream));
    return RT_OK;
}

rt_status rt_batch_set_job(rt_batch *b, int i, const rt_job *job, long long n_bounces)
{
    if (!valid_slot(b, i) || !job || !job_ok(*job)) return RT_EINVAL;
    Slot &s = b->slots[i];
    // Same grid size only; a table pump or a rough mirror needs a slot created with one.
    if (job->n != s.job.n || (pump_eval(job->pump) == PE_TABLE && !s.buf.pump_tab)) return RT_EINVAL;
    if (job_rough(*job) && !s.buf.phase) return RT_EINVAL;
    DeviceGuard g(b->device);
    s.job = *job;
    s.target = n_bounces < 0 ? LLONG_MAX : n_bounces;
    BT_TRY(start_slot(b, i));
    return RT_OK;
}

rt_status rt_batch_sync(rt_batch *b)
{
    if (!b) return RT_EINVAL;
    DeviceGuard g(b->device);
    return check_errors(b);
}

static rt_status batch_copy(rt_batch *b, void *dst, const void *src, size_t bytes, size_t want, bool out)
{
    if (!dst || !src || bytes != want) return RT_EINVAL;
    DeviceGuard g(b->device);
    BT_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, b->stream));
    return out ? check_errors(b) : RT_OK;
}

rt_status rt_batch_read_field(rt_batch *b, int i, void *dst, size_t bytes)
{
    if (!valid_slot(b, i)) return RT_EINVAL;
    return batch_copy(b, dst, b->slots[i].buf.E, bytes, field_bytes(b, i), true);
}

rt_status rt_batch_read_inversion(rt_batch *b, int i, void *dst, size_t bytes)
{
    if (!valid_slot(b, i)) return RT_EINVAL;
    return batch_copy(b, dst, b->slots[i].buf.N, bytes, inv_bytes(b, i), true);
}

rt_status rt_batch_write_field(rt_batch *b, int i, const void *src, size_t bytes)
{
    if (!valid_slot(b, i)) return RT_EINVAL;
    return batch_copy(b, b->slots[i].buf.E, src, bytes, field_bytes(b, i), false);
}

rt_status rt_batch_write_inversion(rt_batch *b, int i, const void *src, size_t bytes)
{
    if (!valid_slot(b, i)) return RT_EINVAL;
    return batch_copy(b, b->slots[i].buf.N, src, bytes, inv_bytes(b, i), false);
}

rt_status rt_batch_stats(rt_batch *b, int i, rt_stats_t *out)
{
    if (!valid_slot(b, i) || !out) return RT_EINVAL;
    DeviceGuard g(b->device);
    SlotCtl c;
    BT_TRY(cudaMemcpyAsync(&c, &b->ctl[i], sizeof(c), cudaMemcpyDeviceToHost, b->stream));
    BT_TRY(cudaStreamSynchronize(b->stream));
    const Slot &s = b->slots[i];
    std::memset(out, 0, sizeof(*out));
    out->bounces = c.bounce;
    out->mean_intensity = c.last_mean;
    out->alpha = job_alpha(s.job);
    out->n = s.job.n;
    out->precision = RT_FP32;
    out->last_error = c.err;
    const long long cap = s.buf.hist ? hist_cap(b) : 0;
    out->history_len = cap > 0 ? (c.bounce < cap ? c.bounce : cap) : 0;
    return RT_OK;
}

rt_status rt_batch_read_history(rt_batch *b, int i, double *dst, long long max, long long *got)
{
    if (!valid_slot(b, i) || !got || max < 0 || (max > 0 && !dst)) return RT_EINVAL;
    *got = 0;
    rt_stats_t s;
    rt_status st = rt_batch_stats(b, i, &s);
    if (st != RT_OK) return st;
    const long long cap = hist_cap(b);
    const long long len = s.history_len < max ? s.history_len : max;
    if (len <= 0 || cap <= 0) return RT_OK;
    DeviceGuard g(b->device);
    const long long first = s.bounces - len;
    long long done = 0;
    while (done < len) {
        const long long slot = (first + done) % cap;
        long long run = cap - slot;
        if (run > len - done) run = len - done;
        BT_TRY(cudaMemcpy(dst + done, b->slots[i].buf.hist + slot, sizeof(double) * (size_t)run,
                          cudaMemcpyDeviceToHost));
        done += run;
    }
    *got = len;
    return RT_OK;
}

rt_status rt_batch_bounces(rt_batch *b, long long *counts)
{
    if (!b || !counts) return RT_EINVAL;
    DeviceGuard g(b->device);
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
    for (const Slot &s : b->slots) t += s.buf.bytes;
    *bytes = t;
    return RT_OK;
}

rt_status rt_batch_destroy(rt_batch *b)
{
    if (!b) return RT_OK;
    DeviceGuard g(b->device);
    cudaStreamSynchronize(b->stream);
    release(b);
    delete b;
    return RT_OK;
}

}  // extern "C"
