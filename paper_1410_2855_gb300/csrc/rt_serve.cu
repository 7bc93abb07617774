// Serving loop (include/rt.h, rt_serve_*): continuous batching of simulation
// requests on one GPU stream.
//
// A worker thread repeats rounds.  A round first admits queued requests,
// oldest first, into slots of their grid size: an idle slot of that size is
// reused, otherwise a new one is allocated if the resident footprint stays
// within the budget (idle slots of other sizes are released to make room).
// It then runs `chunk` bounces of every resident request through the
// batched sweeps (one graph per class layout; a request stops exactly at its
// own bounce count because its slot's target is reached), waits, reads the
// per-slot counters, and retires finished requests: their final field is
// copied to the caller's buffer and a result is posted.  Device state stays
// resident between rounds.  A request that cannot be placed even with
// nothing resident fails (its result is posted) instead of waiting.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"
#include "trace.h"

using namespace rtk;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    long long id = 0;
    rt_job job{};
    long long bounces = 0;
    void *field_out = nullptr;
    double submit_s = 0.0, admit_s = -1.0;
};

struct SSlot {
    SlotBufs buf;
    bool busy = false;
    Request req;
    long long last_bounce = 0;
    long long target = 0;       // bounce target last written to the slot's descriptor
};

struct SClass {
    int logn = 0, colC = 4;
    bool mixed = false;         // runs in the launches shared across sizes
    int order = 0;              // radix order of the column transforms
    float2 *tw_col = nullptr;   // that order's twiddles (order != 0)
    BatchRes *d_res = nullptr;  // capacity entries
    SlotCtl *ctl = nullptr;     // capacity entries
    float2 *tw = nullptr;
    std::vector<SSlot> slots;   // allocated slots (<= capacity)
    std::vector<long long> targets;  // host staging of the slots' bounce targets
};

}  // namespace

struct rt_server {
    rt_serve_opts opts{};
    int device = 0;
    cudaStream_t stream = nullptr, capture = nullptr;
    bool own_stream = false;
    int *d_err = nullptr;
    Clock::time_point t0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;       // wakes the worker (new requests, stop)
    std::condition_variable done_cv;  // wakes drain()
    bool stop = false;
    std::deque<Request> queue;
    std::deque<rt_result> results;
    std::set<long long> live;         // ids queued or running
    std::set<long long> cancel;       // ids to cancel once the worker holds them
    long long next_id = 1, submitted = 0, finished = 0, running = 0, rounds = 0;
    double point_bounces = 0.0, busy_s = 0.0;
    // Device bytes held for requests, and the most ever held.  Only the
    // worker changes them; rt_serve_stats reads them from other threads.
    std::atomic<long long> resident{0}, peak_resident{0};
    // worker-only state
    std::map<int, SClass> classes;
    std::map<std::string, cudaGraphExec_t> graphs;
    Branches branches;                // one graph branch per size class

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

constexpr long long kHistCap = 0;

size_t request_bytes(const rt_job &j) { return slot_bytes(j.n, kHistCap, false, false); }

cudaError_t class_init(rt_server *s, SClass &c, int logn)
{
    c.logn = logn;
    c.colC = class_col_tile(logn, 0, &c.mixed);
    c.order = class_col_order(logn, c.colC, 0, c.mixed);
    const int cap = s->opts.max_per_size;
    const size_t twb = sizeof(float2) * (twiddle_entries(logn) + 1);
    cudaError_t e = dev_alloc(&c.d_res, sizeof(BatchRes) * cap);
    if (e == cudaSuccess) e = dev_alloc(&c.ctl, sizeof(SlotCtl) * cap);
    if (e == cudaSuccess) e = dev_alloc(&c.tw, twb);
    if (e == cudaSuccess && c.order) e = dev_alloc(&c.tw_col, twb);
    if (e == cudaSuccess && c.order) e = launch_twiddles32(1 << logn, c.order, c.tw_col, s->stream);
    if (e == cudaSuccess) e = c.mixed ? prepare_mixed32() : prepare_batch32(logn, c.colC, c.order);
    if (e != cudaSuccess) {  // the class is dropped: release what it holds
        if (c.d_res) cudaFree(c.d_res);
        if (c.ctl) cudaFree(c.ctl);
        if (c.tw) cudaFree(c.tw);
        if (c.tw_col) cudaFree(c.tw_col);
        c.d_res = nullptr;
        c.ctl = nullptr;
        c.tw = nullptr;
        c.tw_col = nullptr;
    }
    return e;
}

// Release idle slots of other sizes (largest first) until `need` more bytes fit.
void make_room(rt_server *s, long long need, int keep_logn)
{
    for (auto it = s->classes.rbegin(); it != s->classes.rend() && s->resident + need > s->opts.budget_bytes; ++it) {
        if (it->first == keep_logn) continue;
        SClass &c = it->second;
        // only trailing idle slots can go (slot indices must stay dense)
        while (!c.slots.empty() && !c.slots.back().busy && s->resident + need > s->opts.budget_bytes) {
            s->resident -= (long long)c.slots.back().buf.bytes;
            slot_free(&c.slots.back().buf);
            c.slots.pop_back();
        }
    }
}

// Release every idle slot that can go (trailing idle slots of each class).
void release_idle(rt_server *s)
{
    for (auto &kv : s->classes) {
        SClass &c = kv.second;
        while (!c.slots.empty() && !c.slots.back().busy) {
            s->resident -= (long long)c.slots.back().buf.bytes;
            slot_free(&c.slots.back().buf);
            c.slots.pop_back();
        }
    }
}

// Try to place a request; returns true if admitted.  A CUDA failure on the
// way (set-up of its size class, slot allocation or start) is left in *why.
bool admit(rt_server *s, Request &r, cudaError_t *why)
{
    *why = cudaSuccess;
    const int logn = log2_of(r.job.n);
    auto it = s->classes.find(logn);
    if (it == s->classes.end()) {
        SClass c;
        if ((*why = class_init(s, c, logn)) != cudaSuccess) return false;
        it = s->classes.emplace(logn, c).first;
    }
    SClass &c = it->second;
    int idx = -1;
    for (size_t k = 0; k < c.slots.size(); ++k)
        if (!c.slots[k].busy) {
            idx = (int)k;
            break;
        }
    if (idx < 0) {
        if ((int)c.slots.size() >= s->opts.max_per_size) return false;
        const long long need = (long long)request_bytes(r.job);
        if (s->resident + need > s->opts.budget_bytes) make_room(s, need, logn);
        if (s->resident + need > s->opts.budget_bytes) return false;
        SSlot ns;
        if ((*why = slot_alloc(r.job.n, kHistCap, false, false, &ns.buf)) != cudaSuccess) return false;
        const long long now_resident = s->resident += (long long)ns.buf.bytes;
        if (now_resident > s->peak_resident.load()) s->peak_resident.store(now_resident);
        c.slots.push_back(ns);
        idx = (int)c.slots.size() - 1;
    }
    SSlot &sl = c.slots[idx];
    if ((*why = slot_start(r.job, sl.buf, c.colC, c.tw, &c.ctl[idx], c.d_res + idx, kHistCap, r.bounces,
                           s->stream)) != cudaSuccess)
        return false;
    sl.target = r.bounces;
    sl.busy = true;
    sl.req = r;
    sl.req.admit_s = s->now();
    sl.last_bounce = 0;
    return true;
}

cudaError_t round_graph(rt_server *s, cudaGraphExec_t *out)
{
    std::vector<ClassLaunch> cl;
    std::string key = std::to_string(s->opts.chunk);
    for (auto &kv : s->classes) {
        SClass &c = kv.second;
        if (c.slots.empty()) continue;
        cl.push_back({c.logn, c.colC, c.d_res, (int)c.slots.size(), c.tw, c.mixed, c.order, c.tw_col});
        key += "/" + std::to_string(c.logn) + ":" + std::to_string(c.slots.size());
    }
    auto it = s->graphs.find(key);
    if (it != s->graphs.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaError_t e = branches_prepare(s->branches, cl, kServeSplit);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(s->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t le = capture_class_bounces(cl, s->d_err, s->opts.chunk, s->capture, s->branches, kServeSplit);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->capture, &g);
    if (le != cudaSuccess) e = le;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    s->graphs[key] = ge;
    *out = ge;
    return cudaSuccess;
}

// Result of a request that never ran (cancelled while queued); s->mu held.
void post_unrun_locked(rt_server *s, const Request &q, int status)
{
    rt_result r{};
    r.id = q.id;
    r.status = status;
    r.n = q.job.n;
    r.submit_s = q.submit_s;
    r.admit_s = -1.0;
    r.finish_s = s->now();
    s->results.push_back(r);
    ++s->finished;
    s->live.erase(q.id);
    s->cancel.erase(q.id);
}

void post(rt_server *s, const SSlot &sl, int status, long long bounces, double mean)
{
    rt_result r{};
    r.id = sl.req.id;
    r.status = status;
    r.n = sl.req.job.n;
    r.bounces = bounces;
    r.mean_intensity = mean;
    r.submit_s = sl.req.submit_s;
    r.admit_s = sl.req.admit_s;
    r.finish_s = s->now();
    std::lock_guard<std::mutex> lk(s->mu);
    s->results.push_back(r);
    ++s->finished;
    --s->running;
    s->live.erase(r.id);
    s->cancel.erase(r.id);
}

// Shortest-first: advance only the resident requests with the least work
// left this round (their grid points up to round_points), by writing every
// slot's bounce target; the batched kernels skip slots at their target.
cudaError_t select_round(rt_server *s)
{
    struct Cand {
        SClass *c;
        int k;
        double left;
        long long id;
    };
    std::vector<Cand> cand;
    for (auto &kv : s->classes)
        for (size_t k = 0; k < kv.second.slots.size(); ++k) {
            const SSlot &sl = kv.second.slots[k];
            if (!sl.busy) continue;
            const double n2 = (double)sl.req.job.n * sl.req.job.n;
            cand.push_back({&kv.second, (int)k, n2 * (double)(sl.req.bounces - sl.last_bounce), sl.req.id});
        }
    std::sort(cand.begin(), cand.end(),
              [](const Cand &a, const Cand &b) { return a.left < b.left || (a.left == b.left && a.id < b.id); });
    const double budget = s->opts.round_points > 0 ? (double)s->opts.round_points : (double)(1ll << 23);
    double pts = 0.0;
    for (const Cand &cd : cand) {
        SSlot &sl = cd.c->slots[cd.k];
        const bool active = pts < budget;
        if (active) pts += (double)sl.req.job.n * sl.req.job.n;
        sl.target = active ? std::min(sl.req.bounces, sl.last_bounce + (long long)s->opts.chunk) : sl.last_bounce;
    }
    for (auto &kv : s->classes) {
        SClass &c = kv.second;
        if (c.slots.empty()) continue;
        c.targets.resize(c.slots.size());
        for (size_t k = 0; k < c.slots.size(); ++k) c.targets[k] = c.slots[k].target;
        cudaError_t e = cudaMemcpy2DAsync(&c.d_res[0].target, sizeof(BatchRes), c.targets.data(), sizeof(long long),
                                          sizeof(long long), c.slots.size(), cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One scheduling round: launch, wait, retire.  Returns false on a CUDA failure.
bool run_round(rt_server *s)
{
    TraceRange tr("serve round");
    const double t_start = s->now();
    cudaGraphExec_t ge;
    std::set<long long> cancel;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        cancel = s->cancel;
    }
    cudaError_t e = s->opts.policy == RT_SERVE_SHORTEST_FIRST ? select_round(s) : cudaSuccess;
    if (e == cudaSuccess) e = round_graph(s, &ge);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    double pb = 0.0;
    for (auto &kv : s->classes) {
        SClass &c = kv.second;
        if (c.slots.empty()) continue;
        std::vector<SlotCtl> ctl(c.slots.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(ctl.data(), c.ctl, sizeof(SlotCtl) * ctl.size(), cudaMemcpyDeviceToHost);
        for (size_t k = 0; k < c.slots.size(); ++k) {
            SSlot &sl = c.slots[k];
            if (!sl.busy) continue;
            if (e != cudaSuccess || err) {
                post(s, sl, e != cudaSuccess ? RT_ECUDA : err, sl.last_bounce, 0.0);
                sl.busy = false;
                continue;
            }
            const long long b = ctl[k].bounce;
            pb += (double)(b - sl.last_bounce) * (double)sl.req.job.n * (double)sl.req.job.n;
            sl.last_bounce = b;
            if (ctl[k].err || b >= sl.req.bounces) {
                int status = ctl[k].err ? ctl[k].err : RT_OK;
                if (sl.req.field_out && status == RT_OK) {
                    const size_t bytes = (size_t)sl.req.job.n * sl.req.job.n * sizeof(float2);
                    if (cudaMemcpy(sl.req.field_out, sl.buf.E, bytes, cudaMemcpyDefault) != cudaSuccess)
                        status = RT_ECUDA;
                }
                post(s, sl, status, b, ctl[k].last_mean);
                sl.busy = false;
            } else if (cancel.count(sl.req.id)) {
                // stop the slot (later rounds skip it) and report what it ran
                if (e == cudaSuccess) e = slot_set_target(c.d_res + k, 0, s->stream);
                sl.target = 0;
                post(s, sl, RT_ECANCELED, b, ctl[k].last_mean);
                sl.busy = false;
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->point_bounces += pb;
        s->busy_s += s->now() - t_start;
        ++s->rounds;
    }
    s->done_cv.notify_all();
    if (err && e == cudaSuccess) cudaMemset(s->d_err, 0, sizeof(int));
    return e == cudaSuccess;
}

void worker_main(rt_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<Request> fresh;
        bool any_running;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            for (const Request &q : s->queue) {
                if (s->cancel.count(q.id)) post_unrun_locked(s, q, RT_ECANCELED);
                else fresh.push_back(q);
            }
            s->queue.clear();
            any_running = s->running > 0;
            if (fresh.empty() && !any_running) {
                s->cv.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        // admission, oldest first; what does not fit goes back to the queue front
        std::vector<Request> waiting;
        long long admitted = 0;
        cudaError_t why = cudaSuccess;
        for (Request &r : fresh) {
            if (admit(s, r, &why)) ++admitted;
            else waiting.push_back(r);
        }
        // Nothing resident and nothing admitted: no later round can free room,
        // so release every idle slot and try once more.  A request that still
        // cannot be placed before anything else is admitted has failed
        // (RT_ENOMEM, or RT_ECUDA after another CUDA error) rather than wait
        // for ever.
        std::vector<std::pair<Request, int>> failed;
        if (!waiting.empty() && admitted == 0 && !any_running) {
            release_idle(s);
            std::vector<Request> still;
            for (Request &r : waiting) {
                if (admit(s, r, &why)) ++admitted;
                else if (admitted == 0)
                    failed.emplace_back(r, why == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA);
                else still.push_back(r);
            }
            waiting.swap(still);
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (auto &f : failed) post_unrun_locked(s, f.first, s->cancel.count(f.first.id) ? RT_ECANCELED : f.second);
            s->running += admitted;
            for (auto it = waiting.rbegin(); it != waiting.rend(); ++it) {
                if (s->cancel.count(it->id)) post_unrun_locked(s, *it, RT_ECANCELED);
                else s->queue.push_front(*it);
            }
            any_running = s->running > 0;
        }
        if (!any_running) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::milliseconds(5));
            continue;
        }
        run_round(s);
    }
}

void release(rt_server *s)
{
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    for (auto &kv : s->classes) {
        SClass &c = kv.second;
        for (SSlot &sl : c.slots) slot_free(&sl.buf);
        if (c.d_res) cudaFree(c.d_res);
        if (c.ctl) cudaFree(c.ctl);
        if (c.tw) cudaFree(c.tw);
        if (c.tw_col) cudaFree(c.tw_col);
    }
    if (s->d_err) cudaFree(s->d_err);
    if (s->capture) cudaStreamDestroy(s->capture);
    branches_free(s->branches);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
}

}  // namespace

extern "C" {

rt_status rt_serve_opts_default(rt_serve_opts *o)
{
    if (!o) return RT_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->budget_bytes = 8ll << 30;
    o->chunk = 500;
    o->max_per_size = 128;
    o->cuda_stream = nullptr;
    return RT_OK;
}

rt_status rt_serve_create(const rt_serve_opts *opts, rt_server **out)
{
    if (!out) return RT_EINVAL;
    *out = nullptr;
    rt_serve_opts o;
    if (opts) o = *opts;
    else rt_serve_opts_default(&o);
    if (o.budget_bytes <= 0 || o.chunk <= 0 || o.max_per_size <= 0 || o.round_points < 0) return RT_EINVAL;
    if (o.policy != RT_SERVE_FIFO && o.policy != RT_SERVE_SHORTEST_FIRST) return RT_EINVAL;
    rt_server *s = new (std::nothrow) rt_server();
    if (!s) return RT_ENOMEM;
    s->opts = o;
    s->t0 = Clock::now();
    cudaGetDevice(&s->device);
    auto fail = [&](rt_status st) {
        release(s);
        delete s;
        return st;
    };
    if (o.cuda_stream) {
        s->stream = static_cast<cudaStream_t>(o.cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(RT_ECUDA);
        s->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking) != cudaSuccess) return fail(RT_ECUDA);
    if (dev_alloc(&s->d_err, sizeof(int)) != cudaSuccess) return fail(RT_ENOMEM);
    if (cudaMemset(s->d_err, 0, sizeof(int)) != cudaSuccess) return fail(RT_ECUDA);
    s->worker = std::thread(worker_main, s);
    *out = s;
    return RT_OK;
}

rt_status rt_serve_submit(rt_server *s, const rt_job *job, long long n_bounces, void *field_out, long long *id)
{
    if (!s || !job || !id || n_bounces <= 0 || !job_ok(*job)) return RT_EINVAL;
    if (pump_eval(job->pump) == PE_TABLE || job_rough(*job)) return RT_EINVAL;
    if ((long long)request_bytes(*job) > s->opts.budget_bytes) return RT_EINVAL;
    Request r;
    r.job = *job;
    r.job.pump.profile = nullptr;
    r.bounces = n_bounces;
    r.field_out = field_out;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r.id = s->next_id++;
        r.submit_s = s->now();
        s->queue.push_back(r);
        s->live.insert(r.id);
        ++s->submitted;
    }
    s->cv.notify_one();
    *id = r.id;
    return RT_OK;
}

rt_status rt_serve_cancel(rt_server *s, long long id)
{
    if (!s) return RT_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->live.count(id)) return RT_EINVAL;
        bool dropped = false;
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
            if (it->id == id) {
                post_unrun_locked(s, *it, RT_ECANCELED);
                s->queue.erase(it);
                dropped = true;
                break;
            }
        }
        if (!dropped) s->cancel.insert(id);  // being admitted or running: the worker stops it
    }
    s->done_cv.notify_all();
    s->cv.notify_one();
    return RT_OK;
}

rt_status rt_serve_poll(rt_server *s, rt_result *out, int max, int *got)
{
    if (!s || !got || max < 0 || (max > 0 && !out)) return RT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    int k = 0;
    while (k < max && !s->results.empty()) {
        out[k++] = s->results.front();
        s->results.pop_front();
    }
    *got = k;
    return RT_OK;
}

rt_status rt_serve_drain(rt_server *s, double timeout_s)
{
    if (!s || timeout_s < 0) return RT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [s] { return s->finished >= s->submitted; });
    return ok ? RT_OK : RT_ETIMEOUT;
}

rt_status rt_serve_stats(rt_server *s, rt_serve_stats_t *out)
{
    if (!s || !out) return RT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->queued = (long long)s->queue.size();
    out->running = s->running;
    out->done = s->finished;
    out->resident_bytes = s->resident.load();
    out->peak_resident_bytes = s->peak_resident.load();
    out->point_bounces = s->point_bounces;
    out->busy_s = s->busy_s;
    out->rounds = s->rounds;
    return RT_OK;
}

rt_status rt_serve_destroy(rt_server *s)
{
    if (!s) return RT_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    DeviceGuard g(s->device);
    cudaStreamSynchronize(s->stream);
    release(s);
    delete s;
    return RT_OK;
}

}  // extern "C"
