// Shared by batches and the server (engine.h): slot set-up, the batched
// bounce launches, and their capture into graphs with one branch per part
// of a size class.
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>

#include "engine.h"

namespace rtk {

namespace {
size_t al256(size_t b) { return (b + 255) / 256 * 256; }
bool fpos(double v) { return std::isfinite(v) && v > 0.0; }
}  // namespace

int log2_of(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

bool job_ok(const rt_job &j)
{
    if (j.n < 32 || j.n > 2048 || (j.n & (j.n - 1))) return false;
    if (!fpos(j.fresnel) || !std::isfinite(j.g0) || j.g0 < 0.0 || !std::isfinite(j.T1) || j.T1 < 1.0) return false;
    if (!std::isfinite(j.R) || j.R <= 0.0 || j.R > 1.0) return false;
    if (!fpos(j.Isat) || j.edge_px < 0 || j.edge_px > j.n / 2 || !fpos(j.pump_diam_over_window)) return false;
    if (!std::isfinite(j.noise_amp) || j.noise_amp < 0.0) return false;
    if (j.pump.kind < RT_PUMP_SUPERGAUSS || j.pump.kind > RT_PUMP_ARRAY) return false;
    if (j.pump.kind == RT_PUMP_SUPERGAUSS && (!fpos(j.pump.order) || !fpos(j.pump.radius))) return false;
    if (j.pump.kind == RT_PUMP_ARRAY && !j.pump.profile) return false;
    if (!std::isfinite(j.z_over_F)) return false;
    if (j.taper_px < 0 || j.taper_px > j.n / 2 || (j.relax != RT_RELAX_EULER && j.relax != RT_RELAX_EXACT)) return false;
    return true;
}

bool job_rough(const rt_job &j) { return j.roughness != nullptr; }

int pump_eval(const rt_pump &p)
{
    return p.kind == RT_PUMP_UNIFORM ? PE_UNIFORM
                                     : ((p.kind == RT_PUMP_SUPERGAUSS && p.order == 10.0) ? PE_SG10 : PE_TABLE);
}

double job_alpha(const rt_job &j) { return j.pump_diam_over_window * j.pump_diam_over_window / j.fresnel; }

namespace {
constexpr int kParts = 9;

void slot_layout(int n, long long hist_cap, bool table, bool rough, size_t off[kParts], size_t *total)
{
    const size_t N = (size_t)n, P = N * N, cap = hist_cap > 0 ? (size_t)hist_cap : 0;
    const size_t sz[kParts] = {al256(P * sizeof(float2)),                                  // E
                               al256(P * sizeof(float)),                                   // N
                               al256(N * sizeof(float2)),                                  // h
                               al256((size_t)row_groups32(log2_of(n)) * sizeof(double)),  // part
                               al256(cap * sizeof(double)),                                // history
                               al256(sizeof(CUtensorMap)),                                 // tensor map
                               table ? al256(P * sizeof(float)) : 0,                       // N0 table
                               al256(N * sizeof(float2)),                                  // lens
                               rough ? al256(P * sizeof(float2)) : 0};                     // aperture table
    size_t t = 0;
    for (int k = 0; k < kParts; ++k) {
        off[k] = t;
        t += sz[k];
    }
    *total = t;
}
}  // namespace

size_t slot_bytes(int n, long long hist_cap, bool table, bool rough)
{
    size_t off[kParts], t;
    slot_layout(n, hist_cap, table, rough, off, &t);
    return t;
}

cudaError_t slot_alloc(int n, long long hist_cap, bool table, bool rough, SlotBufs *out)
{
    size_t off[kParts], total;
    slot_layout(n, hist_cap, table, rough, off, &total);
    SlotBufs b;
    cudaError_t e = dev_alloc(&b.mem, total);
    if (e != cudaSuccess) return e;
    b.bytes = total;
    b.E = reinterpret_cast<float2 *>(b.mem + off[0]);
    b.N = reinterpret_cast<float *>(b.mem + off[1]);
    b.h = reinterpret_cast<float2 *>(b.mem + off[2]);
    b.part = reinterpret_cast<double *>(b.mem + off[3]);
    b.hist = hist_cap > 0 ? reinterpret_cast<double *>(b.mem + off[4]) : nullptr;
    b.tmap = reinterpret_cast<CUtensorMap *>(b.mem + off[5]);
    b.pump_tab = table ? reinterpret_cast<float *>(b.mem + off[6]) : nullptr;
    b.lens = reinterpret_cast<float2 *>(b.mem + off[7]);
    b.phase = rough ? reinterpret_cast<float2 *>(b.mem + off[8]) : nullptr;
    *out = b;
    return cudaSuccess;
}

void slot_free(SlotBufs *b)
{
    if (b->mem) cudaFree(b->mem);
    *b = SlotBufs();
}

BatchRes slot_descriptor(const rt_job &job, const SlotBufs &b, SlotCtl *ctl, long long hist_cap, long long target)
{
    BatchRes r{};
    r.E = b.E;
    r.N = b.N;
    r.h = b.h;
    r.tmap = b.tmap;
    const int pe = pump_eval(job.pump);
    GainParams<float> &g = r.g;
    g.sqrtR = (float)std::sqrt(job.R);
    g.invT1 = (float)(1.0 / job.T1);
    g.invIsat = (float)(1.0 / job.Isat);
    g.g0 = (float)job.g0;
    g.inv_rp2 = job.pump.kind == RT_PUMP_SUPERGAUSS ? (float)(1.0 / (job.pump.radius * job.pump.radius)) : 0.0f;
    g.half_order = (float)(0.5 * job.pump.order);
    g.int_half_order = pe == PE_SG10 ? 5 : 0;
    g.edge = job.edge_px;
    g.pump_kind = job.pump.kind;
    g.pump_tab = b.pump_tab;
    g.lens = (!job_rough(job) && (job.z_over_F != 0.0 || job.taper_px > 0 || job.relax == RT_RELAX_EXACT)) ? b.lens
                                                                                                         : nullptr;
    g.phase = job_rough(job) ? b.phase : nullptr;
    g.relax_exact = job.relax == RT_RELAX_EXACT;
    r.pe = pe;
    r.target = target;
    r.st.part = b.part;
    r.st.count = &ctl->count;
    r.st.hist = b.hist;
    r.st.hist_cap = b.hist ? hist_cap : 0;
    r.st.bounce = &ctl->bounce;
    r.st.last_mean = &ctl->last_mean;
    r.st.err = &ctl->err;
    return r;
}

cudaError_t slot_start(const rt_job &job, const SlotBufs &b, int colC, float2 *class_tw, SlotCtl *ctl,
                       BatchRes *d_desc, long long hist_cap, long long target, cudaStream_t s)
{
    const int n = job.n;
    const size_t P = (size_t)n * n;
    cudaError_t e;
    if ((e = launch_tables32(n, job_alpha(job), class_tw, b.h, s)) != cudaSuccess) return e;
    if ((e = launch_noise32(n, job.seed, job.noise_amp, b.E, s)) != cudaSuccess) return e;
    double *profile = nullptr;
    if (job.pump.kind == RT_PUMP_ARRAY) {
        if ((e = cudaMallocAsync(reinterpret_cast<void **>(&profile), P * sizeof(double), s)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(profile, job.pump.profile, P * sizeof(double), cudaMemcpyDefault, s)) != cudaSuccess)
            return e;
    }
    e = launch_pump32(n, job.pump.kind, job.g0, job.pump.order, job.pump.radius, profile, b.N, s);
    if (profile) cudaFreeAsync(profile, s);
    if (e != cudaSuccess) return e;
    if (pump_eval(job.pump) == PE_TABLE) {
        if (!b.pump_tab) return cudaErrorInvalidValue;
        if ((e = cudaMemcpyAsync(b.pump_tab, b.N, P * sizeof(float), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
    }
    const double c = lens_curvature(job_alpha(job), job.z_over_F);
    if (job_rough(job)) {
        if (!b.phase) return cudaErrorInvalidValue;
        double *psi = nullptr;
        if ((e = cudaMallocAsync(reinterpret_cast<void **>(&psi), P * sizeof(double), s)) != cudaSuccess) return e;
        e = cudaMemcpyAsync(psi, job.roughness, P * sizeof(double), cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = launch_phase32(n, c, job.edge_px, job.taper_px, psi, b.phase, s);
        cudaFreeAsync(psi, s);
        if (e != cudaSuccess) return e;
    } else if (job.z_over_F != 0.0 || job.taper_px > 0 || job.relax == RT_RELAX_EXACT) {
        if ((e = launch_lens32(n, c, job.edge_px, job.taper_px, b.lens, s)) != cudaSuccess) return e;
    }
    alignas(64) unsigned char map[128];
    if ((e = make_col_tensor_map(map, b.E, n, colC)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(b.tmap, map, sizeof(map), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(SlotCtl), s)) != cudaSuccess) return e;
    const BatchRes r = slot_descriptor(job, b, ctl, hist_cap, target);
    return cudaMemcpyAsync(d_desc, &r, sizeof(r), cudaMemcpyHostToDevice, s);
}

cudaError_t slot_set_target(BatchRes *d_desc, long long target, cudaStream_t s)
{
    // The host value is staged before cudaMemcpyAsync returns (pageable source).
    return cudaMemcpyAsync(&d_desc->target, &target, sizeof(target), cudaMemcpyHostToDevice, s);
}

static std::atomic<bool> g_batch_mixed{false};
bool batch_mixed() { return g_batch_mixed.load(); }
void set_batch_mixed(bool on) { g_batch_mixed.store(on); }

int class_col_tile(int logn, int requested, bool *mixed)
{
    *mixed = requested == 0 && batch_mixed() && mix_supported(logn);
    if (*mixed) return mix_col_tile(logn);
    return requested ? requested : default_col_tile32(logn);
}

int class_col_order(int logn, int colC, int requested, bool mixed)
{
    if (mixed || requested != 0) return 0;
    const int ord = tuned_col_order32(logn);
    return ord < col_orders32(logn, colC) ? ord : 0;
}

static std::vector<MixLaunch> mixed_of(const std::vector<ClassLaunch> &cls)
{
    std::vector<MixLaunch> m;
    for (const ClassLaunch &c : cls)
        if (c.mixed && c.nres > 0) m.push_back({c.logn, c.d_res, c.nres, c.tw});
    return m;
}

static std::vector<ClassLaunch> unmixed_of(const std::vector<ClassLaunch> &cls)
{
    std::vector<ClassLaunch> r;
    for (const ClassLaunch &c : cls)
        if (!c.mixed) r.push_back(c);
    return r;
}

cudaError_t enqueue_sweep(const std::vector<ClassLaunch> &cls, int which, int *err, cudaStream_t s)
{
    cudaError_t e;
    const std::vector<MixLaunch> m = mixed_of(cls);
    if (!m.empty()) {
        e = which == RT_SWEEP_COLUMNS ? launch_col_mixed32(m.data(), (int)m.size(), err, s)
                                      : launch_row_mixed32(m.data(), (int)m.size(), err, s);
        if (e != cudaSuccess) return e;
    }
    for (const ClassLaunch &c : cls) {
        if (c.mixed) continue;
        e = which == RT_SWEEP_COLUMNS ? launch_col_batch32(c.logn, c.colC, c.d_res, c.nres, c.col_tw(), err, s, c.order)
                                      : launch_row_batch32(c.logn, c.d_res, c.nres, c.tw, err, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_classes_bounce(const std::vector<ClassLaunch> &cls, int *err, cudaStream_t s)
{
    cudaError_t e = enqueue_sweep(cls, RT_SWEEP_COLUMNS, err, s);
    return e == cudaSuccess ? enqueue_sweep(cls, RT_SWEEP_ROWS, err, s) : e;
}

cudaError_t prepare_classes(const std::vector<ClassLaunch> &cls)
{
    cudaError_t e;
    bool any_mixed = false;
    for (const ClassLaunch &c : cls) {
        if (c.mixed) any_mixed = true;
        else if ((e = prepare_batch32(c.logn, c.colC, c.order)) != cudaSuccess) return e;
    }
    return any_mixed ? prepare_mixed32() : cudaSuccess;
}


// The launch sets that get a branch each: every class, split into up to
// `split` parts of consecutive resonators.  Measured on GB300 for batches
// (256 resonators of side 256/512/1024; 64 of side 1024): one part 183k and
// 72k round trips/s, two 198k and 80k, three 204k and 89k, four 201k and 89k.
// Serving rounds (a few requests per class): one part 49k round trips/s,
// three 44k.
static std::vector<ClassLaunch> class_parts(const std::vector<ClassLaunch> &cls, int split)
{
    std::vector<ClassLaunch> out;
    for (const ClassLaunch &c : cls) {
        const int parts = c.nres < split ? (c.nres > 0 ? c.nres : 1) : (split > 0 ? split : 1);
        int first = 0;
        for (int q = 0; q < parts; ++q) {
            const int cnt = c.nres / parts + (q < c.nres % parts ? 1 : 0);
            ClassLaunch part = c;
            part.d_res = c.d_res + first;
            part.nres = cnt;
            out.push_back(part);
            first += cnt;
        }
    }
    return out;
}

// The mixed classes split into up to `split` parts: part q holds the q-th
// share of the resonators of every mixed class, so each part is one launch
// per sweep across sizes and the parts (on their own graph branches) fill
// one another's phases and tails.
static std::vector<std::vector<MixLaunch>> mixed_parts(const std::vector<ClassLaunch> &cls, int split)
{
    const std::vector<MixLaunch> m = mixed_of(cls);
    int most = 0;
    for (const MixLaunch &c : m) most = c.nres > most ? c.nres : most;
    const int parts = most == 0 ? 0 : (split < 1 ? 1 : (most < split ? most : split));
    std::vector<std::vector<MixLaunch>> out(parts);
    for (const MixLaunch &c : m) {
        int first = 0;
        for (int q = 0; q < parts; ++q) {
            const int cnt = c.nres / parts + (q < c.nres % parts ? 1 : 0);
            if (cnt > 0) out[q].push_back({c.logn, c.res + first, cnt, c.tw});
            first += cnt;
        }
    }
    return out;
}

static std::atomic<int> g_batch_split{0};
int batch_split_setting() { return g_batch_split.load(); }
void set_batch_split(int parts) { g_batch_split.store(parts); }

int batch_split(const std::vector<ClassLaunch> &cls)
{
    const int set = g_batch_split.load();
    if (set > 0) return set;
    int chains = mixed_of(cls).empty() ? 0 : 1;
    for (const ClassLaunch &c : cls)
        if (!c.mixed && c.nres > 0) ++chains;
    return chains <= 0 ? 1 : (3 + chains - 1) / chains;
}

// Chains of a capture: the parts of the mixed launches, then the parts of
// the other classes.
static size_t chain_count(const std::vector<ClassLaunch> &cls, int split)
{
    return mixed_parts(cls, split).size() + class_parts(unmixed_of(cls), split).size();
}

cudaError_t branches_prepare(Branches &br, const std::vector<ClassLaunch> &cls, int split)
{
    const size_t nb = chain_count(cls, split);
    const size_t want = nb > 1 ? nb - 1 : 0;
    if (want > 0 && !br.fork) {
        cudaError_t e = cudaEventCreateWithFlags(&br.fork, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    while (br.streams.size() < want) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (st) cudaStreamDestroy(st);
            return e;
        }
        br.streams.push_back(st);
        br.join.push_back(ev);
    }
    return cudaSuccess;
}

void branches_free(Branches &br)
{
    for (cudaStream_t st : br.streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : br.join) cudaEventDestroy(ev);
    if (br.fork) cudaEventDestroy(br.fork);
    br.streams.clear();
    br.join.clear();
    br.fork = nullptr;
}

static cudaError_t enqueue_class_chain(const ClassLaunch &c, int *err, long long k, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    for (long long i = 0; i < k && e == cudaSuccess; ++i) {
        e = launch_col_batch32(c.logn, c.colC, c.d_res, c.nres, c.col_tw(), err, s, c.order);
        if (e == cudaSuccess) e = launch_row_batch32(c.logn, c.d_res, c.nres, c.tw, err, s);
    }
    return e;
}

static cudaError_t enqueue_mixed_chain(const std::vector<MixLaunch> &m, int *err, long long k, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    for (long long i = 0; i < k && e == cudaSuccess; ++i) {
        e = launch_col_mixed32(m.data(), (int)m.size(), err, s);
        if (e == cudaSuccess) e = launch_row_mixed32(m.data(), (int)m.size(), err, s);
    }
    return e;
}

cudaError_t capture_class_bounces(const std::vector<ClassLaunch> &classes, int *err, long long k, cudaStream_t cap,
                                  Branches &br, int split)
{
    const std::vector<std::vector<MixLaunch>> mix = mixed_parts(classes, split);
    const std::vector<ClassLaunch> cls = class_parts(unmixed_of(classes), split);
    const size_t chains = mix.size() + cls.size();
    // chain j: the mixed parts first, then the parts of the other classes
    auto chain = [&](size_t j, cudaStream_t s) {
        if (j < mix.size()) return enqueue_mixed_chain(mix[j], err, k, s);
        return enqueue_class_chain(cls[j - mix.size()], err, k, s);
    };
    if (chains == 0) return cudaSuccess;
    if (chains == 1) return chain(0, cap);
    if (br.streams.size() < chains - 1 || !br.fork) return cudaErrorInvalidValue;
    cudaError_t e = cudaEventRecord(br.fork, cap);
    if (e != cudaSuccess) return e;
    size_t joined = 0;  // branches forked into the capture
    for (size_t j = 1; j < chains && e == cudaSuccess; ++j)
        if ((e = cudaStreamWaitEvent(br.streams[j - 1], br.fork, 0)) == cudaSuccess) ++joined;
    if (e == cudaSuccess) e = chain(0, cap);
    for (size_t j = 1; j < chains && e == cudaSuccess; ++j) e = chain(j, br.streams[j - 1]);
    // join every branch that was forked, whatever happened
    for (size_t j = 0; j < joined; ++j) {
        cudaError_t je = cudaEventRecord(br.join[j], br.streams[j]);
        if (je == cudaSuccess) je = cudaStreamWaitEvent(cap, br.join[j], 0);
        if (e == cudaSuccess) e = je;
    }
    return e;
}

}  // namespace rtk
