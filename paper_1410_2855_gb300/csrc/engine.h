// Host-side engine shared by batches and the server: one resonator "slot"
// (its device buffers, counters and batched-launch descriptor) and the size
// classes that group slots of one grid size into shared launches.
#pragma once

#include <vector>

#include "rt.h"
#include "rt_internal.h"

namespace rtk {

// Per-slot device counters (one 64-byte line each).
struct SlotCtl {
    unsigned int count;  // arrival counter of the row-sweep reduction
    int err;             // sticky error (RT_ENUMERIC)
    long long bounce;    // bounces done since the slot's job started
    double last_mean;    // mean intensity after the last bounce
    long long pad[5];
};
static_assert(sizeof(SlotCtl) == 64, "slot control block is one line");

// Device buffers of one slot, carved from one allocation.
struct SlotBufs {
    unsigned char *mem = nullptr;
    size_t bytes = 0;
    float2 *E = nullptr;
    float *N = nullptr;
    float2 *h = nullptr;
    double *part = nullptr;
    double *hist = nullptr;
    CUtensorMap *tmap = nullptr;
    float *pump_tab = nullptr;
    float2 *lens = nullptr;   // per-axis curved-mirror factors (always present, n entries)
    float2 *phase = nullptr;  // n*n aperture factors of a rough mirror (only when allocated for one)
};

bool job_ok(const rt_job &j);            // 32 <= n <= 2048 and parameters in range
bool job_rough(const rt_job &j);         // the job's mirror has a roughness table
int pump_eval(const rt_pump &p);         // PumpEval of a job's pump
double job_alpha(const rt_job &j);       // lambda z / W^2 = (D/W)^2 / N_F
int log2_of(int n);

// Bytes and allocation of a slot for side n (table: N0 table for PE_TABLE;
// rough: aperture table for a rough mirror).
size_t slot_bytes(int n, long long hist_cap, bool table, bool rough);
cudaError_t slot_alloc(int n, long long hist_cap, bool table, bool rough, SlotBufs *out);
void slot_free(SlotBufs *b);

// Descriptor of a slot for the batched kernels.
BatchRes slot_descriptor(const rt_job &job, const SlotBufs &b, SlotCtl *ctl, long long hist_cap, long long target);

// Start `job` in a slot (as rt_create starts a handle): propagator table,
// class twiddles, aperture phase, noise field, N = N0, tensor map, zeroed
// counters, and the descriptor written to *d_desc.  All on stream s.
cudaError_t slot_start(const rt_job &job, const SlotBufs &b, int colC, float2 *class_tw, SlotCtl *ctl,
                       BatchRes *d_desc, long long hist_cap, long long target, cudaStream_t s);

// Set only the bounce target of a slot's descriptor (stops or idles it).
cudaError_t slot_set_target(BatchRes *d_desc, long long target, cudaStream_t s);

// Grid sizes of one persistent batched launch set.  `mixed`: the class runs
// in the launches shared by every mixed class (one per sweep across sizes;
// its tensor maps use mix_col_tile columns); otherwise it has its own.
struct ClassLaunch {
    int logn, colC;
    const BatchRes *d_res;
    int nres;
    const float2 *tw;
    bool mixed = false;
    int order = 0;                   // radix order of the column transforms (per-class launches)
    const float2 *tw_col = nullptr;  // that order's twiddles (order != 0)
    const float2 *col_tw() const { return order ? tw_col : tw; }
};

// Process-wide choice for batches and servers created from now on: classes
// of sides 128..2048 share one launch per sweep (true) or each class gets its
// own launches (false, the default: measured faster for the 256-resonator
// sweep, 251k against 225k round trips/s, because separate per-class chains
// overlap one another's column and row phases).
bool batch_mixed();
void set_batch_mixed(bool on);
// Column tile width of a new class of side 2^logn: the mixed width when the
// class runs mixed, else `requested` (0: the tuned or built-in width).
int class_col_tile(int logn, int requested, bool *mixed);
// Radix order of a new class's column transforms: the tuned order when the
// class uses the tuned (or built-in) tile width in per-class launches, as a
// handle would; 0 otherwise.
int class_col_order(int logn, int colC, int requested, bool mixed);

// One bounce of every class: all column sweeps, then all row sweeps.
cudaError_t enqueue_classes_bounce(const std::vector<ClassLaunch> &cls, int *err, cudaStream_t s);
// One sweep (RT_SWEEP_COLUMNS or RT_SWEEP_ROWS) of every class.
cudaError_t enqueue_sweep(const std::vector<ClassLaunch> &cls, int which, int *err, cudaStream_t s);
// Kernel attributes (shared memory) of every launch the classes use.
cudaError_t prepare_classes(const std::vector<ClassLaunch> &cls);

// Side streams and fork/join events for capturing graph branches: one per
// size class, or per part of one (class_parts).  Created before a capture
// (branches_prepare), freed by branches_free.
struct Branches {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
};
cudaError_t branches_prepare(Branches &br, const std::vector<ClassLaunch> &cls, int split);
void branches_free(Branches &br);

// Into the capture running on `cap`: k bounces of every class, each class
// split into up to `split` parts of consecutive resonators, each part's chain
// of launches on its own stream (the resonators are independent, so the
// launches may overlap and fill each other's tails), joined back into `cap`.
// The joins are made even when a launch fails.
cudaError_t capture_class_bounces(const std::vector<ClassLaunch> &cls, int *err, long long k, cudaStream_t cap,
                                  Branches &br, int split);

// Parts per size class of a batch's graph.  By default about three chains
// in all: ceil(3 / c) parts per class for c chains at one part each (every
// class of per-class launches, and the mixed launches as one).  A value set
// by set_batch_split (1..8, e.g. by the Python binding's autotune_batch)
// overrides it; 0 restores the rule.  Serving rounds (few requests per
// class, where more, smaller launches cost more than they fill) use one.
int batch_split(const std::vector<ClassLaunch> &cls);
int batch_split_setting();
void set_batch_split(int parts);
constexpr int kServeSplit = 1;

// Device index guard.
struct DeviceGuard {
    int prev = -1, want;
    explicit DeviceGuard(int d) : want(d)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != want) cudaSetDevice(want);
    }
    ~DeviceGuard()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

inline rt_status cuda_to_status(cudaError_t e)
{
    return e == cudaSuccess ? RT_OK : (e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA);
}

}  // namespace rtk
