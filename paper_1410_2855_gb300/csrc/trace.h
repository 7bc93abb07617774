// Host-side trace ranges (NVTX) around the library's API calls and
// scheduling rounds; free when no profiler is attached.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace rtk {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace rtk
