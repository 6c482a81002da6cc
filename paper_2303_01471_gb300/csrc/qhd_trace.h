// qhd_trace.h -- NVTX ranges around the host calls that enqueue device work
// (evolve, its chunks, observables, potential upload), so a profiler's timeline
// groups the kernels by the API call and chunk that launched them.  NVTX is
// header-only; without an attached tool every push/pop is a no-op.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace qhd {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace qhd
