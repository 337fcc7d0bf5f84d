// NVTX ranges around the library's calls (header-only NVTX v3: without a profiler attached the
// calls do nothing).  Names the phases a timeline shows: build, index, query batches, fastest
// paths, shortest durations, server slices.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace kairos {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace kairos
