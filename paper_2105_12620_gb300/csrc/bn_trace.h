// bn_trace.h — NVTX ranges around the library's host-side steps (init, sweeps, energy, criterion,
// serving chunks), so that a timeline profiler shows them next to the kernels.  nvtx3 is
// header-only: without a profiler attached the calls do nothing.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace bn {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace bn
