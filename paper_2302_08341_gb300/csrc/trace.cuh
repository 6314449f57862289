// NVTX ranges around the library's calls, so that a timeline tool (Nsight
// Systems, Nsight Compute's range filters) shows the steps, the particle
// filter and the adjoint by name.  NVTX v3 is header-only; with no tool
// attached a range costs two cheap host calls.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace flood {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace flood
