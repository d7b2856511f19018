// plss_trace.h -- named ranges (NVTX) around the host-side phases of the
// library's calls: a timeline profiler (Nsight Systems) shows where a solve
// spends its time -- context set-up, the iteration loop, the result copies,
// the server's scheduling rounds -- next to the kernels. Without a profiler
// attached each range costs a call that returns at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace plss {

class TraceRange {
public:
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace plss
