// trace.h -- NVTX ranges on the library's entry points, so that a profiler's timeline shows which
// call launched which kernels.  NVTX 3 is header-only: nothing is linked, and with no tool attached
// a range costs a few nanoseconds.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace mq {
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
}  // namespace mq

#define MQ_TRACE(name) ::mq::TraceRange mq_trace_range_(name)
