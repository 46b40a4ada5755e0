// Named ranges on the host timeline (NVTX v3, header-only): plan creation, solves
// and refinement rounds show up in a profiler's timeline.  Without a profiler
// attached the calls return at once.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace fps {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace fps
