// Named ranges on the host timeline (NVTX) around the library's entry points
// and the stages inside them, so that a profiler shows which call and which
// stage enqueued each kernel (and ncu can select kernels by range with
// --nvtx-include). Without a profiler attached NVTX calls return at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace pes {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace pes
