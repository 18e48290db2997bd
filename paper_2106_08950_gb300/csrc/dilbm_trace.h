// NVTX ranges around the library's host entry points: a step call, a batch
// step, a server macro-step, create and autotuning show up as named ranges in
// NVIDIA's profilers.  NVTX v3 is header-only and costs a function call when
// no tool is attached.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace dilbm {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace dilbm
