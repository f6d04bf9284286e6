// dpg_trace.h -- NVTX ranges around the library's launches (internal).  A range covers
// the host-side enqueue of one stage (geometry, contraction, condensation, ...); profilers
// that record NVTX (Nsight Systems, ncu --nvtx) attribute the kernels launched inside it to
// the stage.  Header-only NVTX v3: without an attached tool every call is a no-op.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace dpg {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace dpg
