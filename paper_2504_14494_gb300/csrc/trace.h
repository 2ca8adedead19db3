// NVTX ranges around the C ABI entry points: a profiler (ncu --nvtx, nsys)
// attributes each kernel to the call that enqueued it.  NVTX v3 is
// header-only; without an attached tool a range costs a few nanoseconds.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace lbmgnn {
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
}  // namespace lbmgnn

#define LBM_TRACE(name) ::lbmgnn::TraceRange lbm_trace_range_(name)
