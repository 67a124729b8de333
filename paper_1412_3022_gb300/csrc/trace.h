// NVTX ranges around the C ABI's calls, so that a profiler timeline (ncu's
// NVTX filter, Nsight Systems) shows each library call by name around the
// kernels it launches.  NVTX v3 is header-only: without a tool attached a
// range costs a check of a function pointer.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace pmrc {

struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace pmrc

#define PMRC_TRACE(name) ::pmrc::TraceRange pmrc_trace_range_(name)
