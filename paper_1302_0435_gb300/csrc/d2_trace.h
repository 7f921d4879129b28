// d2_trace.h -- NVTX ranges around the library's entry points and their
// phases (cutting-plane rounds, level rounds, serving requests): a profiler
// attached to the process shows them on its timeline; without one a range
// costs one indirect call.  Header-only NVTX 3.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace d2k {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace d2k
