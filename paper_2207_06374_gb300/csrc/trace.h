// NVTX ranges around the library's entry points, so a timeline (Nsight
// Systems, Nsight Compute's range filters) shows which call issued which
// kernels.  Header-only NVTX 3; without a tool attached a range costs a
// branch.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace trstmi {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace trstmi
