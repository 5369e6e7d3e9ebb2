// Host-side NVTX ranges of the library calls (header-only NVTX 3).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace ccg {

// A named range around the launches of one library call or phase: Nsight
// Systems shows it over the kernels launched inside it; without a tool
// attached the calls do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace ccg
