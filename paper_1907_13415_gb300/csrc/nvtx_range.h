// nvtx_range.h -- NVTX ranges around the library's calls and the phases of
// the adjoint, for timeline profilers (visible when a profiler attaches an
// NVTX tool; otherwise each range costs a few nanoseconds).  Header-only
// NVTX v3 from the CUDA toolkit.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace nlc {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace nlc
