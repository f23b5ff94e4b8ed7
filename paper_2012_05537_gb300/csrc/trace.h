// Host-side tracing of the library's public calls.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace sllbm {

// A named NVTX range over the rest of the enclosing scope (each public call that launches
// work opens one, so that a profiler's timeline shows the library's calls; with no tool
// attached the NVTX calls return at once).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace sllbm
