// Host-side NVTX ranges (visible in Nsight Systems timelines; free when no
// tool is attached).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace tc {

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace tc
