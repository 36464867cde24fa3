// NVTX ranges around the library's entry points, so that a timeline tool (or
// ncu --nvtx) shows which call a kernel belongs to. Host-side only. Without an
// attached tool each range costs a check of a function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <cstdio>

namespace sindi {

class NvtxRange {
public:
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    // a name formatted from two integers (printf-style)
    NvtxRange(const char* fmt, long long a, long long b) {
        char buf[96];
        std::snprintf(buf, sizeof(buf), fmt, a, b);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace sindi
