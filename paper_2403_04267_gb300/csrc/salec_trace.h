// salec_trace.h -- named ranges on the host timeline for profilers (NVTX v3, header only):
// every stepping and training entry point opens one for the length of the call, so that a
// timeline shows which call issued which kernels.  Without a tool attached the calls return
// at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace salec {

struct HostRange {
    explicit HostRange(const char* name) { nvtxRangePushA(name); }
    ~HostRange() { nvtxRangePop(); }
    HostRange(const HostRange&) = delete;
    HostRange& operator=(const HostRange&) = delete;
};

}  // namespace salec
