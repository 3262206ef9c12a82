// NVTX ranges around the library's host entry points (lbm_step, lbm_batch_step, the
// surrogate's training, inference and rollout), so that a timeline profiler shows
// which call enqueued which kernels.  NVTX v3 is header-only and looks for a tool at
// run time: without one attached a range costs a function call and nothing else.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace evtrace {

struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

}  // namespace evtrace
