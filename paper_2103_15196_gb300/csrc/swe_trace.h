// Named NVTX ranges over the library's host calls (step, state copies,
// ensemble and surrogate phases), so profilers can attribute and filter the
// launches; without a profiler attached a range costs a few nanoseconds.
#pragma once
#include <nvtx3/nvToolsExt.h>

struct SweRange {
    explicit SweRange(const char *name) { nvtxRangePushA(name); }
    ~SweRange() { nvtxRangePop(); }
    SweRange(const SweRange &) = delete;
    SweRange &operator=(const SweRange &) = delete;
};
