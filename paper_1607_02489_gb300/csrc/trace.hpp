// NVTX ranges (header-only NVTX 3: no library to link, and a no-op unless a tool
// such as Nsight Systems or Nsight Compute attaches) marking the library's
// phases: setup steps per level, the device setup, graph capture and autotuning,
// the V-cycle's launches per level and kernel class (when the cycle is enqueued
// for capture or profiled), and the FGMRES chunks.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <cstdio>

namespace emin {

class TraceRange {
 public:
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  TraceRange(const char* fmt, int a) {
    char buf[96];
    std::snprintf(buf, sizeof(buf), fmt, a);
    nvtxRangePushA(buf);
  }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

inline void trace_push(const char* name) { nvtxRangePushA(name); }
inline void trace_pop() { nvtxRangePop(); }

}  // namespace emin
