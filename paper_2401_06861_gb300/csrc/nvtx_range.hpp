// NVTX ranges around the library's entry points and sweep launches, for
// profilers (nsys, ncu --nvtx); off unless the environment sets NWQ_NVTX=1.
#pragma once
#include <nvtx3/nvToolsExt.h>

#include <cstdlib>

namespace nwq {

inline bool nvtx_on() {
  static const bool on = [] {
    const char* e = std::getenv("NWQ_NVTX");
    return e && e[0] == '1';
  }();
  return on;
}

struct NvtxRange {
  bool on;
  explicit NvtxRange(const char* name) : on(nvtx_on()) {
    if (on) nvtxRangePushA(name);
  }
  ~NvtxRange() {
    if (on) nvtxRangePop();
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace nwq
