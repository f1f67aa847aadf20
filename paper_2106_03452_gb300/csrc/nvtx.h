// NVTX ranges around the library's entry points and around each stage's
// launches (host side), so that a timeline profiler shows which call and
// which stage a kernel belongs to. NVTX v3 is header-only: without a
// profiler attached a range costs one predictable branch.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace dpsr {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Stage names by DPSR_K_* index (include/dpsr.h).
inline const char* stage_name(int kind) {
  static const char* const names[] = {"dpsr.bin",        "dpsr.plane_fwd",  "dpsr.xpass_fwd",
                                      "dpsr.final_fwd",  "dpsr.plane_inv",  "dpsr.plane_bfwd",
                                      "dpsr.final_bwd",  "dpsr.xpass_bwd",  "dpsr.plane_binv",
                                      "dpsr.combine"};
  return kind >= 0 && kind < (int)(sizeof(names) / sizeof(names[0])) ? names[kind] : "dpsr.stage";
}

}  // namespace dpsr
