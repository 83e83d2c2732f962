// Line-pass kernels for lines of 48 points (see ffx_plans.h for the line plan).
#include "ffx_pass.cuh"
#include "ffx_plans.h"

namespace ffx {

bool pass_kernel_48(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan48, KIND_FWD_PAPER, kGroups48>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan48, KIND_FWD_FOLD, kGroups48>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan48, KIND_ADJ_FOLD, kGroups48>(); return true;
    default: return false;
  }
}

}  // namespace ffx
