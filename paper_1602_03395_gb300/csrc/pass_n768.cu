// Line-pass kernels for lines of 768 points (see ffx_plans.h for the line plan).
#include "ffx_pass.cuh"
#include "ffx_plans.h"

namespace ffx {

bool pass_kernel_768(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan768, KIND_FWD_PAPER, kGroups768>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan768, KIND_FWD_FOLD, kGroups768>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan768, KIND_ADJ_FOLD, kGroups768>(); return true;
    default: return false;
  }
}

}  // namespace ffx
