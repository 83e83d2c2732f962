// Line-pass kernels for lines of 128 points (see ffx_plans.h for the line plan).
#include "ffx_pass.cuh"
#include "ffx_plans.h"

namespace ffx {

bool pass_kernel_128(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan128, KIND_FWD_PAPER, kGroups128>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan128, KIND_FWD_FOLD, kGroups128>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan128, KIND_ADJ_FOLD, kGroups128>(); return true;
    default: return false;
  }
}

}  // namespace ffx
