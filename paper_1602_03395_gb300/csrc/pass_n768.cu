// Line-pass kernels for lines of 768 points (generated list of instantiations;
// the line plan: 768 = 4x4x4x4x3, 12 points per thread, 4 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan768 = LinePlan<768, 12, 4,4,4,4,3>;

bool pass_kernel_768(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan768, KIND_FWD_PAPER, 4>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan768, KIND_FWD_FOLD, 4>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan768, KIND_ADJ_FOLD, 4>(); return true;
    default: return false;
  }
}

}  // namespace ffx
