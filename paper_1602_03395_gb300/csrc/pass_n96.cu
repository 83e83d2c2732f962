// Line-pass kernels for lines of 96 points (generated list of instantiations;
// the line plan: 96 = 4x4x3x2, 12 points per thread, 32 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan96 = LinePlan<96, 12, 4,4,3,2>;

bool pass_kernel_96(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan96, KIND_FWD_PAPER, 32>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan96, KIND_FWD_FOLD, 32>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan96, KIND_ADJ_FOLD, 32>(); return true;
    default: return false;
  }
}

}  // namespace ffx
