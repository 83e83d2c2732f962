// Line-pass kernels for lines of 192 points (generated list of instantiations;
// the line plan: 192 = 4x4x4x3, 12 points per thread, 16 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan192 = LinePlan<192, 12, 4,4,4,3>;

bool pass_kernel_192(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan192, KIND_FWD_PAPER, 16>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan192, KIND_FWD_FOLD, 16>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan192, KIND_ADJ_FOLD, 16>(); return true;
    default: return false;
  }
}

}  // namespace ffx
