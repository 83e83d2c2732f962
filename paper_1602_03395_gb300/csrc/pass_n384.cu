// Line-pass kernels for lines of 384 points (generated list of instantiations;
// the line plan: 384 = 4x4x4x3x2, 12 points per thread, 8 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan384 = LinePlan<384, 12, 4,4,4,3,2>;

bool pass_kernel_384(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan384, KIND_FWD_PAPER, 8>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan384, KIND_FWD_FOLD, 8>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan384, KIND_ADJ_FOLD, 8>(); return true;
    default: return false;
  }
}

}  // namespace ffx
