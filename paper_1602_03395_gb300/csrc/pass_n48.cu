// Line-pass kernels for lines of 48 points (generated list of instantiations;
// the line plan: 48 = 4x4x3, 12 points per thread, 64 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan48 = LinePlan<48, 12, 4,4,3>;

bool pass_kernel_48(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan48, KIND_FWD_PAPER, 64>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan48, KIND_FWD_FOLD, 64>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan48, KIND_ADJ_FOLD, 64>(); return true;
    default: return false;
  }
}

}  // namespace ffx
