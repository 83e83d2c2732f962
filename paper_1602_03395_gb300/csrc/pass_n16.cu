// Line-pass kernels for lines of 16 points (generated list of instantiations;
// the line plan: 16 = 4x4, 4 points per thread, 64 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan16 = LinePlan<16, 4, 4,4>;

bool pass_kernel_16(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan16, KIND_FWD_PAPER, 64>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan16, KIND_FWD_FOLD, 64>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan16, KIND_ADJ_FOLD, 64>(); return true;
    default: return false;
  }
}

}  // namespace ffx
