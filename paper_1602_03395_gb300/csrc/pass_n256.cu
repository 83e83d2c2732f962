// Line-pass kernels for lines of 256 points (generated list of instantiations;
// the line plan: 256 = 16x16, 16 points per thread, 16 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan256 = LinePlan<256, 16, 16,16>;

bool pass_kernel_256(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan256, KIND_FWD_PAPER, 16>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan256, KIND_FWD_FOLD, 16>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan256, KIND_ADJ_FOLD, 16>(); return true;
    default: return false;
  }
}

}  // namespace ffx
