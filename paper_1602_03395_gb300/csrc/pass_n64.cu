// Line-pass kernels for lines of 64 points (generated list of instantiations;
// the line plan: 64 = 8x8, 8 points per thread, 32 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan64 = LinePlan<64, 8, 8,8>;

bool pass_kernel_64(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan64, KIND_FWD_PAPER, 32>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan64, KIND_FWD_FOLD, 32>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan64, KIND_ADJ_FOLD, 32>(); return true;
    default: return false;
  }
}

}  // namespace ffx
