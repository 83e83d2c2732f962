// Line-pass kernels for lines of 2048 points (generated list of instantiations;
// the line plan: 2048 = 16x16x8, 16 points per thread, 2 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan2048 = LinePlan<2048, 16, 16,16,8>;

bool pass_kernel_2048(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan2048, KIND_FWD_PAPER, 2>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan2048, KIND_FWD_FOLD, 2>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan2048, KIND_ADJ_FOLD, 2>(); return true;
    default: return false;
  }
}

}  // namespace ffx
