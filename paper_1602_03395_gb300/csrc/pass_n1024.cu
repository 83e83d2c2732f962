// Line-pass kernels for lines of 1024 points (generated list of instantiations;
// the line plan: 1024 = 16x16x4, 16 points per thread, 4 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan1024 = LinePlan<1024, 16, 16,16,4>;

bool pass_kernel_1024(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan1024, KIND_FWD_PAPER, 4>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan1024, KIND_FWD_FOLD, 4>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan1024, KIND_ADJ_FOLD, 4>(); return true;
    default: return false;
  }
}

}  // namespace ffx
