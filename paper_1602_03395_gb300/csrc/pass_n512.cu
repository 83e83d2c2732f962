// Line-pass kernels for lines of 512 points (generated list of instantiations;
// the line plan: 512 = 16x8x4, 16 points per thread, 8 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan512 = LinePlan<512, 16, 16,8,4>;

bool pass_kernel_512(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan512, KIND_FWD_PAPER, 8>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan512, KIND_FWD_FOLD, 8>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan512, KIND_ADJ_FOLD, 8>(); return true;
    default: return false;
  }
}

}  // namespace ffx
