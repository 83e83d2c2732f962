// Line-pass kernels for lines of 128 points (generated list of instantiations;
// the line plan: 128 = 16x8, 16 points per thread, 32 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan128 = LinePlan<128, 16, 16,8>;

bool pass_kernel_128(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan128, KIND_FWD_PAPER, 32>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan128, KIND_FWD_FOLD, 32>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan128, KIND_ADJ_FOLD, 32>(); return true;
    default: return false;
  }
}

}  // namespace ffx
