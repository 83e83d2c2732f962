// Line-pass kernels for lines of 32 points (generated list of instantiations;
// the line plan: 32 = 8x4, 8 points per thread, 64 lines per block).
#include "ffx_pass.cuh"

namespace ffx {

using Plan32 = LinePlan<32, 8, 8,4>;

bool pass_kernel_32(int kind, PassKernelInfo* out) {
  switch (kind) {
    case KIND_FWD_PAPER: *out = pass_info<Plan32, KIND_FWD_PAPER, 64>(); return true;
    case KIND_FWD_FOLD: *out = pass_info<Plan32, KIND_FWD_FOLD, 64>(); return true;
    case KIND_ADJ_FOLD: *out = pass_info<Plan32, KIND_ADJ_FOLD, 64>(); return true;
    default: return false;
  }
}

}  // namespace ffx
