// Dense form, few-lines kernel: one pass over fewer than kDenseFewLines lines
// in the whole call (batch x lines), one warp per row of T.
#pragma once

#include "ffx_internal.h"

namespace ffx {

constexpr int kDenseFewLines = 32;
// A pass of the dense form (DenseArgs as for launch_dense) by the few-lines
// kernel; not in place.
cudaError_t launch_dense_lines(const DenseArgs& a, cudaStream_t stream);

}  // namespace ffx
