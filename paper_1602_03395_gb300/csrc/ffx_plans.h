// Line plans: points per thread (E; the threads per line follow, T = N/E) and
// line-groups per block (G) of every supported line length.  Every plan uses
// 256 threads per block (G * T).  One translation unit per length
// instantiates its kernels.
#pragma once

#include "ffx_fft.cuh"

namespace ffx {

using Plan16 = LinePlan<16, 4>;
constexpr int kGroups16 = 64;
using Plan32 = LinePlan<32, 8>;
constexpr int kGroups32 = 64;
using Plan48 = LinePlan<48, 12>;
constexpr int kGroups48 = 64;
using Plan64 = LinePlan<64, 8>;
constexpr int kGroups64 = 32;
using Plan96 = LinePlan<96, 12>;
constexpr int kGroups96 = 32;
using Plan128 = LinePlan<128, 8>;
constexpr int kGroups128 = 16;
using Plan192 = LinePlan<192, 12>;
constexpr int kGroups192 = 16;
using Plan256 = LinePlan<256, 8>;
constexpr int kGroups256 = 8;
using Plan384 = LinePlan<384, 12>;
constexpr int kGroups384 = 8;
using Plan512 = LinePlan<512, 16>;
constexpr int kGroups512 = 8;
using Plan768 = LinePlan<768, 12>;
constexpr int kGroups768 = 4;
using Plan1024 = LinePlan<1024, 16>;
constexpr int kGroups1024 = 4;
using Plan2048 = LinePlan<2048, 16>;
constexpr int kGroups2048 = 2;

}  // namespace ffx
