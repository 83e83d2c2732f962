// Detector readout (Sec. 6): the density integrated along one lattice axis,
// and the fringe-phase estimate of eq. dphase2 from such an image.
//
// axis_sum_kernel: out[o][i] = scale * sum_n rho[o][n][i] (+= with acc), for a
// density laid out [outer][N][inner]; scale = lam_axis * dx_axis, the spacing
// of the magnified lattice along the axis (eq. wbx).  A thread owns one output
// when inner > 1 (reads coalesced along i); a warp owns one output when the
// axis is contiguous (inner = 1), its lanes striding over n and reducing by a
// fixed shuffle tree.  Either way the sum order is fixed: deterministic.
//
// fringe_kernel: per image row (one warp each), the interior local maximum
// rho[j] > rho[j-1], rho[j] >= rho[j+1] with the smallest |y_j| (the lower j on
// a tie), y_j = y0 + j dy; its position refined by the vertex of the parabola
// through log rho at j-1, j, j+1 (FP64); phase = y_peak D / t (hbar = m = 1).
// Rows without an interior maximum get NaN.
#include <cmath>

#include "ffx_internal.h"

namespace ffx {

namespace {

__global__ void axis_sum_kernel(const float* __restrict__ rho, int64_t outer, int N, int64_t inner, float scale,
                                int acc, float* __restrict__ out) {
  const int64_t total = outer * inner;
  if (inner == 1) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < total; o += warps) {
      const float* line = rho + o * N;
      float s = 0.f;
      for (int n = lane; n < N; n += 32) s += line[n];
#pragma unroll
      for (int w = 16; w >= 1; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
      if (lane == 0) out[o] = acc ? out[o] + scale * s : scale * s;
    }
    return;
  }
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = idx / inner, i = idx - o * inner;
    const float* p = rho + o * N * inner + i;
    float s = 0.f;
    for (int n = 0; n < N; ++n) s += p[(int64_t)n * inner];
    out[idx] = acc ? out[idx] + scale * s : scale * s;
  }
}

__device__ __forceinline__ double y_at(double y0, double dy, int64_t j) {
  return __dadd_rn(y0, __dmul_rn(dy, (double)j));  // no contraction: y0 + dy * j as written
}

__global__ void fringe_kernel(const float* __restrict__ img, int64_t rows, int64_t ny, int64_t rs, int64_t ys,
                              double y0, double dy, double D, double t, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += warps) {
    const float* row = img + r * rs;
    int64_t best = -1;
    double best_ay = 0.0;
    for (int64_t j = 1 + lane; j < ny - 1; j += 32) {
      const float v = row[j * ys];
      if (v > row[(j - 1) * ys] && v >= row[(j + 1) * ys]) {
        const double ay = fabs(y_at(y0, dy, j));
        if (best < 0 || ay < best_ay) {  // j grows within a lane: ties keep the lower j
          best = j;
          best_ay = ay;
        }
      }
    }
    // warp argmin over (|y|, j)
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
      const int64_t ob = __shfl_xor_sync(0xffffffffu, best, w);
      const double oa = __shfl_xor_sync(0xffffffffu, best_ay, w);
      if (ob >= 0 && (best < 0 || oa < best_ay || (oa == best_ay && ob < best))) {
        best = ob;
        best_ay = oa;
      }
    }
    if (lane == 0) {
      double phase = nan("");
      if (best >= 0) {
        const double rm = row[(best - 1) * ys], r0 = row[best * ys], rp = row[(best + 1) * ys];
        double shift = 0.0;
        if (rm > 0.0 && r0 > 0.0 && rp > 0.0) {
          const double lm = log(rm), l0 = log(r0), lp = log(rp);
          const double curv = lm - 2.0 * l0 + lp;
          if (curv != 0.0) shift = 0.5 * (lm - lp) / curv;
        }
        phase = (y_at(y0, dy, best) + shift * dy) * D / t;
      }
      out[r] = phase;
    }
  }
}

}  // namespace

cudaError_t launch_axis_sum(const float* rho, int64_t outer, int N, int64_t inner, float scale, int acc, float* out,
                            int sms, cudaStream_t s) {
  const int64_t total = outer * inner;
  const int64_t threads = inner == 1 ? total * 32 : total;
  int64_t blocks = (threads + 255) / 256;
  if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
  if (blocks < 1) blocks = 1;
  axis_sum_kernel<<<(unsigned)blocks, 256, 0, s>>>(rho, outer, N, inner, scale, acc, out);
  return cudaGetLastError();
}

cudaError_t launch_fringe(const float* img, int64_t rows, int64_t ny, int64_t rs, int64_t ys, double y0, double dy,
                          double D, double t, double* out, int sms, cudaStream_t s) {
  int64_t blocks = (rows * 32 + 255) / 256;
  if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
  if (blocks < 1) blocks = 1;
  fringe_kernel<<<(unsigned)blocks, 256, 0, s>>>(img, rows, ny, rs, ys, y0, dy, D, t, out);
  return cudaGetLastError();
}

}  // namespace ffx
