// The per-axis dense map (see ffx_dense.cu) applied to a handful of lines.
#include "ffx_dense_lines.h"
#include "ffx_dense_tile.cuh"

namespace ffx {

namespace {

// Passes over fewer than kDenseFewLines lines (a 1-D field, a handful of
// realizations).  A 32-line tile would stay mostly empty and the work would sit
// on a few SMs; the FFT forms would take each line through its lam + 1 line
// transforms inside one block.  Here each warp owns one output row m and keeps
// T[m][.] in registers (lane l holds k = l + 32 i), so the rows of T spread
// over N / 8 blocks; the block stages LCOLS input lines at a time in shared
// memory (rows padded with zeros to 32 KPL >= N points, KPL a power of two),
// every thread's loads in flight together, and every dot product ends
// in the same shuffle tree.  With ensemble summing the realizations run in
// order, as in the tile kernels.  Not in place: every block reads every line.
constexpr int LCOLS = 4, LWARPS = 8;

template <int KPL>
__global__ void __launch_bounds__(32 * LWARPS) dense_lines_kernel(const DenseArgs a) {
  constexpr int XS = 32 * KPL;  // staged line stride (points)
  constexpr int FILL = LCOLS * XS / (32 * LWARPS);  // staged points per thread
  static_assert(FILL * 32 * LWARPS == LCOLS * XS, "staging covers the lines exactly");
  __shared__ __align__(16) float2 xs[LCOLS * XS];
  __shared__ long long cbase[LCOLS];
  __shared__ int cbr[LCOLS];
  const int N = a.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = blockIdx.x * LWARPS + warp;  // rows past N load zeros and store nothing
  const int64_t inner = a.inner;
  float2 t[KPL];
#pragma unroll
  for (int i = 0; i < KPL; ++i) {
    const int k = lane + 32 * i;
    t[i] = (m < N && k < N) ? __ldg(a.A + (size_t)m * N + k) : make_float2(0.f, 0.f);
  }
  const int nb = a.acc ? (int)a.batch : 1;
  const int64_t groups = (a.ncols + LCOLS - 1) / LCOLS;
  for (int64_t g = 0; g < groups; ++g) {
    float racc[LCOLS];
#pragma unroll
    for (int cc = 0; cc < LCOLS; ++cc) racc[cc] = 0.f;
    for (int b = 0; b < nb; ++b) {
      __syncthreads();  // the previous step is done with xs and cbase
      if (threadIdx.x < LCOLS) {
        const int64_t c = g * LCOLS + threadIdx.x;
        long long base = -1;
        int br = 0;
        if (c < a.ncols) {
          int64_t bo = c / inner;
          const int64_t i = c - bo * inner;
          if (a.acc) {
            br = b;
            bo += (int64_t)b * a.outer;
          } else {
            br = (int)(c / (a.outer * inner));
          }
          base = bo * (int64_t)N * inner + i;
        }
        cbase[threadIdx.x] = base;
        cbr[threadIdx.x] = br;
      }
      __syncthreads();
      {
        // all of a thread's loads in flight at once, then the stores
        float2 v[FILL];
        float gr[FILL];
#pragma unroll
        for (int r = 0; r < FILL; ++r) {
          const int idx = threadIdx.x + r * 32 * LWARPS;
          const int cc = idx / XS, k = idx - cc * XS;
          const long long base = cbase[cc];
          v[r] = make_float2(0.f, 0.f);
          gr[r] = 1.f;
          if (base >= 0 && k < N) {
            const int64_t addr = base + (int64_t)k * inner;
            v[r] = a.in[addr];
            if (a.grad) gr[r] = 2.f * __ldg(a.grad + (a.grad_shared ? addr - (int64_t)cbr[cc] * a.M : addr));
          }
        }
#pragma unroll
        for (int r = 0; r < FILL; ++r) xs[threadIdx.x + r * 32 * LWARPS] = make_float2(v[r].x * gr[r], v[r].y * gr[r]);
      }
      __syncthreads();
      float2 acc[LCOLS];
#pragma unroll
      for (int cc = 0; cc < LCOLS; ++cc) acc[cc] = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < KPL; ++i)
#pragma unroll
        for (int cc = 0; cc < LCOLS; ++cc) dcfma(acc[cc], t[i], xs[cc * XS + lane + 32 * i]);
#pragma unroll
      for (int cc = 0; cc < LCOLS; ++cc)
#pragma unroll
        for (int w = 16; w >= 1; w >>= 1) {
          acc[cc].x += __shfl_xor_sync(0xffffffffu, acc[cc].x, w);
          acc[cc].y += __shfl_xor_sync(0xffffffffu, acc[cc].y, w);
        }
      if (a.acc) {
#pragma unroll
        for (int cc = 0; cc < LCOLS; ++cc) racc[cc] += acc[cc].x * acc[cc].x + acc[cc].y * acc[cc].y;
      } else if (lane == 0 && m < N) {
#pragma unroll
        for (int cc = 0; cc < LCOLS; ++cc) {
          const long long base = cbase[cc];
          if (base < 0) continue;
          const int64_t addr = base + (int64_t)m * inner;
          if (a.out_c)
            a.out_c[addr] = acc[cc];
          else
            a.out_d[addr] = acc[cc].x * acc[cc].x + acc[cc].y * acc[cc].y;
        }
      }
    }
    if (a.acc && lane == 0 && m < N) {
      // cbase holds the last realization's bases
#pragma unroll
      for (int cc = 0; cc < LCOLS; ++cc) {
        const long long base = cbase[cc];
        if (base < 0) continue;
        a.out_d[base - (int64_t)(nb - 1) * a.M + (int64_t)m * inner] += racc[cc];
      }
    }
  }
}

}  // namespace

cudaError_t launch_dense_lines(const DenseArgs& a, cudaStream_t stream) {
  const int grid = (a.N + LWARPS - 1) / LWARPS;
  if (a.N <= 64)
    dense_lines_kernel<2><<<grid, 32 * LWARPS, 0, stream>>>(a);
  else if (a.N <= 128)
    dense_lines_kernel<4><<<grid, 32 * LWARPS, 0, stream>>>(a);
  else if (a.N <= 256)
    dense_lines_kernel<8><<<grid, 32 * LWARPS, 0, stream>>>(a);
  else if (a.N <= 512)
    dense_lines_kernel<16><<<grid, 32 * LWARPS, 0, stream>>>(a);
  else
    dense_lines_kernel<32><<<grid, 32 * LWARPS, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace ffx
