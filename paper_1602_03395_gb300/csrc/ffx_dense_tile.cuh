// One 64 x 32 output tile of the generic dense pass (ffx_dense.cu), shared by
// the uniform dense kernel and the many-instance dense phases (ffx_many.cu).
// Thread (tx, ty) of 256 owns rows ty + 16 i (i < 4) and columns tx + 16 j
// (j < 2); K runs in chunks of 16 through shared memory.  The epilogue writes
// complex64, or |.|^2, or |.|^2 summed over the batch (the tile then loops
// over b in order).  Not in place for N > 64: the row blocks of one column
// run in different tiles.
#pragma once

#include "ffx_internal.h"

namespace ffx {

constexpr int DBM = 64, DBN = 32, DBK = 16, DTX = 16, DTY = 16, DTM = 4, DTN = 2;

struct DenseTileSmem {
  float2 As[DBK][DBM + 1];
  float2 Bs[DBK][DBN + 1];
  long long cbase[DBN];
  int cb[DBN];
};

__device__ __forceinline__ void dcfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

__host__ __device__ inline int64_t dense_tile_count(int N, int64_t ncols) {
  return (int64_t)((N + DBM - 1) / DBM) * ((ncols + DBN - 1) / DBN);
}

// Tile `tile` of the pass a (tiles run row block fastest).
__device__ __forceinline__ void dense_tile(const DenseArgs& a, int64_t tile, DenseTileSmem& sm) {
  auto& As = sm.As;
  auto& Bs = sm.Bs;
  auto& cbase = sm.cbase;
  auto& cb = sm.cb;
  const int N = a.N;
  const int tx = threadIdx.x % DTX, ty = threadIdx.x / DTX;
  const int64_t inner = a.inner;
  const bool contiguous = (inner == 1);
  const int64_t ncols = a.ncols;
  const int row_blocks = (N + DBM - 1) / DBM;
  const int nb_loop = a.acc ? (int)a.batch : 1;
  const int64_t per_real = a.outer * inner;
  const int rb = (int)(tile % row_blocks);
  const int64_t cbk = tile / row_blocks;
  const int m0 = rb * DBM;
  const int64_t c0 = cbk * DBN;
  float racc[DTM][DTN];
#pragma unroll
  for (int i = 0; i < DTM; ++i)
#pragma unroll
    for (int j = 0; j < DTN; ++j) racc[i][j] = 0.f;

  for (int bl = 0; bl < nb_loop; ++bl) {
    __syncthreads();
    if (threadIdx.x < DBN) {
      const int64_t c = c0 + threadIdx.x;
      long long base = -1;
      int b = 0;
      if (c < ncols) {
        int64_t bo = c / inner;
        const int64_t i = c - bo * inner;
        if (a.acc) {
          b = bl;
          bo += (int64_t)bl * a.outer;
        } else {
          b = (int)(c / per_real);
        }
        base = bo * (int64_t)N * inner + i;
      }
      cbase[threadIdx.x] = base;
      cb[threadIdx.x] = b;
    }
    float2 acc[DTM][DTN];
#pragma unroll
    for (int i = 0; i < DTM; ++i)
#pragma unroll
      for (int j = 0; j < DTN; ++j) acc[i][j] = make_float2(0.f, 0.f);

    for (int k0 = 0; k0 < N; k0 += DBK) {
      __syncthreads();  // previous chunk consumed; cbase visible
      // A chunk: As[kk][mm] = T[m0 + mm][k0 + kk]
      for (int idx = threadIdx.x; idx < DBK * DBM; idx += 256) {
        const int mm = idx / DBK, kk = idx - mm * DBK;
        const int m = m0 + mm, k = k0 + kk;
        As[kk][mm] = (m < N && k < N) ? __ldg(a.A + (size_t)m * N + k) : make_float2(0.f, 0.f);
      }
      // B chunk: Bs[kk][cc] = in[col c0 + cc][row k0 + kk]
      for (int idx = threadIdx.x; idx < DBK * DBN; idx += 256) {
        int kk, cc;
        if (contiguous) {
          cc = idx / DBK;
          kk = idx - cc * DBK;
        } else {
          kk = idx / DBN;
          cc = idx - kk * DBN;
        }
        const int k = k0 + kk;
        const long long base = cbase[cc];
        float2 v = make_float2(0.f, 0.f);
        if (base >= 0 && k < N) {
          const int64_t addr = base + (int64_t)k * inner;
          v = a.in[addr];  // plain load: passes may run in place
          if (a.grad) {
            const int64_t gaddr = a.grad_shared ? addr - (int64_t)cb[cc] * a.M : addr;
            const float gr = 2.f * __ldg(a.grad + gaddr);
            v.x *= gr;
            v.y *= gr;
          }
        }
        Bs[kk][cc] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < DBK; ++kk) {
        float2 av[DTM], bv[DTN];
#pragma unroll
        for (int i = 0; i < DTM; ++i) av[i] = As[kk][ty + DTY * i];
#pragma unroll
        for (int j = 0; j < DTN; ++j) bv[j] = Bs[kk][tx + DTX * j];
#pragma unroll
        for (int i = 0; i < DTM; ++i)
#pragma unroll
          for (int j = 0; j < DTN; ++j) dcfma(acc[i][j], av[i], bv[j]);
      }
    }
    // epilogue for this realization
    __syncthreads();  // all reads of this realization's inputs are done (in-place passes)
    if (a.acc) {
#pragma unroll
      for (int i = 0; i < DTM; ++i)
#pragma unroll
        for (int j = 0; j < DTN; ++j) racc[i][j] += acc[i][j].x * acc[i][j].x + acc[i][j].y * acc[i][j].y;
    } else {
#pragma unroll
      for (int i = 0; i < DTM; ++i) {
        const int m = m0 + ty + DTY * i;
        if (m >= N) continue;
#pragma unroll
        for (int j = 0; j < DTN; ++j) {
          const int cc = tx + DTX * j;
          const long long base = cbase[cc];
          if (base < 0) continue;
          const int64_t addr = base + (int64_t)m * inner;
          if (a.out_c)
            a.out_c[addr] = acc[i][j];
          else
            a.out_d[addr] = acc[i][j].x * acc[i][j].x + acc[i][j].y * acc[i][j].y;
        }
      }
    }
  }
  if (a.acc) {
#pragma unroll
    for (int i = 0; i < DTM; ++i) {
      const int m = m0 + ty + DTY * i;
      if (m >= N) continue;
#pragma unroll
      for (int j = 0; j < DTN; ++j) {
        const int cc = tx + DTX * j;
        const long long base = cbase[cc];
        if (base < 0) continue;
        const int64_t addr = base - (int64_t)(nb_loop - 1) * a.M + (int64_t)m * inner;
        a.out_d[addr] += racc[i][j];
      }
    }
  }
}

}  // namespace ffx
