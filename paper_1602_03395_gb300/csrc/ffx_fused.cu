// The whole forward map of a small lattice in one launch.
//
// When every axis is short (N_j <= 64) and takes the dense form, one pass of
// a realization is a few microseconds of work, and a batch of one cannot fill
// the GPU with three separate launches: each pass is a latency chain (launch,
// T arrives, input arrives, product, store) on a fraction of the SMs.  This
// kernel runs the d passes of the map (eq. FF factorised per axis, each axis
// a matrix T_j) in one cooperative launch with one block per SM:
//   * every block starts bulk copies of the shared-memory images of all d
//     matrices (one mbarrier each) and waits for T_j only when pass j needs it;
//   * pass p spreads its lines (64-point tiles of 32 lines) over all blocks,
//     reads its input with L2-only loads (the previous pass's output was
//     written by other SMs), and writes the next pass's input to the workspace
//     (in place from the second pass on: a tile's lines are read whole before
//     they are written, and the tiles of one pass are disjoint);
//   * a grid-wide barrier (an arrival counter in global memory with a bounded
//     wait; the last block to leave resets it for the next launch) separates
//     the passes;
//   * the last pass writes complex64, |.|^2, or |.|^2 summed over the batch
//     (a tile then loops over the realizations in order), or the detector
//     image: |.|^2 summed along the pass's axis, one value per line (Sec. 6).
// The arithmetic of a tile is that of the per-axis dense kernels (FP32 FMA,
// k ascending), so results match the unfused path bit for bit.
#include <cstring>

#include "ffx_internal.h"

namespace ffx {

namespace {

constexpr int FN = 64, FBN = 32;
constexpr int IMG_STRIDE = FN + 1;   // image rows: img[k][m] = T[m][k]
constexpr int BS_STRIDE = FBN + 1;
constexpr int BS_FLOATS2 = FN * BS_STRIDE;
constexpr long long kSpinLimit = 1ll << 22;

__device__ __forceinline__ void fcfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

__device__ __forceinline__ uint32_t fsm_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Line c of a pass (realization b when summing over the batch): offset of its
// first point, or -1 past the end.
__device__ __forceinline__ long long fused_line(const FusedPass& P, int64_t c, int b) {
  if (c >= P.ncols) return -1;
  int64_t bo = c / P.inner;
  const int64_t i = c - bo * P.inner;
  if (P.acc) bo += (int64_t)b * P.outer;
  return bo * (int64_t)P.N * P.inner + i;
}

// Bounded grid-wide barrier: block arrivals counted in bar[0]; barrier k of
// the launch waits for (k + 1) * gridDim.x arrivals.
__device__ bool grid_barrier(unsigned* bar, unsigned target, volatile int* s_abort) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this block's writes of the pass, before its arrival
    atomicAdd(bar, 1u);
    bool ok = false;
    for (long long i = 0; i < kSpinLimit; ++i) {
      if (*(volatile unsigned*)bar >= target) {
        ok = true;
        break;
      }
    }
    if (!ok) *s_abort = 1;
    __threadfence();
  }
  __syncthreads();
  return !*s_abort;
}

// Bounded wait on a phase-0 mbarrier by every thread; false if it ran out.
__device__ __forceinline__ bool wait_image(uint64_t* bar) {
  for (long long i = 0; i < kSpinLimit; ++i) {
    uint32_t d;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(d)
        : "r"(fsm_u32(bar))
        : "memory");
    if (d) return true;
  }
  return false;
}

// THREADS = 16 x TY threads cover a 64 x 32 tile; thread (tx, ty) owns rows
// ty + TY i (i < TM = 64 / TY) and lines tx + 16 j (j < 2): reads of both
// operands in shared memory are broadcasts or conflict-free.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1) fused_small_kernel(const FusedArgs a) {
  constexpr int TX = 16, TY = THREADS / TX, TM = FN / TY, TN = FBN / TX;
  constexpr int LOADS = FN * FBN / THREADS;  // input elements each thread loads per tile
  extern __shared__ __align__(16) unsigned char fsm[];
  float2* imgs = reinterpret_cast<float2*>(fsm);  // the passes' images, one after another
  float2* Bs = imgs + a.img_floats2;               // [2][FN][FBN + 1]
  __shared__ long long cbase[2][FBN];
  __shared__ __align__(8) uint64_t ibar[3];
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;

  // each pass's image on its own mbarrier: pass p waits only for T_p
  if (tid == 0) {
    s_abort = 0;
    for (int p = 0; p < a.npass; ++p)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(fsm_u32(&ibar[p])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int p = 0; p < a.npass; ++p) {
      const uint32_t nbytes = (uint32_t)(a.pass[p].N * IMG_STRIDE * sizeof(float2));
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fsm_u32(&ibar[p])), "r"(nbytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              fsm_u32(imgs + a.pass[p].img_off)),
          "l"(a.pass[p].img), "r"(nbytes), "r"(fsm_u32(&ibar[p]))
          : "memory");
    }
  }
  __syncthreads();

  for (int p = 0; p < a.npass && !s_abort; ++p) {
    const FusedPass& P = a.pass[p];
    const float2* As = imgs + P.img_off;
    const int N = P.N;
    const int64_t inner = P.inner;
    const bool contiguous = (inner == 1);
    const int64_t col_tiles = (P.ncols + FBN - 1) / FBN;
    const int nb = P.acc ? (int)a.batch : 1;
    const int64_t my_tiles = (blockIdx.x < col_tiles) ? (col_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const int64_t n_items = my_tiles * nb;

    float2 pre[LOADS];  // next tile's input, in flight during the current product
    auto bases = [&](int64_t it, int buf) {
      if (tid < FBN) {
        const int64_t cbk = blockIdx.x + (it / nb) * gridDim.x;
        cbase[buf][tid] = fused_line(P, cbk * FBN + tid, (int)(it % nb));
      }
    };
    auto load = [&](int buf) {
#pragma unroll
      for (int r = 0; r < LOADS; ++r) {
        const int idx = tid + r * THREADS;
        int k, cc;
        if (contiguous) {
          cc = idx / FN;
          k = idx - cc * FN;
        } else {
          k = idx / FBN;
          cc = idx - k * FBN;
        }
        const long long base = cbase[buf][cc];
        // L2 loads: the previous pass's output was written by other SMs
        pre[r] = (k < N && base >= 0) ? __ldcg(P.in + base + (int64_t)k * inner) : make_float2(0.f, 0.f);
      }
    };
    auto park = [&](int buf) {
      float2* dst = Bs + buf * BS_FLOATS2;
#pragma unroll
      for (int r = 0; r < LOADS; ++r) {
        const int idx = tid + r * THREADS;
        int k, cc;
        if (contiguous) {
          cc = idx / FN;
          k = idx - cc * FN;
        } else {
          k = idx / FBN;
          cc = idx - k * FBN;
        }
        dst[k * BS_STRIDE + cc] = pre[r];
      }
    };

    if (n_items > 0) {
      bases(0, 0);
      __syncthreads();
      load(0);
      park(0);
    }
    // T_p is needed from here on (its copy ran under the previous passes)
    if (!wait_image(&ibar[p])) s_abort = 1;
    float racc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) racc[i][j] = 0.f;

    for (int64_t it = 0; it < n_items; ++it) {
      const int buf = (int)(it & 1);
      __syncthreads();  // Bs[buf] is complete; Bs[buf ^ 1] and cbase[buf ^ 1] are free
      if (s_abort) break;
      const bool more = it + 1 < n_items;
      if (more) bases(it + 1, buf ^ 1);
      __syncthreads();
      if (more) load(buf ^ 1);
      const float2* B = Bs + buf * BS_FLOATS2;

      float2 acc[TM][TN];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int k = 0; k < N; ++k) {
        float2 av[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) av[i] = As[k * IMG_STRIDE + ty + TY * i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = B[k * BS_STRIDE + tx + TX * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) fcfma(acc[i][j], av[i], bv[j]);
      }

      const int b = (int)(it % nb);
      const bool tile_done = !P.acc || b == nb - 1;
      if (P.acc) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) racc[i][j] += acc[i][j].x * acc[i][j].x + acc[i][j].y * acc[i][j].y;
      }
      if (tile_done) {
        // stage the tile (rows m, columns cc) in Bs[buf] and store it coalesced
        float2* S = Bs + buf * BS_FLOATS2;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            float2 v = acc[i][j];
            if (P.acc) v = make_float2(racc[i][j], 0.f);
            S[(ty + TY * i) * BS_STRIDE + tx + TX * j] = v;
          }
        __syncthreads();
        if (P.out_col) {
          // detector image: one sum over the tile's rows per line, in row order
          if (tid < FBN) {
            const int64_t c = (blockIdx.x + (it / nb) * gridDim.x) * FBN + tid;
            if (c < P.ncols) {
              float sum = 0.f;
              for (int m = 0; m < N; ++m) {
                const float2 v = S[m * BS_STRIDE + tid];
                sum += P.acc ? v.x : v.x * v.x + v.y * v.y;
              }
              P.out_col[c] = P.acc ? P.out_col[c] + P.col_scale * sum : P.col_scale * sum;
            }
          }
        } else {
          for (int idx = tid; idx < N * FBN; idx += THREADS) {
            int m, cc;
            if (contiguous) {
              cc = idx / N;
              m = idx - cc * N;
            } else {
              m = idx / FBN;
              cc = idx - m * FBN;
            }
            const long long base = cbase[buf][cc];
            if (base < 0) continue;
            const float2 v = S[m * BS_STRIDE + cc];
            if (P.acc) {
              P.out_d[base - (int64_t)b * a.M + (int64_t)m * inner] += v.x;
            } else {
              const int64_t addr = base + (int64_t)m * inner;
              if (P.out_c)
                P.out_c[addr] = v;
              else
                P.out_d[addr] = v.x * v.x + v.y * v.y;
            }
          }
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) racc[i][j] = 0.f;
      }
      if (more) park(buf ^ 1);
    }
    if (p + 1 < a.npass && !grid_barrier(a.bar, (unsigned)(p + 1) * gridDim.x, &s_abort)) break;
  }
  // copies of images not waited for must land before the block exits
  for (int p = 0; p < a.npass; ++p)
    if (!wait_image(&ibar[p])) s_abort = 1;
  __syncthreads();
  if (tid == 0) {
    if (s_abort && a.err) atomicAdd(a.err, 1);
    // the last block out resets the barrier counters for the next launch
    // (every block has left every barrier by then)
    __threadfence();
    if (atomicAdd(a.bar + 1, 1u) == gridDim.x - 1) {
      atomicExch(a.bar, 0u);
      atomicExch(a.bar + 1, 0u);
    }
  }
}

constexpr int kFusedThreads = 512;

}  // namespace

size_t fused_smem(const int* N, int npass) {
  size_t img = 0;
  for (int p = 0; p < npass; ++p) img += (size_t)N[p] * IMG_STRIDE;
  return (img + 2 * BS_FLOATS2) * sizeof(float2);
}
int fused_img_stride() { return IMG_STRIDE; }
const void* fused_func() { return (const void*)fused_small_kernel<kFusedThreads>; }
int fused_threads() { return kFusedThreads; }

cudaError_t launch_fused(const FusedArgs& a, int grid, size_t smem, cudaStream_t stream) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)kFusedThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;  // every block resident at once, or no launch
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fused_small_kernel<kFusedThreads>, a);
}

}  // namespace ffx
