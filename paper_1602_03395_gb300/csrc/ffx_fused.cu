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
#include "ffx_tcgen05.cuh"

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
// the launch waits for (k + 1) * gridDim.x arrivals, polling at most `spin`
// times (the plan's budget for waits on other blocks).
__device__ bool grid_barrier(unsigned* bar, unsigned target, long long spin, volatile int* s_abort) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this block's writes of the pass, before its arrival
    atomicAdd(bar, 1u);
    bool ok = false;
    for (long long i = 0; i < spin; ++i) {
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
    if (p + 1 < a.npass && !grid_barrier(a.bar, (unsigned)(p + 1) * gridDim.x, a.spin, &s_abort)) break;
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

// ---------------------------------------------------------------------------
// The same launch on the tensor cores, for lattices whose axes all have 64
// points.  A pass is D[line][row] = sum_K X[line][K] T[row][K] over real
// K = 128 (complex entries as 2 x 2 real blocks, rows and K interleaved as
// (re, im)), with split-TF32 operands as in the per-axis tensor-core kernel:
// head products in one TMEM accumulator, the cross terms in a second.  Work
// item = 128 lines (MMA M) x 32 real rows (MMA N = 16 complex outputs); block
// b owns row block b % 4 for the whole launch, so it keeps only that 32-row
// slice of each T_j (32 KB per axis) in shared memory.  Per item: each thread
// loads half of one line from L2 into registers and writes its values and
// tails into tensor memory (lane = line), where the MMAs read their A operand
// (shared memory then carries only T: reading both operands from it bounded
// the products); one thread issues 16 K-steps x 2 tcgen05.mma (N = 64 over the
// slice's head and tail rows for X_hi, N = 32 for X_lo) and commits to an
// mbarrier, and eight warps read the accumulators back (warp w: lane quarter
// w % 4, column half w / 4) and store.  Summing |.|^2 over the batch stays in
// registers.
// ---------------------------------------------------------------------------

constexpr int FT_N = 64;                       // points per line, every axis
constexpr int FT_K = 2 * FT_N;                 // real K
constexpr int FT_LINES = 128;                  // lines per item = MMA M
constexpr int FT_ROWS = 32;                    // real rows per item = MMA N
constexpr int FT_RB = FT_K / FT_ROWS;          // row blocks
constexpr int FT_THREADS = 256;
constexpr int FT_SBO = (FT_K / 4) * 128;       // 4096: between 8-row groups
constexpr int FT_TS_PART = FT_ROWS * FT_K * 4;  // 16 KB
constexpr int FT_TS_BYTES = 2 * FT_TS_PART;     // one row block's slice, head and tail
constexpr int FT_SMEM_USED = 3 * FT_TS_BYTES;   // 96 KB: the T slices (the input lives in tensor memory)
// requested per block: more than half an SM's shared memory, so that no two
// blocks share an SM (each allocates all 512 tensor-memory columns, and the
// grid barrier needs every block running)
constexpr int FT_SMEM = 160 * 1024;
static_assert(FT_SMEM >= FT_SMEM_USED && 2 * FT_SMEM > 228 * 1024, "one block per SM");
// Tensor memory: head and cross-term accumulators (FT_ROWS columns each), then
// the item's input as the MMAs' A operand, one line per lane: its FP32 values
// (head: an MMA of kind::tf32 reads only their TF32 bits) and its tails.
constexpr int FT_A_HI = 128, FT_A_LO = FT_A_HI + FT_K;
constexpr int FT_COLS = 512;                    // allocation (a power of two >= FT_A_LO + FT_K)
static_assert(FT_A_LO + FT_K <= FT_COLS && 2 * FT_ROWS <= FT_A_HI, "tensor-memory layout");
constexpr uint32_t kIdescFT = tc::idesc_tf32(FT_LINES, FT_ROWS);
// the slice's head and tail rows are contiguous 8-row groups: one N = 64
// product forms X_hi T_hi and X_hi T_lo side by side in the two accumulators
constexpr uint32_t kIdescFT2 = tc::idesc_tf32(FT_LINES, 2 * FT_ROWS);

__global__ void __launch_bounds__(FT_THREADS, 1) fused_tc_kernel(const FusedArgs a) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char fts[];
  unsigned char* tsl = fts;
  __shared__ __align__(8) uint64_t tbar, mbar, dbar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rb = (int)(blockIdx.x % FT_RB);  // gridDim.x is a multiple of FT_RB
  const int64_t cstep = gridDim.x / FT_RB, c0 = blockIdx.x / FT_RB;

  if (warp == 0) tmem_alloc(&tmem_slot, FT_COLS);
  if (tid == 0) {
    s_abort = 0;
    mbar_init(smem_u32(&tbar), 1);
    mbar_init(smem_u32(&mbar), 1);
    mbar_init(smem_u32(&dbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(smem_u32(&tbar), (uint32_t)(a.npass * FT_TS_BYTES));
    for (int p = 0; p < a.npass; ++p)
      bulk_g2s(smem_u32(tsl + p * FT_TS_BYTES), a.ts[p] + (size_t)rb * FT_TS_BYTES, FT_TS_BYTES, smem_u32(&tbar));
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  uint32_t phase = 0;
  unsigned barriers = 0;  // grid barriers passed
  bool slices = false;  // (thread 0) the T slices have landed
  bool issued = false;
  for (int p = 0; p < a.npass && !s_abort; ++p) {
    const FusedPass& P = a.pass[p];
    const int64_t inner = P.inner;
    const bool contiguous = (inner == 1);
    const int nb = P.acc ? (int)a.batch : 1;
    const int64_t ctiles = (P.ncols + FT_LINES - 1) / FT_LINES;
    const uint32_t th = smem_u32(tsl + p * FT_TS_BYTES);  // head rows, then the tail rows
    for (int64_t ct = c0; ct < ctiles && !s_abort; ct += cstep) {
      if (p == a.local_pass) {
        // this tile's input is written once the previous pass's four row blocks of it are
        if (tid == 0) {
          bool ok = false;
          for (long long i = 0; i < a.spin; ++i) {
            if (*(volatile unsigned*)(a.tile_done + ct) >= (unsigned)FT_RB) {
              ok = true;
              break;
            }
          }
          if (!ok) s_abort = 1;
          __threadfence();
        }
        __syncthreads();
        if (s_abort) break;
      }
      float racc[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) racc[m] = 0.f;
      for (int b = 0; b < nb && !s_abort; ++b) {
        // ---- the item's 128 lines into tensor memory, split: warp w writes the
        // lanes (lines) of its quarter w % 4 and the K half w / 4; every load
        // of the thread is issued before the first store
        {
          const int q = warp & 3, h = warp >> 2;
          const long long base = fused_line(P, ct * FT_LINES + 32 * q + lane, b);
          float x[64];  // complex points 32 h .. 32 h + 31 of the line, (re, im)
          if (contiguous) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float4 v = base >= 0 ? __ldcg(reinterpret_cast<const float4*>(P.in + base + 32 * h + 2 * j))
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
              x[4 * j] = v.x;
              x[4 * j + 1] = v.y;
              x[4 * j + 2] = v.z;
              x[4 * j + 3] = v.w;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float2 v = base >= 0 ? __ldcg(P.in + base + (int64_t)(32 * h + j) * inner) : make_float2(0.f, 0.f);
              x[2 * j] = v.x;
              x[2 * j + 1] = v.y;
            }
          }
          const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(64 * h);
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int m = 0; m < 16; ++m) {
              const float v = x[16 * g + m];
              hi[m] = __float_as_uint(v);
              lo[m] = __float_as_uint(v - tf32_head(v));
            }
            tmem_st16(trow + FT_A_HI + 16 * g, hi);
            tmem_st16(trow + FT_A_LO + 16 * g, lo);
          }
          tmem_wait_st();
        }
        tc_fence_before();
        __syncthreads();
        // ---- the product: 16 K-steps x 3 split products in 2 MMAs
        if (tid == 0 && !slices) slices = mbar_wait(smem_u32(&tbar), 0u, &s_abort);  // under the first load
        if (tid == 0 && slices) {
          tc_fence_after();
#pragma unroll 4
          for (int ks = 0; ks < FT_K / 8; ++ks) {
            const uint64_t dth = make_desc(th + (uint32_t)(ks * 256), 128, FT_SBO);
            const uint32_t more = ks > 0 ? 1u : 0u;
            // A from tensor memory: K columns 8 ks .. 8 ks + 7 of the head and tail
            mma_tf32_ts(tmem, tmem + FT_A_HI + 8 * ks, dth, kIdescFT2, more);         // [X_hi T_hi | X_hi T_lo]
            mma_tf32_ts(tmem + FT_ROWS, tmem + FT_A_LO + 8 * ks, dth, kIdescFT, 1u);  // + X_lo T_hi
          }
          mma_commit(smem_u32(&mbar));
          issued = true;
        }
        // warp-uniform outcome: the tensor-memory loads below need whole warps
        const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&mbar), phase, &s_abort));
        phase ^= 1u;
        if (!ok) break;
        tc_fence_after();
        // ---- epilogue: lanes = lines, columns = real rows
        const int q = warp & 3, h = warp >> 2;
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * h);
        float y[16];
        {
          uint32_t x1[16], x2[16];
          tmem_ld16(taddr, x1);
          tmem_ld16(taddr + FT_ROWS, x2);
          tmem_wait_ld();
#pragma unroll
          for (int m = 0; m < 16; ++m) y[m] = __uint_as_float(x1[m]) + __uint_as_float(x2[m]);
        }
        const long long base = fused_line(P, ct * FT_LINES + 32 * q + lane, b);
        const int n0 = rb * (FT_ROWS / 2) + 8 * h;  // complex outputs n0 .. n0 + 7
        if (P.acc) {
#pragma unroll
          for (int m = 0; m < 8; ++m) racc[m] += y[2 * m] * y[2 * m] + y[2 * m + 1] * y[2 * m + 1];
          if (b == nb - 1 && base >= 0) {
            const int64_t o0 = base - (int64_t)b * a.M + (int64_t)n0 * inner;
#pragma unroll
            for (int m = 0; m < 8; ++m) P.out_d[o0 + (int64_t)m * inner] += racc[m];
          }
        } else if (base >= 0) {
          if (contiguous && P.out_c && ((uintptr_t)P.out_c & 15) == 0) {
            float4* o = reinterpret_cast<float4*>(P.out_c + base + n0);  // base, n0 even: 16-byte aligned
#pragma unroll
            for (int m = 0; m < 4; ++m) o[m] = make_float4(y[4 * m], y[4 * m + 1], y[4 * m + 2], y[4 * m + 3]);
          } else if (contiguous && P.out_d && ((uintptr_t)P.out_d & 15) == 0) {
            float d[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) d[m] = y[2 * m] * y[2 * m] + y[2 * m + 1] * y[2 * m + 1];
            float4* o = reinterpret_cast<float4*>(P.out_d + base + n0);  // base, n0 multiples of 8
            o[0] = make_float4(d[0], d[1], d[2], d[3]);
            o[1] = make_float4(d[4], d[5], d[6], d[7]);
          } else {
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              const int64_t addr = base + (int64_t)(n0 + m) * inner;
              if (P.out_c)
                P.out_c[addr] = make_float2(y[2 * m], y[2 * m + 1]);
              else
                P.out_d[addr] = y[2 * m] * y[2 * m] + y[2 * m + 1] * y[2 * m + 1];
            }
          }
        }
        tc_fence_before();
        __syncthreads();  // accumulators read and shared tiles free before the next item
      }
      if (p + 1 == a.local_pass && tid == 0) {
        __threadfence();  // this row block of the tile is written
        atomicAdd(a.tile_done + ct, 1u);
      }
    }
    if (p + 1 < a.npass && p + 1 != a.local_pass) {
      ++barriers;
      if (!grid_barrier(a.bar, (unsigned)barriers * gridDim.x, a.spin, &s_abort)) break;
    }
  }
  // the tensor cores finish this block's work, and the slice copies have
  // landed, before the block exits
  if (tid == 0) {
    if (issued) {
      mma_commit(smem_u32(&dbar));
      mbar_wait_own(smem_u32(&dbar), 0u, &s_abort);
    }
    mbar_wait_own(smem_u32(&tbar), 0u, &s_abort);
  }
  tc_fence_before();
  __syncthreads();
  __shared__ int s_last;
  if (tid == 0) {
    if (s_abort && a.err) atomicAdd(a.err, 1);
    __threadfence();
    s_last = atomicAdd(a.bar + 1, 1u) == gridDim.x - 1;  // every block has left every barrier
  }
  __syncthreads();
  if (s_last) {
    // the last block out resets the counters for the next launch (stream order publishes them)
    if (a.local_pass > 0)
      for (int i = tid; i < kFusedTileFlags; i += FT_THREADS) a.tile_done[i] = 0u;
    if (tid == 0) {
      atomicExch(a.bar, 0u);
      atomicExch(a.bar + 1, 0u);
    }
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_free(tmem, FT_COLS);
  }
}

// Row-block slices of T (complex [64][64]) for the kernel above: block rb,
// [head | tail], real (r, k') with r = 32 rb + r_local, k' < 128 in the
// core-matrix order of a 32-row K-major operand.
__global__ void fused_tc_slices_kernel(const float2* __restrict__ T, unsigned char* __restrict__ out) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < FT_K * FT_K; idx += gridDim.x * blockDim.x) {
    const int r = idx / FT_K, kp = idx % FT_K;
    const float2 t = T[(r >> 1) * FT_N + (kp >> 1)];
    const int po = r & 1, pi = kp & 1;
    const float v = po == 0 ? (pi == 0 ? t.x : -t.y) : (pi == 0 ? t.y : t.x);
    const float hi = tc::tf32_round(v);
    const int blk = r / FT_ROWS, rl = r % FT_ROWS;
    unsigned char* base = out + (size_t)blk * FT_TS_BYTES;
    const int off = (rl >> 3) * FT_SBO + (kp >> 2) * 128 + (rl & 7) * 16 + (kp & 3) * 4;
    *reinterpret_cast<float*>(base + off) = hi;
    *reinterpret_cast<float*>(base + FT_TS_PART + off) = tc::tf32_round(v - hi);
  }
}

}  // namespace

size_t fused_tc_slice_bytes() { return (size_t)FT_RB * FT_TS_BYTES; }

cudaError_t launch_fused_tc_slices(const float2* T, unsigned char* out, cudaStream_t s) {
  fused_tc_slices_kernel<<<64, 256, 0, s>>>(T, out);
  return cudaGetLastError();
}

cudaError_t fused_tc_prepare(int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(fused_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, FT_SMEM);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fused_tc_kernel, FT_THREADS, FT_SMEM);
  return e;
}

cudaError_t launch_fused_tc(const FusedArgs& a, int grid, cudaStream_t stream) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)FT_THREADS);
  cfg.dynamicSmemBytes = FT_SMEM;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fused_tc_kernel, a);
}

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
