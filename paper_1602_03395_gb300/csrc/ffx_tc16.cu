// Dense form on the tensor cores with BF16 operands (tcgen05 kind::f16): the
// per-axis map of lines of N points (N a multiple of 32, from 64 up to 1024)
// as a real matrix product, split into BF16 heads and tails, accumulated in
// FP32 in tensor memory.
//
// The real form of the complex map is that of the split-TF32 kernel
// (ffx_tc.cu): every complex entry t = x + iy of T becomes the 2 x 2 block
// [[x, -y], [y, x]], every complex input v = a + ib the pair (a, b), and the
// product runs transposed, D[line][row] = sum_K X[line][K] T[row][K], so that
// tensor-memory lane = line.  Each FP32 operand value v is split into
// hi = bf16_rn(v) and lo = bf16_rn(v - hi): T at plan time, the input on the
// fly.  X_hi T_hi accumulates in one FP32 accumulator and X_hi T_lo + X_lo T_hi
// in a second one (the large accumulator then takes only 2N/16 steps, which
// keeps the tensor cores' biased FP32 accumulation small); the lo*lo term and
// the tails' own rounding leave ~2^-16 per operand pair, measured ~1e-6 on
// the density.  Unsplit launches run X_hi T_hi alone (~2^-8 per product; the
// reported BF16 variant).
//
// Against the split-TF32 kernel, a K-step covers 16 real K in the same 32
// bytes of every operand row, so the shared-memory bytes per K halve for the
// operands; the products run at the kind::f16 rate.  The FP32 input of a chunk
// (32 KB) is exactly the size of its BF16 head and tail parts, so it lands in
// the stage itself, each thread's bytes where its own BF16 rows go, and is
// converted in place: no separate input ring, three 64 KB stages.
//
// Kernel: one persistent block of 416 threads per SM, warp-specialised.
//  * warps 0-7 (producers), per K chunk of 64 real K, once the products of
//    the chunk three back have freed its stage: thread 0 starts a bulk copy of
//    the pre-split T chunk (head and tail, 128 rows x 64 K each, already in
//    the tensor cores' K-major no-swizzle core-matrix order) on the stage's
//    "copy" barrier, and every producer thread copies its share of the input
//    into the stage (cp.async); two chunks later the thread converts its share
//    into BF16 heads and tails in place (16-byte core-matrix rows, conflict
//    free) and arrives on "full".
//  * warp 8 (MMA): waits "copy" and "full", issues 4 K-steps x 3 products of
//    tcgen05.mma kind::f16 (M = 128 lines, N = 128 rows, K = 16) into one of
//    two accumulator pairs; tcgen05.commit frees the stage ("empty") and,
//    after an item's last chunk, hands the accumulator on ("acc_full").
//  * warps 9-12 (epilogue): read their 32-lane quarter of the accumulators,
//    store complex64 or |.|^2 (or add |.|^2 over the batch in shared memory),
//    and arrive on "acc_empty".
// Items are (128 lines, 128 real rows) of the output, numbered row block
// fastest so that blocks running together share the lines' inputs in L2.
//
// BF16 pass chains: the d passes of a forward map run from the last axis to
// the first, and every pass but the last writes its output as BF16 head and
// tail planes, transposed: point n' of line rho (of R lines per realization)
// goes to n' R + rho, so that the next axis is the contiguous one for the next
// pass and, after the pass along axis 0, the lattice is back in its own
// order.  The epilogue makes the split the next pass would have made of the
// same FP32 value (bitwise the same operands), and writes 32 consecutive
// lines per warp store.  A pass with BF16 planes as input needs no producers:
// thread 0 loads each chunk's head and tail rows as one TMA tile (a 3-D map
// over [plane][line][2N], 128-byte swizzle) straight into the layout the
// tensor cores read (K-major, 128-byte swizzle), next to the T chunk.
// Every wait is bounded; one that runs out sets the block's abort flag, the
// block drains its own copies and products, frees its tensor memory, counts
// the error and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstring>

#include "ffx_internal.h"
#include "ffx_tc_many.h"
#include "ffx_tcgen05.cuh"

namespace ffx {

namespace {

using namespace tc;

constexpr int BL = 128;                      // lines per item = MMA M = tensor-memory lanes
constexpr int BR = 128;                      // real output rows per item = MMA N
constexpr int BKC = 64;                      // real K per chunk: four K-steps of 16
constexpr int BSMAX = 3;  // stages: 3, or 2 in backward launches (their gradient ring)
constexpr int BCORE = 128;                   // bytes between core matrices along K
constexpr int BSBO = (BKC / 8) * BCORE;      // 1024: between 8-row groups
constexpr int BPART = BR * BKC * 2;          // 16 KB: one split part of a chunk (T or X)
constexpr int BTCHUNK = 2 * BPART;           // T chunk: head, tail
// X area of a stage: the BF16 head and tail parts (2 x 16 KB), where the FP32
// input of the chunk (32 KB) lands first
constexpr int BXAREA = 2 * BPART;
constexpr int BSTAGE = BTCHUNK + BXAREA;     // 64 KB
constexpr int BPROD = 256, BEPI = 128;
constexpr int BTHREADS = BPROD + 32 + BEPI;  // 416
constexpr int BMMA_WARP = BPROD / 32;        // warp 8; warps 9-12 are the epilogue
constexpr int BITEMS = BL * (BKC / 8) / BPROD;  // 4 core-matrix rows (8 real K) per producer thread per chunk
constexpr int BGRAD_CHUNK = BPROD * BITEMS * 16;  // 16 KB: a chunk's gradient factors (backward passes)
constexpr int BEXTRA = (BR / 2) * BL * 4;       // accumulating launches: |.|^2 over the batch, [row][line]
constexpr int BCOLS = 4 * BR;                   // two accumulator pairs: all 512 columns
__host__ __device__ constexpr int bstages(bool grad, bool acc) { return grad ? 2 : 3; }
// stages, then the |.|^2 sums of accumulating launches or the gradient ring
__host__ __device__ constexpr int bsmem(bool grad, bool acc) {
  return bstages(grad, acc) * BSTAGE + (acc ? BEXTRA : 0) + (grad ? bstages(grad, acc) * BGRAD_CHUNK : 0);
}
// a launch's dynamic shared memory: 1 KB more, to start the stages on a
// 1024-byte boundary (the swizzled tiles' atoms)
__host__ __device__ constexpr int bsmem_launch(bool grad, bool acc) { return bsmem(grad, acc) + 1024; }
static_assert(bsmem_launch(false, true) <= 227 * 1024 && bsmem_launch(true, false) <= 227 * 1024, "shared memory");

// The 256 producer threads' named barrier (id 1): every thread passes its
// flag and gets the AND of all of them, so that a decision to stop is the
// same in every producer thread; a plain one (id 2) orders their shared-memory
// accesses.
__device__ __forceinline__ bool prod_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(BPROD)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void prod_sync() { asm volatile("bar.sync 2, %0;" ::"n"(BPROD) : "memory"); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
static_assert(BITEMS == 4, "producer mapping");

__host__ __device__ __forceinline__ int brow_count(int N, int mt) {
  const int left = 2 * N - mt * BR;
  return left < BR ? left : BR;
}

// Line c of the pass (realization b when accumulating): offset of its first
// point, or -1 past the end; br = its realization.
__device__ __forceinline__ long long bline(const DenseArgs& a, int64_t c, int b, int& br) {
  br = 0;
  if (c >= a.ncols) return -1;
  int64_t bo = c / a.inner;
  const int64_t i = c - bo * a.inner;
  if (a.acc) {
    br = b;
    bo += (int64_t)b * a.outer;
  } else {
    br = (int)(c / (a.outer * a.inner));
  }
  return bo * (int64_t)a.N * a.inner + i;
}

// The same for the output, with the output's decomposition (oouter, oinner).
__device__ __forceinline__ long long bline_o(const DenseArgs& a, int64_t c, int b, int& br) {
  br = 0;
  if (c >= a.ncols) return -1;
  int64_t bo = c / a.oinner;
  const int64_t i = c - bo * a.oinner;
  if (a.acc) {
    br = b;
    bo += (int64_t)b * a.oouter;
  } else {
    br = (int)(c / (a.oouter * a.oinner));
  }
  return bo * (int64_t)a.N * a.oinner + i;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo_k, hi_k);  // .x (element k) in the low half
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Split 8 consecutive real K values into their BF16 heads and tails.
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo, bool unsplit) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * m], v[2 * m + 1]);
    h[m] = *reinterpret_cast<const uint32_t*>(&hb);
    if (!unsplit) {
      const float2 hf = __bfloat1622float2(hb);
      l[m] = pack_bf16(v[2 * m] - hf.x, v[2 * m + 1] - hf.y);
    } else {
      l[m] = 0u;
    }
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// How a chunk's input reaches the stage: a TMA tile of contiguous lines (a
// 2-D map over [lines][2N floats], two 128 x 32-float boxes with 128-byte
// swizzle; the producers read it, meet at a barrier, and write the BF16 rows
// over it), or per-thread cp.async that lands each thread's points on the
// bytes of its own BF16 rows (strided lines and backward passes; every
// thread converts its own bytes, with no barrier).  Measured on 256^3
// passes: contiguous lines 0.17 ms by TMA against 0.20 ms per thread; strided
// lines 0.17 ms per thread against 0.21 ms by a 3-D TMA tile.
// BF16 planes (a pass of a chain): the head and tail rows as one TMA tile.
enum BLoad { kTmaContiguous = 0, kInPlace = 1, kTmaPlanes = 2 };

// FULL: every row block has BR rows (2N a multiple of 128).  GRAD: backward
// passes, whose input element is 2 grad * psi (the factors come through their
// own ring; two stages).  ACC: the batch's |.|^2 summed in shared memory.
// INBF: the input is BF16 planes (mode kTmaPlanes; never with GRAD).
template <bool FULL, bool GRAD, bool ACC, bool INBF>
__global__ void __launch_bounds__(BTHREADS, 1)
    dense_bf16_kernel(const DenseArgs a, const unsigned char* __restrict__ Tblk, int* err,
                      const __grid_constant__ CUtensorMap xmap, const int mode) {
  static_assert(!(GRAD && INBF), "backward passes take FP32 input");
  constexpr int BSTAGES = bstages(GRAD, ACC);
  extern __shared__ __align__(1024) unsigned char bsm_raw[];
  // the stages on a 1024-byte boundary (the launch adds 1 KB for it)
  unsigned char* const bsm = bsm_raw + ((1024u - (smem_u32(bsm_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t full_bar[BSMAX], empty_bar[BSMAX], copy_bar[BSMAX];
  __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int N = a.N;
  const int mtiles = (2 * N + BR - 1) / BR;
  const int kchunks = (2 * N) / BKC;
  const int64_t items = ((a.ncols + BL - 1) / BL) * mtiles;
  const int64_t my_items = (items - blockIdx.x + gridDim.x - 1) / gridDim.x;
  if (my_items <= 0) return;
  const int nb = ACC ? (int)a.batch : 1;
  const bool unsplit = a.unsplit != 0;

  if (warp == BMMA_WARP) tmem_alloc(&tmem_slot, BCOLS);
  if (tid == 0) {
    for (int s = 0; s < BSTAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), BPROD);
      mbar_init(smem_u32(&empty_bar[s]), 1);
      mbar_init(smem_u32(&copy_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf_bar[b]), 1);
      mbar_init(smem_u32(&acce_bar[b]), BEPI);
    }
    mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t smem_base = smem_u32(bsm);

  if (INBF && warp < BMMA_WARP) {
    // ---------------- loads of a BF16-plane input: thread 0 alone ----------------
    if (tid == 0) {
      const int64_t total = my_items * nb * kchunks;
      const uint64_t map_addr = reinterpret_cast<uint64_t>(&xmap);
      const uint32_t xbytes = unsplit ? (uint32_t)BPART : (uint32_t)BXAREA;
      int64_t iw = blockIdx.x, u = 0;
      int ib = 0, ikc = 0, is = 0;
      int last_u[BSMAX];
#pragma unroll
      for (int q = 0; q < BSMAX; ++q) last_u[q] = -1;
#pragma unroll 1
      for (int64_t ci = 0; ci < total; ++ci) {
        // chunk ci into stage is once the products of chunk ci - BSTAGES freed it
        if (u >= 1 && !mbar_wait(smem_u32(&empty_bar[is]), (uint32_t)((u - 1) & 1), &s_abort)) break;
        const int mt = (int)(iw % mtiles);
        const int64_t ct = iw / mtiles;
        const uint32_t st = smem_u32(bsm + is * BSTAGE);
        const uint32_t part = (uint32_t)(FULL ? BR : brow_count(N, mt)) * (BKC * 2);
        const uint32_t cb = smem_u32(&copy_bar[is]);
        mbar_expect_tx(cb, (unsplit ? part : 2 * part) + xbytes);
        const unsigned char* src = Tblk + ((size_t)mt * kchunks + ikc) * BTCHUNK;
        if (unsplit) {
          bulk_g2s(st, src, part, cb);
        } else if (part == (uint32_t)BPART) {
          bulk_g2s(st, src, BTCHUNK, cb);
        } else {
          bulk_g2s(st, src, part, cb);
          bulk_g2s(st + BPART, src + BPART, part, cb);
        }
        // rows: the tile's lines (realization ib's when accumulating); x: the
        // chunk's 64 real K; z: the head plane (and the tail plane)
        const int row = (int)(ct * BL + (ACC ? (int64_t)ib * a.outer : 0));
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(st + (uint32_t)BTCHUNK),
            "l"(map_addr), "r"(ikc * BKC), "r"(row), "r"(0), "r"(cb)
            : "memory");
        last_u[is] = (int)(u & 1);
        if (++is == BSTAGES) {
          is = 0;
          ++u;
        }
        if (++ikc == kchunks) {
          ikc = 0;
          if (++ib == nb) {
            ib = 0;
            iw += gridDim.x;
          }
        }
      }
      // nothing of this thread's may still be in flight at exit
      for (int q = 0; q < BSTAGES; ++q)
        if (last_u[q] >= 0) mbar_wait_own(smem_u32(&copy_bar[q]), (uint32_t)last_u[q], &s_abort);
    }
  } else if (warp < BMMA_WARP) {
    // ---------------- producers ----------------
    const int t = tid;
    const int64_t inner = a.inner;
    const bool contiguous = (inner == 1);
    const bool tma = mode == kTmaContiguous;
    const int64_t total = my_items * nb * kchunks;
    unsigned char* graw = bsm + BSTAGES * BSTAGE;  // gradient factors, one slot per stage (backward)
    // this thread's 4 core-matrix rows of a chunk: line n_i, K group kp_i
    // (contiguous: two lines, n_0 = n_1 and n_2 = n_3; strided: one), at byte
    // off_i of the stage's X head and X tail parts
    auto item_line = [&](int i) { return contiguous ? (t & 7) + 8 * (t >> 5) + 64 * (i >> 1) : (t & (BL - 1)); };
    auto item_kp = [&](int i) { return contiguous ? ((t >> 3) & 3) + 4 * (i & 1) : (t >> 7) * BITEMS + i; };
    auto item_off = [&](int i) {
      const int n = item_line(i);
      return (n >> 3) * BSBO + item_kp(i) * BCORE + (n & 7) * 16;
    };
    // Issue side, chunk j into stage j % BSTAGES once the products of chunk
    // j - BSTAGES have freed it: thread 0 copies the T chunk (and, with TMA,
    // the input tile), on the stage's "copy" barrier; in place, every thread
    // copies its points (item i's first two complex points onto its head row
    // X_hi + off_i, the next two onto its tail row X_lo + off_i).  The
    // chunk's position (item iw, realization ib, K chunk ikc) advances
    // incrementally; the lines' offsets are computed once per item and
    // realization.
    int64_t ci = 0, iw = blockIdx.x;
    int ib = 0, ikc = 0, is = 0;
    long long ilb[2] = {-1, -1};
    int ibr[2] = {0, 0};
    bool lines_ok = false;
    int last_u[BSMAX];
#pragma unroll
    for (int q = 0; q < BSMAX; ++q) last_u[q] = -1;
    const uint64_t map_addr = reinterpret_cast<uint64_t>(&xmap);
    auto issue = [&]() -> bool {
      if (ci < total) {
        const int64_t u = ci / BSTAGES;
        // the stage's previous products are done: with TMA thread 0 polls
        // (the next barrier passes the outcome on); in place every producer
        // polls for itself and moves on by itself (no barrier couples the
        // warps there: measured 20% faster than a barrier after thread 0's poll)
        if ((tma ? t == 0 : true) && u >= 1 &&
            !mbar_wait(smem_u32(&empty_bar[is]), (uint32_t)((u - 1) & 1), &s_abort))
          return false;
        unsigned char* st = bsm + is * BSTAGE;
        const int mt = (int)(iw % mtiles);
        const int64_t ct = iw / mtiles;
        const uint32_t xh = smem_u32(st + BTCHUNK), xl = xh + BPART;
        if (t == 0) {
          const uint32_t part = (uint32_t)(FULL ? BR : brow_count(N, mt)) * (BKC * 2);
          const uint32_t cb = smem_u32(&copy_bar[is]);
          mbar_expect_tx(cb, (unsplit ? part : 2 * part) + (tma ? (uint32_t)BXAREA : 0u));
          const unsigned char* src = Tblk + ((size_t)mt * kchunks + ikc) * BTCHUNK;
          const uint32_t dst = smem_u32(st);
          if (unsplit) {
            bulk_g2s(dst, src, part, cb);  // the head rows only
          } else if (part == (uint32_t)BPART) {
            bulk_g2s(dst, src, BTCHUNK, cb);  // head and tail in one copy
          } else {
            bulk_g2s(dst, src, part, cb);
            bulk_g2s(dst + BPART, src + BPART, part, cb);
          }
          if (tma) {
            // rows: the tile's lines (realization ib's when accumulating); x: the
            // chunk's 64 real K in two 32-float boxes
            const int row = (int)(ct * BL + (ACC ? (int64_t)ib * a.outer : 0));
#pragma unroll
            for (int h = 0; h < 2; ++h)
              asm volatile(
                  "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                  "[%4];" ::"r"(xh + (uint32_t)(h * BPART)),
                  "l"(map_addr), "r"(ikc * BKC + 32 * h), "r"(row), "r"(cb)
                  : "memory");
          }
          last_u[is] = (int)(u & 1);
        }
        if (!tma) {
          if (!lines_ok) {
            ilb[0] = bline(a, ct * BL + item_line(0), ib, ibr[0]);
            if (contiguous) ilb[1] = bline(a, ct * BL + item_line(2), ib, ibr[1]);
            lines_ok = true;
          }
          const uint32_t gdst0 = smem_u32(graw + is * BGRAD_CHUNK) + (uint32_t)t * 16;
#pragma unroll
          for (int i = 0; i < BITEMS; ++i) {
            const int li = contiguous ? (i >> 1) : 0;
            const long long lb = ilb[li];
            const bool valid = lb >= 0;
            const int k0 = ikc * (BKC / 2) + 4 * item_kp(i);  // first complex point
            const int64_t addr = valid ? lb + (int64_t)k0 * inner : 0;
            const uint32_t off = (uint32_t)item_off(i);
            // invalid lines read nothing and land as zeros (source size 0)
            if (contiguous) {
              cp_async16(xh + off, a.in + addr, valid ? 16 : 0);
              cp_async16(xl + off, a.in + addr + (valid ? 2 : 0), valid ? 16 : 0);
            } else {
              // point k0 + j of the line into half j % 2 of the head (j < 2) or
              // tail row; lanes 8-15 and 24-31 take the points in the order
              // 1, 0, 3, 2 so that each copy instruction's 8-byte pieces fall
              // on every bank twice (two wavefronts) instead of four times
#pragma unroll
              for (int j0 = 0; j0 < 4; ++j0) {
                const int j = j0 ^ ((t >> 3) & 1);
                cp_async8((j < 2 ? xh : xl) + off + (uint32_t)((j & 1) * 8), a.in + addr + (valid ? j * inner : 0),
                          valid ? 8 : 0);
              }
            }
            if (GRAD) {
              const int64_t gaddr = valid && a.grad_shared ? addr - (int64_t)ibr[li] * a.M : addr;
              const uint32_t gd = gdst0 + (uint32_t)(i * BPROD * 16);
#pragma unroll
              for (int j = 0; j < 4; ++j)
                cp_async4(gd + 4 * j, a.grad + gaddr + (valid ? j * inner : 0), valid ? 4 : 0);
            }
          }
          asm volatile("cp.async.commit_group;" ::: "memory");
        }
        ++ci;
        is = is + 1 == BSTAGES ? 0 : is + 1;
        if (++ikc == kchunks) {
          ikc = 0;
          lines_ok = false;
          if (++ib == nb) {
            ib = 0;
            iw += gridDim.x;
          }
        }
      } else if (!tma) {
        asm volatile("cp.async.commit_group;" ::: "memory");  // an empty group past the end keeps the count
      }
      return true;
    };
    bool ok = true;
#pragma unroll 1
    for (int r = 0; r < BSTAGES - 1; ++r) ok = issue() && ok;
#pragma unroll 1
    for (int64_t c = 0; c < total; ++c) {
      const int s = (int)(c % BSTAGES);
      unsigned char* xa = bsm + s * BSTAGE + BTCHUNK;
      const float4* gs = reinterpret_cast<const float4*>(graw + s * BGRAD_CHUNK) + t;
      float v[BITEMS][8];
      if (tma) {
        // the tile has landed: thread 0 polls the copy barrier, the barrier
        // passes the outcome and the data on
        if (t == 0) ok = ok && mbar_wait(smem_u32(&copy_bar[s]), (uint32_t)((c / BSTAGES) & 1), &s_abort);
        if (!prod_all(ok)) break;
#pragma unroll
        for (int i = 0; i < BITEMS; ++i) {
          // box kp / 4, row n, 16-byte chunks 2 (kp % 4) and + 1, swizzled by n % 8
          const int n = item_line(i), kp = item_kp(i);
          const unsigned char* row = xa + (kp >> 2) * BPART + n * 128;
          const int c0 = 2 * (kp & 3);
          const float4 r0 = *reinterpret_cast<const float4*>(row + ((c0 ^ (n & 7)) << 4));
          const float4 r1 = *reinterpret_cast<const float4*>(row + (((c0 + 1) ^ (n & 7)) << 4));
          v[i][0] = r0.x, v[i][1] = r0.y, v[i][2] = r0.z, v[i][3] = r0.w;
          v[i][4] = r1.x, v[i][5] = r1.y, v[i][6] = r1.z, v[i][7] = r1.w;
        }
        // every producer has read its input before any overwrites the tile with BF16 rows
        prod_sync();
      } else {
        // this thread's points of the chunk have landed (of its groups only the
        // BSTAGES - 2 newer ones may be pending); it alone touches their bytes
        asm volatile("cp.async.wait_group %0;" ::"n"(BSTAGES - 2) : "memory");
        if (!ok) break;
#pragma unroll
        for (int i = 0; i < BITEMS; ++i) {
          const int off = item_off(i);
          const float4 r0 = *reinterpret_cast<const float4*>(xa + off);
          const float4 r1 = *reinterpret_cast<const float4*>(xa + BPART + off);
          v[i][0] = r0.x, v[i][1] = r0.y, v[i][2] = r0.z, v[i][3] = r0.w;
          v[i][4] = r1.x, v[i][5] = r1.y, v[i][6] = r1.z, v[i][7] = r1.w;
        }
      }
#pragma unroll
      for (int i = 0; i < BITEMS; ++i) {
        if (GRAD) {
          // the input element is 2 grad * psi
          const float4 g = gs[i * BPROD];
          const float g4[4] = {2.f * g.x, 2.f * g.y, 2.f * g.z, 2.f * g.w};
#pragma unroll
          for (int m = 0; m < 8; ++m) v[i][m] *= g4[m >> 1];
        }
        uint4 hi, lo;
        split8(v[i], hi, lo, unsplit);
        const int off = item_off(i);
        *reinterpret_cast<uint4*>(xa + off) = hi;
        if (!unsplit) *reinterpret_cast<uint4*>(xa + BPART + off) = lo;
      }
      fence_async_smem();
      mbar_arrive(smem_u32(&full_bar[s]));
      // the copies of chunk c + BSTAGES - 1, into the stage chunk c - 1 used
      ok = issue() && ok;
    }
    // nothing of this thread's may still be in flight at exit
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (t == 0)
      for (int q = 0; q < BSTAGES; ++q)
        if (last_u[q] >= 0) mbar_wait_own(smem_u32(&copy_bar[q]), (uint32_t)last_u[q], &s_abort);
  } else if (warp == BMMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int64_t g = 0, sub = 0;
      bool ok = true;
      for (int64_t it = 0; ok && it < my_items; ++it) {
        const int mt = (int)((blockIdx.x + it * gridDim.x) % mtiles);
        const uint32_t idesc = idesc_bf16(BL, FULL ? BR : brow_count(N, mt));
        // whole row blocks: X_hi against [T_hi; T_lo] (the T chunk's 256 rows,
        // head rows then tail rows) in one N = 256 product into the adjacent
        // accumulators [d1 | d2] -- the operand X_hi is read once for both
        for (int b = 0; ok && b < nb; ++b, ++sub) {
          const int buf = (int)(sub & 1);
          const int64_t v = sub >> 1;
          if (v >= 1 && !mbar_wait(smem_u32(&acce_bar[buf]), (uint32_t)((v - 1) & 1), &s_abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d1 = tmem + (uint32_t)(buf * 2 * BR), d2 = d1 + BR;
          for (int kc = 0; kc < kchunks; ++kc, ++g) {
            const int s = (int)(g % BSTAGES);
            const int64_t u = g / BSTAGES;
            if (!mbar_wait(smem_u32(&copy_bar[s]), (uint32_t)(u & 1), &s_abort) ||
                (!INBF && !mbar_wait(smem_u32(&full_bar[s]), (uint32_t)(u & 1), &s_abort))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t th = smem_base + (uint32_t)(s * BSTAGE), tl = th + BPART;
            const uint32_t xh = th + BTCHUNK, xl = xh + BPART;
#pragma unroll
            for (int ks = 0; ks < BKC / 16; ++ks) {
              const uint32_t o = (uint32_t)(ks * 2 * BCORE);
              // X: core matrices of the producers, or the swizzled TMA tile (32 bytes per K step)
              const uint64_t dxh = INBF ? make_desc_sw128(xh + (uint32_t)(ks * 32)) : make_desc(xh + o, BCORE, BSBO);
              const uint64_t dth = make_desc(th + o, BCORE, BSBO);
              const uint32_t more = (kc == 0 && ks == 0) ? 0u : 1u;
              if (unsplit) {
                mma_f16(d1, dxh, dth, idesc, more);
              } else {
                const uint64_t dxl =
                    INBF ? make_desc_sw128(xl + (uint32_t)(ks * 32)) : make_desc(xl + o, BCORE, BSBO);
                if (FULL) {
                  mma_f16(d1, dxh, dth, idesc_bf16(BL, 2 * BR), more);
                } else {
                  mma_f16(d1, dxh, dth, idesc, more);
                  mma_f16(d2, dxh, make_desc(tl + o, BCORE, BSBO), idesc, more);
                }
                mma_f16(d2, dxl, dth, idesc, 1u);
              }
            }
            mma_commit(smem_u32(&empty_bar[s]));
          }
          if (ok) mma_commit(smem_u32(&accf_bar[buf]));
        }
      }
      // whatever happened, the tensor cores finish this thread's work before exit
      mma_commit(smem_u32(&done_bar));
      mbar_wait_own(smem_u32(&done_bar), 0u, &s_abort);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    const int q = warp & 3;       // tensor-memory lane quarter this warp may read
    const int r = q * 32 + lane;  // line within the item
    const int64_t inner = a.oinner;  // the output's decomposition
    const bool contiguous = (inner == 1);
    float* racc = reinterpret_cast<float*>(bsm + BSTAGES * BSTAGE);  // accumulating launches only
    if (ACC)
      for (int m = 0; m < BR / 2; ++m) racc[m * BL + r] = 0.f;
    int64_t sub = 0;
    bool ok = true;
    for (int64_t it = 0; ok && it < my_items; ++it) {
      const int64_t w = blockIdx.x + it * gridDim.x;
      const int64_t ct = w / mtiles;
      const int mt = (int)(w % mtiles);
      const int nbase = mt * (BR / 2);
      const int rows = FULL ? BR : brow_count(N, mt);
      for (int b = 0; b < nb; ++b, ++sub) {
        const int buf = (int)(sub & 1);
        const int64_t v = sub >> 1;
        // lane 0 polls; the outcome is the warp's (its tensor-memory loads need the whole warp)
        bool got = true;
        if (lane == 0) got = mbar_wait(smem_u32(&accf_bar[buf]), (uint32_t)(v & 1), &s_abort);
        ok = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
        if (!ok) break;
        tc_fence_after();
        int br;
        const long long base = bline_o(a, ct * BL + r, b, br);
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 2 * BR);
#pragma unroll 1
        for (int j0 = 0; j0 < rows; j0 += 16) {
          uint32_t x[16], z[16];
          tmem_ld16(taddr + (uint32_t)j0, x);
          if (!unsplit) tmem_ld16(taddr + (uint32_t)(BR + j0), z);
          tmem_wait_ld();
          float y[16];
#pragma unroll
          for (int m = 0; m < 16; ++m) y[m] = __uint_as_float(x[m]) + (unsplit ? 0.f : __uint_as_float(z[m]));
          const int n0 = nbase + j0 / 2;  // complex outputs n0 .. n0 + 7 of this line
          if (ACC) {
#pragma unroll
            for (int m = 0; m < 8; ++m)
              racc[(j0 / 2 + m) * BL + r] += y[2 * m] * y[2 * m] + y[2 * m + 1] * y[2 * m + 1];
          } else if (base >= 0) {
            if (a.out_bf) {
              // BF16 head and tail planes for the next pass of a chain
#pragma unroll
              for (int m = 0; m < 8; ++m) {
                const __nv_bfloat162 hb = __floats2bfloat162_rn(y[2 * m], y[2 * m + 1]);
                const int64_t e = base + (int64_t)(n0 + m) * inner;
                a.out_bf[e] = *reinterpret_cast<const uint32_t*>(&hb);
                if (!unsplit) {
                  const float2 hf = __bfloat1622float2(hb);
                  a.out_bf[a.bf_plane + e] = pack_bf16(y[2 * m] - hf.x, y[2 * m + 1] - hf.y);
                }
              }
            } else if (a.out_c) {
              if (contiguous) {
                float4* o = reinterpret_cast<float4*>(a.out_c + base + n0);
#pragma unroll
                for (int m = 0; m < 4; ++m) o[m] = make_float4(y[4 * m], y[4 * m + 1], y[4 * m + 2], y[4 * m + 3]);
              } else {
#pragma unroll
                for (int m = 0; m < 8; ++m) a.out_c[base + (int64_t)(n0 + m) * inner] = make_float2(y[2 * m], y[2 * m + 1]);
              }
            } else {
              float dd[8];
#pragma unroll
              for (int m = 0; m < 8; ++m) dd[m] = y[2 * m] * y[2 * m] + y[2 * m + 1] * y[2 * m + 1];
              if (contiguous) {
                float4* o = reinterpret_cast<float4*>(a.out_d + base + n0);
                o[0] = make_float4(dd[0], dd[1], dd[2], dd[3]);
                o[1] = make_float4(dd[4], dd[5], dd[6], dd[7]);
              } else {
#pragma unroll
                for (int m = 0; m < 8; ++m) a.out_d[base + (int64_t)(n0 + m) * inner] = dd[m];
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(smem_u32(&acce_bar[buf]));
        if (ACC && b == nb - 1) {
          if (base >= 0) {
            const int64_t o0 = base - (int64_t)br * a.M + (int64_t)nbase * inner;
            if (contiguous) {
              float4* o = reinterpret_cast<float4*>(a.out_d + o0);
#pragma unroll 1
              for (int m = 0; m < rows / 8; ++m) {
                float4 cur = o[m];
                cur.x += racc[(4 * m) * BL + r];
                cur.y += racc[(4 * m + 1) * BL + r];
                cur.z += racc[(4 * m + 2) * BL + r];
                cur.w += racc[(4 * m + 3) * BL + r];
                o[m] = cur;
              }
            } else {
#pragma unroll 1
              for (int m = 0; m < rows / 2; ++m) a.out_d[o0 + (int64_t)m * inner] += racc[m * BL + r];
            }
          }
          for (int m = 0; m < BR / 2; ++m) racc[m * BL + r] = 0.f;
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (tid == 0 && s_abort && err) atomicAdd(err, 1);
  if (warp == BMMA_WARP) {
    tc_fence_after();
    tmem_free(tmem, BCOLS);
  }
}

// Pre-split BF16 T chunks from the complex map T [N][N]: for row block mt and
// K chunk kc, a 32 KB block [head: 128 rows x 64 K][tail] in core-matrix
// order; real (r, k') with r = 2n + p_out, k' = 2k + p_in holds the 2 x 2
// block entry of T[n][k]; rows and K columns past 2N are zero (a last K
// chunk of 2N = 32 mod 64 is half zeros).
__global__ void bf16_build_t_kernel(const float2* __restrict__ T, unsigned char* __restrict__ Tblk, int N) {
  const int R = 2 * N;
  const int RP = (R + BR - 1) / BR * BR;
  const int kchunks = (R + BKC - 1) / BKC;
  const int KP = kchunks * BKC;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)RP * KP;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / KP), kp = (int)(idx - (int64_t)r * KP);
    const int n = r >> 1, po = r & 1, k = kp >> 1, pi = kp & 1;
    float v = 0.f;
    if (r < R && kp < R) {
      const float2 t = T[(int64_t)n * N + k];
      v = po == 0 ? (pi == 0 ? t.x : -t.y) : (pi == 0 ? t.y : t.x);
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    const int mt = r / BR, rr = r % BR, kc = kp / BKC, kk = kp % BKC;
    unsigned char* blk = Tblk + ((size_t)mt * kchunks + kc) * BTCHUNK;
    const int off = (rr >> 3) * BSBO + (kk >> 3) * BCORE + (rr & 7) * 16 + (kk & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(blk + off) = hi;
    *reinterpret_cast<__nv_bfloat16*>(blk + BPART + off) = lo;
  }
}

// The first pass of a BF16 chain reads its FP32 input as BF16 planes too:
// every (re, im) pair v becomes bf16(v) in the head plane and bf16(v - bf16(v))
// in the tail plane (the split the pass would make on the fly), in the same
// order; two pairs per thread step, 16-byte loads.
__global__ void __launch_bounds__(256) bf16_split_kernel(const float4* __restrict__ in, uint2* __restrict__ hi,
                                                          uint2* __restrict__ lo, int64_t n2, int unsplit) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = in[i];
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
    hi[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
    if (!unsplit) {
      const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
      lo[i] = make_uint2(pack_bf16(v.x - f0.x, v.y - f0.y), pack_bf16(v.z - f1.x, v.w - f1.y));
    }
  }
}

// ---------------------------------------------------------------------------
// Many-instance phases (ffx_plan_many): one launch runs the work list of a
// phase, items of 128 lines x 128 real rows of the passes of many instances,
// each pass with its own N, line geometry, buffers and T blocks; block b takes
// items [block_first[b], block_first[b + 1]).  The roles, stages, barriers and
// bounded waits are those of dense_bf16_kernel; three stages, split operands,
// no batch sum and no gradient factors.  The FP32 input of an item reaches the
// stage as a TMA tile where its pass has a tile map (contiguous lines in the
// plan's own workspaces, maps made at plan time), else by per-thread copies in
// place (the caller's input, strided lines).  Row blocks of 128 rows take
// X_hi [T_hi; T_lo] as one N = 256 product, the last (shorter) row block of an
// axis two products.

// What a role needs of one work item.
struct BView {
  const float2* in;
  float2* out_c;
  float* out_d;
  const unsigned char* tblk;
  const void* xmap;  // the input's tile map, or NULL
  uint32_t* out_bf;  // BF16 planes out (chains), or NULL
  int64_t inner, ncols, ct, bf_plane;
  int N, mt;
};

__device__ __forceinline__ const void* many_rebase(const TcBases& c, int base, const void* off) {
  return base < 0 ? nullptr : (const void*)((const char*)c.base[base] + (uintptr_t)off);
}

__device__ __forceinline__ BView many_view(const TcParams& P, int64_t w) {
  const TcItem item = P.items[w];
  const TcPassArg& pa = P.args[item.arg];
  BView v;
  v.in = (const float2*)many_rebase(P.call, pa.in_base, pa.d.in);
  v.out_c = (float2*)many_rebase(P.call, pa.outc_base, pa.d.out_c);
  v.out_d = (float*)many_rebase(P.call, pa.outd_base, pa.d.out_d);
  v.tblk = pa.tblk;
  v.xmap = pa.xmap >= 0 ? (const void*)((const unsigned char*)P.xmaps + (size_t)pa.xmap * 128) : nullptr;
  v.out_bf = pa.out_planes ? (uint32_t*)many_rebase(P.call, pa.outc_base, pa.d.out_bf) : nullptr;
  if (pa.out_planes) v.out_c = nullptr;
  v.bf_plane = pa.d.bf_plane;
  v.inner = pa.d.inner;
  v.ncols = pa.d.ncols;
  v.N = pa.d.N;
  v.ct = item.ct;
  v.mt = item.mt;
  return v;
}

// First point of line c of an item's pass (a batch of one), or -1 past the end.
__device__ __forceinline__ long long many_line(const BView& v, int64_t c) {
  if (c >= v.ncols) return -1;
  const int64_t bo = c / v.inner;
  return bo * (int64_t)v.N * v.inner + (c - bo * v.inner);
}

// Producer thread t's 4 core-matrix rows of a chunk, as in dense_bf16_kernel:
// row i is line prod_line of the item and K group prod_kp, at byte prod_off of
// the stage's X head and X tail parts.
__device__ __forceinline__ int prod_line(bool contiguous, int t, int i) {
  return contiguous ? (t & 7) + 8 * (t >> 5) + 64 * (i >> 1) : (t & (BL - 1));
}
__device__ __forceinline__ int prod_kp(bool contiguous, int t, int i) {
  return contiguous ? ((t >> 3) & 3) + 4 * (i & 1) : (t >> 7) * BITEMS + i;
}
__device__ __forceinline__ int prod_off(bool contiguous, int t, int i) {
  const int n = prod_line(contiguous, t, i);
  return (n >> 3) * BSBO + prod_kp(contiguous, t, i) * BCORE + (n & 7) * 16;
}

constexpr int BMANY_STAGES = 3;
// the stages, and 1 KB to start them on a 1024-byte boundary (the swizzled
// tiles' atoms)
constexpr int BMANY_SMEM = BMANY_STAGES * BSTAGE + 1024;
// XM, the input mode of every pass of the launch (one mode per launch: a
// barrier of the producers that some warps skip would never open):
//  * kInPlace: FP32 input by per-thread copies, each producer polling for
//    itself and the warps moving on independently;
//  * kTmaContiguous: FP32 contiguous lines by TMA tiles (a tile map per
//    pass), thread 0 polling and a producer barrier passing the outcome on;
//  * kTmaPlanes (BF16 chains): BF16 head and tail planes of contiguous lines
//    by one 3-D TMA tile per chunk straight into the tensor cores' swizzled
//    K-major layout (thread 0 alone; no conversion), output transposed
//    (point n of line c at c + n lines) as the next pass's planes or, after
//    the last pass, in the lattice's own order.
// TOUT: the output transposed so, also for FP32 input (a chain's first pass
// reading the caller's input).
template <int XM, bool TOUT>
__global__ void __launch_bounds__(BTHREADS, 1) dense_bf16_many_kernel(const TcParams P) {
  constexpr int BSTAGES = BMANY_STAGES;
  constexpr bool TMA = XM == kTmaContiguous;
  constexpr bool PLANES = XM == kTmaPlanes;
  static_assert(TOUT || !PLANES, "plane input comes with transposed output");
  extern __shared__ __align__(1024) unsigned char bsm_raw[];
  unsigned char* const bsm = bsm_raw + ((1024u - (smem_u32(bsm_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t full_bar[BSTAGES], empty_bar[BSTAGES], copy_bar[BSTAGES];
  __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int64_t first = P.block_first[blockIdx.x], last = P.block_first[blockIdx.x + 1];
  if (first >= last) return;

  if (warp == BMMA_WARP) tmem_alloc(&tmem_slot, BCOLS);
  if (tid == 0) {
    for (int s = 0; s < BSTAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), BPROD);
      mbar_init(smem_u32(&empty_bar[s]), 1);
      mbar_init(smem_u32(&copy_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf_bar[b]), 1);
      mbar_init(smem_u32(&acce_bar[b]), BEPI);
    }
    mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t smem_base = smem_u32(bsm);

  if (PLANES && warp < BMMA_WARP) {
    // ---------------- loads of BF16 planes: thread 0 alone ----------------
    if (tid == 0) {
      int64_t iw = first, ci = 0;
      int ikc = 0, is = 0;
      BView iv = many_view(P, first);
      int ikch = (2 * iv.N + BKC - 1) / BKC;
      int last_u[BSTAGES];
#pragma unroll
      for (int q = 0; q < BSTAGES; ++q) last_u[q] = -1;
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(iv.xmap) : "memory");
#pragma unroll 1
      while (iw < last) {
        // chunk ci into stage is once the products of chunk ci - BSTAGES freed it
        const int64_t u = ci / BSTAGES;
        if (u >= 1 && !mbar_wait(smem_u32(&empty_bar[is]), (uint32_t)((u - 1) & 1), &s_abort)) break;
        const uint32_t st = smem_u32(bsm + is * BSTAGE);
        const uint32_t part = (uint32_t)brow_count(iv.N, iv.mt) * (BKC * 2);
        const uint32_t cb = smem_u32(&copy_bar[is]);
        mbar_expect_tx(cb, 2 * part + (uint32_t)BXAREA);
        const unsigned char* src = iv.tblk + ((size_t)iv.mt * ikch + ikc) * BTCHUNK;
        if (part == (uint32_t)BPART) {
          bulk_g2s(st, src, BTCHUNK, cb);
        } else {
          bulk_g2s(st, src, part, cb);
          bulk_g2s(st + BPART, src + BPART, part, cb);
        }
        // x: the chunk's 64 real K (past 2N: zeros); rows: the tile's lines
        // (past the pass's end: zeros); z: the head and tail planes
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4}], [%5];" ::"r"(st + (uint32_t)BTCHUNK),
            "l"(reinterpret_cast<uint64_t>(iv.xmap)), "r"(ikc * BKC), "r"((int)(iv.ct * BL)), "r"(0), "r"(cb)
            : "memory");
        last_u[is] = (int)(u & 1);
        ++ci;
        is = is + 1 == BSTAGES ? 0 : is + 1;
        if (++ikc == ikch) {
          ikc = 0;
          if (++iw < last) {
            const void* prev = iv.xmap;
            iv = many_view(P, iw);
            ikch = (2 * iv.N + BKC - 1) / BKC;
            if (iv.xmap != prev)
              asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(iv.xmap) : "memory");
          }
        }
      }
      // nothing of this thread's may still be in flight at exit
      for (int q = 0; q < BSTAGES; ++q)
        if (last_u[q] >= 0) mbar_wait_own(smem_u32(&copy_bar[q]), (uint32_t)last_u[q], &s_abort);
    }
  } else if (warp < BMMA_WARP) {
    // ---------------- producers ----------------
    const int t = tid;
    // Issue side: chunk j of the block's run into stage j % BSTAGES once the
    // products of chunk j - BSTAGES have freed it; thread 0 copies the T chunk
    // (and, where the pass has a tile map, the input tile: two 128 x 32-float
    // boxes, 128-byte swizzle) on the stage's "copy" barrier, else every
    // thread its points of the input.  The chunk's position (item iw, K chunk
    // ikc) advances incrementally.
    int64_t iw = first, ci = 0;
    int ikc = 0, is = 0;
    BView iv = many_view(P, first);
    int ikch = (2 * iv.N + BKC - 1) / BKC;
    long long ilb[2] = {-1, -1};
    bool lines_ok = false;
    int last_u[BSTAGES];
#pragma unroll
    for (int q = 0; q < BSTAGES; ++q) last_u[q] = -1;
    auto issue = [&]() -> bool {
      if (iw < last) {
        const int64_t u = ci / BSTAGES;
        if (u >= 1 && !mbar_wait(smem_u32(&empty_bar[is]), (uint32_t)((u - 1) & 1), &s_abort)) return false;
        unsigned char* st = bsm + is * BSTAGE;
        const uint32_t xh = smem_u32(st + BTCHUNK), xl = xh + BPART;
        const bool tma = TMA;
        if (t == 0) {
          const uint32_t part = (uint32_t)brow_count(iv.N, iv.mt) * (BKC * 2);
          const uint32_t cb = smem_u32(&copy_bar[is]);
          mbar_expect_tx(cb, 2 * part + (tma ? (uint32_t)BXAREA : 0u));
          const unsigned char* src = iv.tblk + ((size_t)iv.mt * ikch + ikc) * BTCHUNK;
          const uint32_t dst = smem_u32(st);
          if (part == (uint32_t)BPART) {
            bulk_g2s(dst, src, BTCHUNK, cb);  // head and tail in one copy
          } else {
            bulk_g2s(dst, src, part, cb);
            bulk_g2s(dst + BPART, src + BPART, part, cb);
          }
          if (tma) {
            // rows: the tile's lines (past the pass's end: zeros); x: the
            // chunk's 64 real K (past 2N: zeros) in two 32-float boxes
            const uint64_t map_addr = reinterpret_cast<uint64_t>(iv.xmap);
            const int row = (int)(iv.ct * BL);
#pragma unroll
            for (int h = 0; h < 2; ++h)
              asm volatile(
                  "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                  "%3}], [%4];" ::"r"(xh + (uint32_t)(h * BPART)),
                  "l"(map_addr), "r"(ikc * BKC + 32 * h), "r"(row), "r"(cb)
                  : "memory");
          }
          last_u[is] = (int)(u & 1);
        }
        const int64_t inner = iv.inner;
        const bool contiguous = (inner == 1);
        if (tma) {
          // nothing for the other threads to copy (an empty group keeps the count)
        } else if (!lines_ok) {
          ilb[0] = many_line(iv, iv.ct * BL + prod_line(contiguous, t, 0));
          if (contiguous) ilb[1] = many_line(iv, iv.ct * BL + prod_line(contiguous, t, 2));
          lines_ok = true;
        }
        // lines past the pass's end, and K past 2N in the last chunk of a
        // 2N = 32 mod 64 axis, read nothing and land as zeros (source size 0)
        if (tma) {
        } else if (contiguous) {
          // lanes t and t ^ 8 hold the rows (line, kp) and (line, kp + 1) of
          // a row pair, 8 complex points: the even lane copies points 0-1 and
          // 4-5 (the head rows), the odd lane 2-3 and 6-7 (the tail rows), so
          // that each copy instruction requests whole 32-byte sectors; a row's
          // two halves then come from both lanes (a warp barrier before the
          // conversion)
          const int e = (t >> 3) & 1;
          const uint32_t dst = e ? xl : xh;
#pragma unroll
          for (int i = 0; i < BITEMS; ++i) {
            const long long lb = ilb[i >> 1];
            const int kpe = prod_kp(true, t, i) & ~1;
            const int k0 = ikc * (BKC / 2) + 4 * kpe;  // first complex point of the row pair
            const bool valid = lb >= 0 && k0 < iv.N;
            const int64_t addr = valid ? lb + k0 + 2 * e : 0;
            const uint32_t off = (uint32_t)(prod_off(true, t, i) - ((t >> 3) & 1) * BCORE);  // the even row
            cp_async16(dst + off, iv.in + addr, valid ? 16 : 0);
            cp_async16(dst + off + BCORE, iv.in + addr + (valid ? 4 : 0), valid ? 16 : 0);
          }
        } else {
#pragma unroll
          for (int i = 0; i < BITEMS; ++i) {
            const long long lb = ilb[0];
            const int k0 = ikc * (BKC / 2) + 4 * prod_kp(false, t, i);  // first complex point
            const bool valid = lb >= 0 && k0 < iv.N;
            const int64_t addr = valid ? lb + (int64_t)k0 * inner : 0;
            const uint32_t off = (uint32_t)prod_off(false, t, i);
            // the point order of dense_bf16_kernel's strided copies (two
            // wavefronts per instruction)
#pragma unroll
            for (int j0 = 0; j0 < 4; ++j0) {
              const int j = j0 ^ ((t >> 3) & 1);
              cp_async8((j < 2 ? xh : xl) + off + (uint32_t)((j & 1) * 8), iv.in + addr + (valid ? j * inner : 0),
                        valid ? 8 : 0);
            }
          }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        ++ci;
        is = is + 1 == BSTAGES ? 0 : is + 1;
        if (++ikc == ikch) {
          ikc = 0;
          lines_ok = false;
          if (++iw < last) {
            const void* prev = iv.xmap;
            iv = many_view(P, iw);
            ikch = (2 * iv.N + BKC - 1) / BKC;
            // a map written before the launch, read by the tensor copies
            if (TMA && t == 0 && iv.xmap != prev)
              asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(iv.xmap) : "memory");
          }
        }
      } else {
        asm volatile("cp.async.commit_group;" ::: "memory");  // an empty group past the end keeps the count
      }
      return true;
    };
    if (TMA && t == 0) asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(iv.xmap) : "memory");
    bool ok = true;
#pragma unroll 1
    for (int r = 0; r < BSTAGES - 1; ++r) ok = issue() && ok;
    // Conversion side: its own position (item cw, K chunk ckc), BSTAGES - 1
    // chunks behind the issue side.
    int64_t cw = first;
    int ckc = 0;
    int cN = P.args[P.items[first].arg].d.N;
    bool ccontig = P.args[P.items[first].arg].d.inner == 1;
#pragma unroll 1
    for (int64_t c = 0; cw < last; ++c) {
      const int s = (int)(c % BSTAGES);
      unsigned char* xa = bsm + s * BSTAGE + BTCHUNK;
      if (TMA) {
        // the tile has landed: thread 0 polls the copy barrier, the barrier
        // passes the outcome and the data on
        if (t == 0) ok = ok && mbar_wait(smem_u32(&copy_bar[s]), (uint32_t)((c / BSTAGES) & 1), &s_abort);
        if (!prod_all(ok)) break;
      } else {
        // this thread's points of the chunk have landed (of its groups only
        // the BSTAGES - 2 newer ones may be pending); the warp stops as one
        // and sees the partner lane's halves of this thread's rows
        asm volatile("cp.async.wait_group %0;" ::"n"(BSTAGES - 2) : "memory");
        if (!__all_sync(0xffffffffu, ok)) break;
        if (ccontig) __syncwarp();
      }
      float v[BITEMS][8];
#pragma unroll
      for (int i = 0; i < BITEMS; ++i) {
        if (TMA) {
          // box kp / 4, row n, 16-byte chunks 2 (kp % 4) and + 1, swizzled by n % 8
          const int n = prod_line(true, t, i), kp = prod_kp(true, t, i);
          const unsigned char* row = xa + (kp >> 2) * BPART + n * 128;
          const int c0 = 2 * (kp & 3);
          const float4 r0 = *reinterpret_cast<const float4*>(row + ((c0 ^ (n & 7)) << 4));
          const float4 r1 = *reinterpret_cast<const float4*>(row + (((c0 + 1) ^ (n & 7)) << 4));
          v[i][0] = r0.x, v[i][1] = r0.y, v[i][2] = r0.z, v[i][3] = r0.w;
          v[i][4] = r1.x, v[i][5] = r1.y, v[i][6] = r1.z, v[i][7] = r1.w;
        } else {
          const int off = prod_off(ccontig, t, i);
          const float4 r0 = *reinterpret_cast<const float4*>(xa + off);
          const float4 r1 = *reinterpret_cast<const float4*>(xa + BPART + off);
          v[i][0] = r0.x, v[i][1] = r0.y, v[i][2] = r0.z, v[i][3] = r0.w;
          v[i][4] = r1.x, v[i][5] = r1.y, v[i][6] = r1.z, v[i][7] = r1.w;
        }
      }
      // every producer has read its input before any overwrites the tile with BF16 rows
      if (TMA) prod_sync();
#pragma unroll
      for (int i = 0; i < BITEMS; ++i) {
        const int off = prod_off(ccontig, t, i);
        uint4 hi, lo;
        split8(v[i], hi, lo, false);
        *reinterpret_cast<uint4*>(xa + off) = hi;
        *reinterpret_cast<uint4*>(xa + BPART + off) = lo;
      }
      fence_async_smem();
      mbar_arrive(smem_u32(&full_bar[s]));
      // the copies of chunk c + BSTAGES - 1, into the stage chunk c - 1 used
      ok = issue() && ok;
      if (++ckc == (2 * cN + BKC - 1) / BKC) {
        ckc = 0;
        if (++cw < last) {
          const TcPassArg& pa = P.args[P.items[cw].arg];
          cN = pa.d.N;
          ccontig = pa.d.inner == 1;
        }
      }
    }
    // nothing of this thread's may still be in flight at exit
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (t == 0)
      for (int q = 0; q < BSTAGES; ++q)
        if (last_u[q] >= 0) mbar_wait_own(smem_u32(&copy_bar[q]), (uint32_t)last_u[q], &s_abort);
  } else if (warp == BMMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int64_t g = 0, sub = 0;
      bool ok = true;
      for (int64_t w = first; ok && w < last; ++w, ++sub) {
        const TcItem item = P.items[w];
        const int N = P.args[item.arg].d.N;
        const int rows = brow_count(N, item.mt);
        const int kchunks = (2 * N + BKC - 1) / BKC;
        const uint32_t idesc = idesc_bf16(BL, rows);
        const bool whole = rows == BR;
        const int buf = (int)(sub & 1);
        const int64_t v = sub >> 1;
        if (v >= 1 && !mbar_wait(smem_u32(&acce_bar[buf]), (uint32_t)((v - 1) & 1), &s_abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d1 = tmem + (uint32_t)(buf * 2 * BR), d2 = d1 + BR;
        for (int kc = 0; kc < kchunks; ++kc, ++g) {
          const int s = (int)(g % BSTAGES);
          const int64_t u = g / BSTAGES;
          if (!mbar_wait(smem_u32(&copy_bar[s]), (uint32_t)(u & 1), &s_abort) ||
              (!PLANES && !mbar_wait(smem_u32(&full_bar[s]), (uint32_t)(u & 1), &s_abort))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t th = smem_base + (uint32_t)(s * BSTAGE), tl = th + BPART;
          const uint32_t xh = th + BTCHUNK, xl = xh + BPART;
#pragma unroll
          for (int ks = 0; ks < BKC / 16; ++ks) {
            const uint32_t o = (uint32_t)(ks * 2 * BCORE);
            // X: the producers' core matrices, or the swizzled TMA tile (32 bytes per K step)
            const uint64_t dxh = PLANES ? make_desc_sw128(xh + (uint32_t)(ks * 32)) : make_desc(xh + o, BCORE, BSBO);
            const uint64_t dxl = PLANES ? make_desc_sw128(xl + (uint32_t)(ks * 32)) : make_desc(xl + o, BCORE, BSBO);
            const uint64_t dth = make_desc(th + o, BCORE, BSBO);
            const uint32_t more = (kc == 0 && ks == 0) ? 0u : 1u;
            if (whole) {
              // the T chunk's 256 rows (head rows, then tail rows) into [d1 | d2]
              mma_f16(d1, dxh, dth, idesc_bf16(BL, 2 * BR), more);
            } else {
              mma_f16(d1, dxh, dth, idesc, more);
              mma_f16(d2, dxh, make_desc(tl + o, BCORE, BSBO), idesc, more);
            }
            mma_f16(d2, dxl, dth, idesc, 1u);
          }
          mma_commit(smem_u32(&empty_bar[s]));
        }
        if (ok) mma_commit(smem_u32(&accf_bar[buf]));
      }
      // whatever happened, the tensor cores finish this thread's work before exit
      mma_commit(smem_u32(&done_bar));
      mbar_wait_own(smem_u32(&done_bar), 0u, &s_abort);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    const int q = warp & 3;       // tensor-memory lane quarter this warp may read
    const int r = q * 32 + lane;  // line within the item
    int64_t sub = 0;
    bool ok = true;
    for (int64_t w = first; ok && w < last; ++w, ++sub) {
      const BView ev = many_view(P, w);
      // the output's stride between a line's points: the input's, or (chains)
      // the transposed order's, the pass's line count
      const int64_t inner = TOUT ? ev.ncols : ev.inner;
      const bool contiguous = !TOUT && inner == 1;
      const int nbase = ev.mt * (BR / 2);
      const int rows = brow_count(ev.N, ev.mt);
      const int buf = (int)(sub & 1);
      const int64_t v = sub >> 1;
      // lane 0 polls; the outcome is the warp's (its tensor-memory loads need the whole warp)
      bool got = true;
      if (lane == 0) got = mbar_wait(smem_u32(&accf_bar[buf]), (uint32_t)(v & 1), &s_abort);
      ok = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
      if (!ok) break;
      tc_fence_after();
      const int64_t line = ev.ct * BL + r;
      const long long base = TOUT ? (line < ev.ncols ? line : -1) : many_line(ev, line);
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 2 * BR);
#pragma unroll 1
      for (int j0 = 0; j0 < rows; j0 += 16) {
        uint32_t x[16], z[16];
        tmem_ld16(taddr + (uint32_t)j0, x);
        tmem_ld16(taddr + (uint32_t)(BR + j0), z);
        tmem_wait_ld();
        float y[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) y[m] = __uint_as_float(x[m]) + __uint_as_float(z[m]);
        const int n0 = nbase + j0 / 2;  // complex outputs n0 .. n0 + 7 of this line
        if (base < 0) continue;
        if (TOUT && ev.out_bf) {
          // BF16 head and tail planes for the next pass (the split that pass
          // would make of the same FP32 value)
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const __nv_bfloat162 hb = __floats2bfloat162_rn(y[2 * m], y[2 * m + 1]);
            const int64_t e = base + (int64_t)(n0 + m) * inner;
            ev.out_bf[e] = *reinterpret_cast<const uint32_t*>(&hb);
            const float2 hf = __bfloat1622float2(hb);
            ev.out_bf[ev.bf_plane + e] = pack_bf16(y[2 * m] - hf.x, y[2 * m + 1] - hf.y);
          }
        } else if (ev.out_c) {
          if (contiguous) {
            float4* o = reinterpret_cast<float4*>(ev.out_c + base + n0);
#pragma unroll
            for (int m = 0; m < 4; ++m) o[m] = make_float4(y[4 * m], y[4 * m + 1], y[4 * m + 2], y[4 * m + 3]);
          } else {
#pragma unroll
            for (int m = 0; m < 8; ++m) ev.out_c[base + (int64_t)(n0 + m) * inner] = make_float2(y[2 * m], y[2 * m + 1]);
          }
        } else {
          float dd[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) dd[m] = y[2 * m] * y[2 * m] + y[2 * m + 1] * y[2 * m + 1];
          if (contiguous) {
            float4* o = reinterpret_cast<float4*>(ev.out_d + base + n0);
            o[0] = make_float4(dd[0], dd[1], dd[2], dd[3]);
            o[1] = make_float4(dd[4], dd[5], dd[6], dd[7]);
          } else {
#pragma unroll
            for (int m = 0; m < 8; ++m) ev.out_d[base + (int64_t)(n0 + m) * inner] = dd[m];
          }
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&acce_bar[buf]));
    }
  }

  tc_fence_before();
  __syncthreads();
  if (tid == 0 && s_abort && P.err) atomicAdd(P.err, 1);
  if (warp == BMMA_WARP) {
    tc_fence_after();
    tmem_free(tmem, BCOLS);
  }
}

// The split of a backward call's adjoint chain: x = 2 g psi (psi the forward
// field, g the density gradient: per realization, or one [M] array shared by
// the batch), into BF16 head and tail planes as bf16_split_kernel does.
__global__ void __launch_bounds__(256) bf16_split_grad_kernel(const float4* __restrict__ field,
                                                               const float2* __restrict__ grad, uint2* __restrict__ hi,
                                                               uint2* __restrict__ lo, int64_t n2, int64_t m2,
                                                               int shared, int unsplit) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = field[i];
    const float2 g = grad[shared ? i % m2 : i];
    const float a = 2.f * g.x, b = 2.f * g.y;
    const float x0 = a * v.x, x1 = a * v.y, x2 = b * v.z, x3 = b * v.w;
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(x0, x1), h1 = __floats2bfloat162_rn(x2, x3);
    hi[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
    if (!unsplit) {
      const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
      lo[i] = make_uint2(pack_bf16(x0 - f0.x, x1 - f0.y), pack_bf16(x2 - f1.x, x3 - f1.y));
    }
  }
}

}  // namespace

cudaError_t launch_bf16_split_grad(const float2* field, const float* grad, int grad_shared, int64_t M,
                                   uint32_t* planes, int64_t n, int64_t plane, int unsplit, int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = bf16_split_grid(n, sms);
  bf16_split_grad_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(field),
                                              reinterpret_cast<const float2*>(grad), reinterpret_cast<uint2*>(planes),
                                              reinterpret_cast<uint2*>(planes + plane), n / 2, M / 2, grad_shared,
                                              unsplit);
  return cudaGetLastError();
}

const void* bf16_split_grad_func() { return (const void*)bf16_split_grad_kernel; }
int bf16_split_grid(int64_t n, int sms) {
  int64_t grid = (n / 2 + 255) / 256;
  if (grid > 8 * (int64_t)sms) grid = 8 * (int64_t)sms;
  return grid < 1 ? 1 : (int)grid;
}

cudaError_t launch_bf16_split(const float2* in, uint32_t* planes, int64_t n, int64_t plane, int unsplit, int sms,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t n2 = n / 2;  // n is even: whole realizations of lattices of >= 64 points
  const int grid = bf16_split_grid(n, sms);
  bf16_split_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(in), reinterpret_cast<uint2*>(planes),
                                              reinterpret_cast<uint2*>(planes + plane), n2, unsplit);
  return cudaGetLastError();
}

bool dense_bf16_supported(int N) { return N >= 64 && N <= kDenseMaxN && N % 32 == 0; }

size_t dense_bf16_t_bytes(int N) { return (size_t)((2 * N + BR - 1) / BR) * ((2 * N + BKC - 1) / BKC) * BTCHUNK; }

namespace {

// the kernel's variants, indexed [FULL][kind], kind 0 plain, 1 ACC, 2 GRAD,
// 3 INBF, 4 INBF + ACC
using BKernel = void (*)(const DenseArgs, const unsigned char*, int*, const CUtensorMap, const int);
constexpr int kBKinds = 5;
BKernel bf16_kernel(bool full, int kind) {
  static const BKernel k[2][kBKinds] = {
      {dense_bf16_kernel<false, false, false, false>, dense_bf16_kernel<false, false, true, false>,
       dense_bf16_kernel<false, true, false, false>, dense_bf16_kernel<false, false, false, true>,
       dense_bf16_kernel<false, false, true, true>},
      {dense_bf16_kernel<true, false, false, false>, dense_bf16_kernel<true, false, true, false>,
       dense_bf16_kernel<true, true, false, false>, dense_bf16_kernel<true, false, false, true>,
       dense_bf16_kernel<true, false, true, true>}};
  return k[full ? 1 : 0][kind];
}
int bf16_kind_smem(int kind) { return bsmem_launch(kind == 2, kind == 1 || kind == 4); }

}  // namespace

cudaError_t dense_bf16_prepare() {
  cudaError_t e = cudaSuccess;
  for (int f = 0; f < 2 && e == cudaSuccess; ++f)
    for (int k = 0; k < kBKinds && e == cudaSuccess; ++k)
      e = cudaFuncSetAttribute((const void*)bf16_kernel(f == 1, k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               bf16_kind_smem(k));
  return e;
}

const void* many_bf16_func(int mode) {
  switch (mode) {
    case 1: return (const void*)dense_bf16_many_kernel<kTmaContiguous, false>;
    case 2: return (const void*)dense_bf16_many_kernel<kTmaPlanes, true>;
    case 4: return (const void*)dense_bf16_many_kernel<kTmaContiguous, true>;
    default: return (const void*)dense_bf16_many_kernel<kInPlace, false>;
  }
}
int many_bf16_threads() { return BTHREADS; }
size_t many_bf16_smem() { return (size_t)BMANY_SMEM; }
cudaError_t many_bf16_prepare() {
  cudaError_t e = cudaSuccess;
  for (int m : {0, 1, 2, 4})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(many_bf16_func(m), cudaFuncAttributeMaxDynamicSharedMemorySize, BMANY_SMEM);
  return e;
}
int many_bf16_lines() { return BL; }
int many_bf16_row_blocks(int N) { return (2 * N + BR - 1) / BR; }
bool many_bf16_supported(int N) { return N >= 32 && N <= 256 && N % 16 == 0; }

cudaError_t launch_bf16_build_t(const float2* T, unsigned char* Tblk, int N, cudaStream_t s) {
  bf16_build_t_kernel<<<256, 256, 0, s>>>(T, Tblk, N);
  return cudaGetLastError();
}

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); NULL if the driver does not offer it
EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// The input tile map of a launch and how the kernel loads its chunks: BF16
// planes as 3-D TMA tiles; FP32 TMA tiles for contiguous lines of forward and
// adjoint passes; in place otherwise (or when the FP32 map cannot be made).
// Returns false when BF16 planes come without a map.
bool input_map(const DenseArgs& a, CUtensorMap* map, int* mode) {
  std::memset(map, 0, sizeof(*map));
  *mode = kInPlace;
  const EncodeTiledFn enc = encode_tiled();
  if (a.in_bf) {
    // [plane][line][2N bf16]: the lines of every realization (contiguous:
    // inner == 1), the tail plane bf_plane pairs after the head plane; a box
    // of 64 values x 128 lines x the planes the launch reads
    if (!enc || a.inner != 1 || a.grad) return false;
    const cuuint64_t rows = (cuuint64_t)a.batch * (cuuint64_t)a.outer;
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * a.N), rows, a.unsplit ? 1u : 2u};
    const cuuint64_t strides[2] = {(cuuint64_t)(2 * a.N) * 2, (cuuint64_t)a.bf_plane * 4};
    const cuuint32_t box[3] = {(cuuint32_t)BKC, (cuuint32_t)BL, a.unsplit ? 1u : 2u}, estr[3] = {1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)a.in_bf, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    *mode = kTmaPlanes;
    return true;
  }
  if (a.grad || a.inner != 1 || !enc) return true;
  const cuuint64_t rows = (cuuint64_t)a.batch * (cuuint64_t)a.outer;  // every realization's lines
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * a.N), rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(2 * a.N) * 4};
  const cuuint32_t box[2] = {32, (cuuint32_t)BL}, estr[2] = {1, 1};
  if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)a.in, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
    *mode = kTmaContiguous;
  else
    std::memset(map, 0, sizeof(*map));
  return true;
}

}  // namespace

bool dense_bf16_chain_supported() { return encode_tiled() != nullptr; }

bool many_bf16_line_map(const float2* base, int N, int64_t lines, void* map) {
  // [lines][2N floats], boxes of 32 floats x 128 lines, 128-byte swizzle: the
  // map of the uniform kernel's TMA tiles of contiguous lines
  std::memset(map, 0, sizeof(CUtensorMap));
  const EncodeTiledFn enc = encode_tiled();
  if (!enc || lines < 1 || (reinterpret_cast<uintptr_t>(base) & 15u)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * N), (cuuint64_t)lines};
  const cuuint64_t strides[1] = {(cuuint64_t)(2 * N) * 4};
  const cuuint32_t box[2] = {32, (cuuint32_t)BL}, estr[2] = {1, 1};
  if (enc(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    std::memset(map, 0, sizeof(CUtensorMap));
    return false;
  }
  return true;
}
static_assert(sizeof(CUtensorMap) == 128, "tile maps are 128 bytes");

bool many_bf16_plane_map(const uint32_t* head, int N, int64_t lines, int64_t plane, void* map) {
  // [plane][line][2N bf16], boxes of 64 values x 128 lines x both planes, 128-byte
  // swizzle: the map of the uniform kernel's BF16-plane tiles
  std::memset(map, 0, sizeof(CUtensorMap));
  const EncodeTiledFn enc = encode_tiled();
  if (!enc || lines < 1 || (reinterpret_cast<uintptr_t>(head) & 15u) || ((plane * 4) & 15)) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * N), (cuuint64_t)lines, 2u};
  const cuuint64_t strides[2] = {(cuuint64_t)(2 * N) * 2, (cuuint64_t)plane * 4};
  const cuuint32_t box[3] = {(cuuint32_t)BKC, (cuuint32_t)BL, 2u}, estr[3] = {1, 1, 1};
  if (enc(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)head, dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    std::memset(map, 0, sizeof(CUtensorMap));
    return false;
  }
  return true;
}

cudaError_t launch_dense_bf16(const DenseArgs& args, const unsigned char* Tblk, int* err, int grid, cudaStream_t s) {
  DenseArgs a = args;
  if (a.oinner == 0) {
    a.oouter = a.outer;
    a.oinner = a.inner;
  }
  CUtensorMap map;
  int mode;
  if (!input_map(a, &map, &mode)) return cudaErrorInvalidValue;
  const bool full = (2 * a.N) % BR == 0;
  // backward passes never accumulate over the batch, nor read BF16 planes
  const int kind = a.grad ? 2 : a.in_bf ? (a.acc ? 4 : 3) : (a.acc ? 1 : 0);
  bf16_kernel(full, kind)<<<grid, BTHREADS, bf16_kind_smem(kind), s>>>(a, Tblk, err, map, mode);
  return cudaGetLastError();
}

}  // namespace ffx
