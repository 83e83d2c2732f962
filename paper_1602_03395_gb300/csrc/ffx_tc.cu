// Dense form on the tensor cores (tcgen05): the per-axis map of lines of N
// points (N a multiple of 16, from 32 up to 1024) as a real matrix product
// with split-TF32 operands, accumulated in tensor memory.
//
// The complex map OUT[n][c] = sum_k T[n][k] IN[k][c] becomes a real product
// with every complex entry t = x + iy of T replaced by the 2 x 2 block
// [[x, -y], [y, x]] and every complex input v = a + ib by the pair (a, b):
// real row 2n is Re OUT[n], row 2n + 1 is Im OUT[n]; real K index 2k + p is
// part p of IN[k].  The MMA runs transposed, D[line][row] = sum_K X[line][K]
// T[row][K], so that tensor-memory lane = line and each epilogue thread owns
// one line's outputs (coalesced stores along either memory order).  Each FP32
// operand is split into a TF32 head and tail: T at plan time (hi =
// rna_tf32(t), lo = rna_tf32(t - hi)), the input on the fly (head = the TF32
// bits of x, tail = x - head, exact).  X_hi T_hi accumulates in one FP32
// tensor-memory accumulator and the cross terms X_hi T_lo + X_lo T_hi in a
// second one, added in the epilogue (the dropped lo*lo term is ~2^-22
// relative).  The tensor cores' FP32 accumulation rounds with a bias, so its
// error grows with the number of MMAs into one accumulator; keeping the small
// cross terms apart leaves the large one N/4 accumulation steps instead of
// 3N/4.
//
// Kernel: one persistent block of 416 threads per SM, warp-specialised.
//  * warps 0-7 (producers), per K chunk of 32 real K: thread 0 starts a bulk
//    (TMA) copy of the pre-split T chunk (128 rows x 32 K, head and tail,
//    stored in global memory already in the tensor cores' K-major no-swizzle
//    core-matrix order) on the stage's "copy" barrier; every producer thread
//    keeps RAW - 1 chunks of its share of the input (16-byte cp.async) in
//    flight in a ring, splits the chunk that has landed into the stage (same
//    core-matrix order, bank-conflict free) and arrives on "full".
//  * warp 8 (MMA): waits "copy" and "full", issues 4 K-steps x 3 products of
//    tcgen05.mma (M = 128 lines, N = 128 rows, K = 8, kind::tf32) into one of
//    two tensor-memory accumulator pairs; tcgen05.commit releases the stage
//    ("empty") and, after a sub-tile's last chunk, hands the accumulator on
//    ("acc_full").
//  * warps 9-12 (epilogue): read their 32-lane quarter of the accumulator
//    (tcgen05.ld), store complex64 or |.|^2 (or add |.|^2 over the batch in
//    shared memory), and arrive on "acc_empty".
// Work items are (128 lines, 128 real rows) of the output, rows fastest
// varying across the items that run together so the lines' inputs are shared
// in L2; with N > 64 a line's outputs span several items, so such passes do
// not run in place.  When 2N is not a multiple of 128 the last row block is
// narrower: its MMAs run with N = the rows that exist (a multiple of 32), its
// T chunks are copied only that far, and the epilogue stops there.
//
// Every wait is bounded; a wait that runs out sets a block-wide abort flag
// (every other wait then gives up at once); producers drain their own copies,
// the MMA thread waits (bounded) for its own tensor-core work, the block frees
// its tensor memory, counts an error in `err` and exits.
//
// Lines of 32 or 64 points (plain passes) also have dense_tm_kernel: T stays
// resident in shared memory and the input operand goes from registers
// straight into tensor memory, with no stage pipeline; launch_dense_tc picks
// it for every 32-point pass (two blocks per SM) and for 64-point passes with
// at most four items per block.  Unsplit launches (FFX_TC_UNSPLIT) run one
// product per K-step on operands rounded to TF32.
#include <algorithm>
#include <cstring>

#include "ffx_internal.h"
#include "ffx_tc_many.h"
#include "ffx_tcgen05.cuh"

namespace ffx {

namespace {

constexpr int LINES = 128;         // lines per item = MMA M = tensor-memory lanes
constexpr int ROWS = 128;          // real output rows per item = MMA N
constexpr int TKC = 32;            // real K per chunk
constexpr int TSTAGES = 2;
constexpr int CORE_LBO = 128;      // bytes between core matrices along K
constexpr int CHUNK_SBO = (TKC / 4) * 128;  // 1024: between 8-row groups of a chunk
constexpr int T_PART = ROWS * TKC * 4;      // 16 KB per split part
constexpr int X_PART = LINES * TKC * 4;     // 16 KB per split part
constexpr int T_CHUNK = 2 * T_PART;         // head + tail, one bulk copy
constexpr int NPROD = 256, NEPI = 128;
constexpr int PITEMS = LINES * (TKC / 4) / NPROD;  // 16-byte input items per producer thread per chunk
constexpr int RAW_CHUNK = NPROD * PITEMS * 16;  // 16 KB
constexpr int GRAD_CHUNK = NPROD * PITEMS * 8;  // 8 KB of gradient factors (backward passes)
// accumulating launches: |.|^2 sums over the batch, [row][line]; backward
// launches: the gradient ring (the two never meet in one launch)
constexpr int EXTRA_SMEM = (ROWS / 2) * 128 * 4;
constexpr int RES_CHUNKS = (2 * 64) / TKC;  // N = 64: all of T is 4 chunks (128 KB)

// Shared-memory layout.  Streaming (any N): stages of [T chunk | X head | X
// tail], a 4-deep input ring, and the optional extra region.  Resident (N = 64,
// plain forward and adjoint passes): all of T stays in shared memory for the
// launch, stages hold only the split input, and the input ring is 2 deep.
template <bool RES>
struct TcLayout {
  static constexpr int T_RES = RES ? RES_CHUNKS * T_CHUNK : 0;
  static constexpr int STAGE = (RES ? 0 : T_CHUNK) + 2 * X_PART;
  static constexpr int X_OFF = RES ? 0 : T_CHUNK;  // split input within a stage
  static constexpr int RAW = RES ? 2 : 4;           // input chunks in flight per producer thread
  static constexpr int RAW_OFF = T_RES + TSTAGES * STAGE;
  static constexpr int SMEM = RAW_OFF + RAW * RAW_CHUNK;  // 224 KB resident, 192 KB streaming
};
static_assert(TcLayout<false>::RAW * GRAD_CHUNK <= EXTRA_SMEM, "gradient ring");
static_assert(TcLayout<false>::SMEM + EXTRA_SMEM <= 227 * 1024 && TcLayout<true>::SMEM <= 227 * 1024, "smem");
constexpr int NTHREADS = NPROD + 32 + NEPI;  // 416
constexpr int MMA_WARP = NPROD / 32;         // warp 8; warps 9-12 are the epilogue
constexpr int ACC_COLS = 4 * ROWS;           // two buffers x (head product, cross terms): all 512

using namespace tc;

// Real output rows of row block mt: ROWS, or what is left of 2N in the last
// block (a multiple of 32, since N is a multiple of 16).
// kind::tf32, M = LINES, N = 2 ROWS: a whole row block's head and tail rows at once
constexpr uint32_t kIdescStack = idesc_tf32(LINES, 2 * ROWS);

__host__ __device__ __forceinline__ int row_count(int N, int mt) {
  const int left = 2 * N - mt * ROWS;
  return left < ROWS ? left : ROWS;
}

// What a role of the kernel needs of one work item: its pass (pointers,
// geometry, split operand blocks of T), its line tile ct and row block mt, and
// the realizations it sums over (nb > 1 only when accumulating).
struct TcView {
  const float2* in;
  const float* grad;
  float2* out_c;
  float* out_d;
  const unsigned char* tblk;
  int64_t outer, inner, M, ncols, ct;
  int N, acc, grad_shared, mt, nb;
};

__device__ __forceinline__ const void* tc_rebase(const TcBases& c, int base, const void* off) {
  return base < 0 ? nullptr : (const void*)((const char*)c.base[base] + (uintptr_t)off);
}

template <bool MANY>
__device__ __forceinline__ TcView tc_view(const TcParams& P, int64_t w) {
  TcView v;
  if (MANY) {
    const TcItem item = P.items[w];
    const TcPassArg& pa = P.args[item.arg];
    const DenseArgs& d = pa.d;
    v.in = (const float2*)tc_rebase(P.call, pa.in_base, d.in);
    v.grad = (const float*)tc_rebase(P.call, pa.grad_base, d.grad);
    v.out_c = (float2*)tc_rebase(P.call, pa.outc_base, d.out_c);
    v.out_d = (float*)tc_rebase(P.call, pa.outd_base, d.out_d);
    v.tblk = pa.tblk;
    v.outer = d.outer;
    v.inner = d.inner;
    v.M = d.M;
    v.ncols = d.ncols;
    v.N = d.N;
    v.acc = 0;
    v.grad_shared = d.grad_shared;
    v.nb = 1;
    v.ct = item.ct;
    v.mt = item.mt;
  } else {
    const DenseArgs& d = P.a;
    const int mtiles = (2 * d.N + ROWS - 1) / ROWS;
    v.in = d.in;
    v.grad = d.grad;
    v.out_c = d.out_c;
    v.out_d = d.out_d;
    v.tblk = P.tblk;
    v.outer = d.outer;
    v.inner = d.inner;
    v.M = d.M;
    v.ncols = d.ncols;
    v.N = d.N;
    v.acc = d.acc;
    v.grad_shared = d.grad_shared;
    v.nb = d.acc ? (int)d.batch : 1;
    v.ct = w / mtiles;
    v.mt = (int)(w % mtiles);
  }
  return v;
}

// Item w of a launch: a new view for many-instance launches; uniform launches
// keep the pass (so its fields stay loop-invariant) and move the item only.
template <bool MANY>
__device__ __forceinline__ void tc_next(const TcParams& P, int64_t w, TcView& v) {
  if (MANY) {
    v = tc_view<true>(P, w);
  } else {
    const int mtiles = (2 * P.a.N + ROWS - 1) / ROWS;
    v.ct = w / mtiles;
    v.mt = (int)(w % mtiles);
  }
}

// Line c of the pass (realization b of the batch when accumulating): offset
// of its first point, or -1 past the end; br = its realization.
__device__ __forceinline__ void line_ref(const TcView& a, int64_t c, int b, long long& base, int& br) {
  base = -1;
  br = 0;
  if (c < a.ncols) {
    const int64_t inner = a.inner;
    int64_t bo = c / inner;
    const int64_t i = c - bo * inner;
    if (a.acc) {
      br = b;
      bo += (int64_t)b * a.outer;
    } else {
      br = (int)(c / (a.outer * inner));
    }
    base = bo * (int64_t)a.N * inner + i;
  }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void split_store(unsigned char* xh, unsigned char* xl, int off, float4 v) {
  const float4 hi = make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
  const float4 lo = make_float4(v.x - hi.x, v.y - hi.y, v.z - hi.z, v.w - hi.w);
  *reinterpret_cast<float4*>(xh + off) = hi;
  *reinterpret_cast<float4*>(xl + off) = lo;
}

// RES: T of a 64-point axis resident (uniform plain passes); MANY: the work
// list of a many-instance phase (every item streams its own T chunks).
// FULL: every row block has ROWS rows (uniform launches with 2N a multiple of
// 128), so the row count, MMA shape and T copy are constants.
template <bool RES, bool MANY, bool FULL>
__global__ void __launch_bounds__(NTHREADS, 1) dense_tc_kernel(const TcParams P) {
  static_assert(!(RES && MANY) && !(MANY && FULL), "many-instance launches stream T, rows vary");
  using L = TcLayout<RES>;
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ __align__(8) uint64_t full_bar[TSTAGES], empty_bar[TSTAGES], copy_bar[TSTAGES];
  __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], done_bar, tres_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  // this block's items: first, first + stride, ... (my_items of them)
  int64_t first, stride, my_items;
  if (MANY) {
    first = P.block_first[blockIdx.x];  // a contiguous run of the work list
    stride = 1;
    my_items = P.block_first[blockIdx.x + 1] - first;
  } else {
    const int mtiles = (2 * P.a.N + ROWS - 1) / ROWS;
    const int64_t items = ((P.a.ncols + LINES - 1) / LINES) * mtiles;
    first = blockIdx.x;
    stride = gridDim.x;
    my_items = (items - blockIdx.x + gridDim.x - 1) / gridDim.x;
  }
  if (my_items <= 0) return;
  // one product per K-step: X and T rounded to TF32, no tails (a reported,
  // less accurate variant)
  const bool unsplit = !MANY && P.a.unsplit;

  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ACC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full_bar[s])), "r"(NPROD) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&copy_bar[s])) : "memory");
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf_bar[b])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce_bar[b])), "r"(NEPI) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done_bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tres_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    if (RES) {
      // all of T (N = 64: one row block, 4 chunks), once for the launch
      const uint32_t tb = smem_u32(&tres_bar);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tb), "r"(L::T_RES) : "memory");
      for (int c = 0; c < RES_CHUNKS; ++c)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(tsm + c * T_CHUNK)),
            "l"(P.tblk + (size_t)c * T_CHUNK), "r"(T_CHUNK), "r"(tb)
            : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t smem_base = smem_u32(tsm);

  if (warp < MMA_WARP) {
    // ---------------- producers ----------------
    const int t = tid;
    unsigned char* raw = tsm + L::RAW_OFF;  // RAW chunks of this thread's inputs
    unsigned char* graw = tsm + L::SMEM;    // and of its gradient factors (backward)
    constexpr int RAW = L::RAW;
    // issue side: chunk (iit, ib, ikc), RAW - 1 ahead of the consumer
    int64_t iit = 0, ci_issue = 0;
    int ib = 0, ikc = 0;
    TcView iv = tc_view<MANY>(P, first);
    int ikchunks = (2 * iv.N) / TKC;
    long long lb[2];
    int lbr[2];
    bool lines_ok = false;
    auto issue = [&]() {
      if (iit < my_items) {
        const bool contiguous = (iv.inner == 1);
        if (!lines_ok) {
          if (contiguous) {
#pragma unroll
            for (int j = 0; j < 2; ++j)
              line_ref(iv, iv.ct * LINES + (t & 7) + 8 * (t >> 5) + 64 * j, ib, lb[j], lbr[j]);
          } else {
            line_ref(iv, iv.ct * LINES + (t & (LINES - 1)), ib, lb[0], lbr[0]);
          }
          lines_ok = true;
        }
        const int64_t inner = iv.inner;
        const int slot = (int)(ci_issue % RAW);
        const uint32_t dst0 = smem_u32(raw + slot * RAW_CHUNK) + (uint32_t)t * 16;
        const uint32_t gdst0 = smem_u32(graw + slot * GRAD_CHUNK) + (uint32_t)t * 8;
#pragma unroll
        for (int i = 0; i < PITEMS; ++i) {
          const uint32_t dst = dst0 + (uint32_t)(i * NPROD * 16);
          long long lbi;
          int bri, kp;
          if (contiguous) {
            lbi = (i < 2) ? lb[0] : lb[1];
            bri = (i < 2) ? lbr[0] : lbr[1];
            kp = ((t >> 3) & 3) + 4 * (i & 1);
          } else {
            lbi = lb[0];
            bri = lbr[0];
            kp = (t >> 7) * PITEMS + i;
          }
          const bool valid = lbi >= 0;
          const int64_t addr = valid ? lbi + (int64_t)(ikc * 16 + 2 * kp) * inner : 0;
          // invalid lines read nothing and land as zeros (source size 0)
          if (contiguous) {
            cp_async16(dst, iv.in + addr, valid ? 16 : 0);
          } else {
            cp_async8(dst, iv.in + addr, valid ? 8 : 0);
            cp_async8(dst + 8, iv.in + addr + (valid ? inner : 0), valid ? 8 : 0);
          }
          if (iv.grad) {
            const int64_t gaddr = valid && iv.grad_shared ? addr - (int64_t)bri * iv.M : addr;
            const uint32_t gdst = gdst0 + (uint32_t)(i * NPROD * 8);
            cp_async4(gdst, iv.grad + gaddr, valid ? 4 : 0);
            cp_async4(gdst + 4, iv.grad + gaddr + (valid ? inner : 0), valid ? 4 : 0);
          }
        }
        ++ci_issue;
        if (++ikc == ikchunks) {
          ikc = 0;
          lines_ok = false;
          if (++ib == iv.nb) {
            ib = 0;
            if (++iit < my_items) {
              tc_next<MANY>(P, first + iit * stride, iv);
              ikchunks = (2 * iv.N) / TKC;
            }
          }
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");  // one group per call, empty past the end
    };
#pragma unroll 1
    for (int r = 0; r < RAW - 1; ++r) issue();
    // consumer side: chunk c = (it, b, kc) of the sequence
    int b = 0, kc = 0;
    TcView cv = tc_view<MANY>(P, first);
    int kchunks = (2 * cv.N) / TKC;
    int last_u[TSTAGES];
#pragma unroll
    for (int q = 0; q < TSTAGES; ++q) last_u[q] = -1;
    int64_t c = 0;
#pragma unroll 1
    for (int64_t it = 0; it < my_items;) {
      issue();
      asm volatile("cp.async.wait_group %0;" ::"n"(RAW - 1) : "memory");  // chunk c has landed
      const int s = (int)(c % TSTAGES);
      const int64_t u = c / TSTAGES;
      if (u >= 1 && !mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)((u - 1) & 1), &s_abort)) break;
      unsigned char* st = tsm + L::T_RES + s * L::STAGE;
      if (!RES && t == 0) {
        // the row block's rows that exist, head and tail parts
        const uint32_t part = (uint32_t)(FULL ? ROWS : row_count(cv.N, cv.mt)) * (TKC * 4);
        const uint32_t cb = smem_u32(&copy_bar[s]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cb),
                     "r"(unsplit ? part : 2 * part)
                     : "memory");
        const unsigned char* src = cv.tblk + ((size_t)cv.mt * kchunks + kc) * T_CHUNK;
        if (unsplit) {
          bulk_g2s(smem_u32(st), src, part, cb);  // the head rows only
        } else if (part == (uint32_t)T_PART) {
          bulk_g2s(smem_u32(st), src, T_CHUNK, cb);  // a whole row block: head and tail in one copy
        } else {
          bulk_g2s(smem_u32(st), src, part, cb);
          bulk_g2s(smem_u32(st + T_PART), src + T_PART, part, cb);
        }
        last_u[s] = (int)(u & 1);
      }
      const int slot = (int)(c % RAW);
      const unsigned char* rs = raw + slot * RAW_CHUNK + t * 16;
      const unsigned char* gs = graw + slot * GRAD_CHUNK + t * 8;
      unsigned char* xh = st + L::X_OFF;
      unsigned char* xl = xh + X_PART;
      const bool contiguous = (cv.inner == 1);
#pragma unroll
      for (int i = 0; i < PITEMS; ++i) {
        float4 v = *reinterpret_cast<const float4*>(rs + i * NPROD * 16);
        if (cv.grad) {
          // the input element is 2 grad * psi
          const float2 gg = *reinterpret_cast<const float2*>(gs + i * NPROD * 8);
          v.x *= 2.f * gg.x;
          v.y *= 2.f * gg.x;
          v.z *= 2.f * gg.y;
          v.w *= 2.f * gg.y;
        }
        int n, kp;
        if (contiguous) {
          n = (t & 7) + 8 * (t >> 5) + 64 * (i >> 1);
          kp = ((t >> 3) & 3) + 4 * (i & 1);
        } else {
          n = t & (LINES - 1);
          kp = (t >> 7) * PITEMS + i;
        }
        const int off = (n >> 3) * CHUNK_SBO + kp * CORE_LBO + (n & 7) * 16;
        if (unsplit)
          *reinterpret_cast<float4*>(xh + off) =
              make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
        else
          split_store(xh, xl, off, v);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&full_bar[s]));
      ++c;
      if (++kc == kchunks) {
        kc = 0;
        if (++b == cv.nb) {
          b = 0;
          if (++it < my_items) {
            tc_next<MANY>(P, first + it * stride, cv);
            kchunks = (2 * cv.N) / TKC;
          }
        }
      }
    }
    // nothing of this thread's may still be in flight at exit
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (t == 0)
      for (int q = 0; q < TSTAGES; ++q)
        if (last_u[q] >= 0) mbar_wait_own(smem_u32(&copy_bar[q]), (uint32_t)last_u[q], &s_abort);
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int64_t g = 0, sub = 0;
      bool ok = !RES || mbar_wait(smem_u32(&tres_bar), 0u, &s_abort);  // resident T has landed
      TcView mv = tc_view<MANY>(P, first);
      for (int64_t it = 0; ok && it < my_items; ++it) {
        if (it > 0) tc_next<MANY>(P, first + it * stride, mv);
        const int kchunks = (2 * mv.N) / TKC;
        const uint32_t idesc = idesc_tf32(LINES, FULL ? ROWS : row_count(mv.N, mv.mt));
        for (int b = 0; ok && b < mv.nb; ++b, ++sub) {
          const int buf = (int)(sub & 1);
          const int64_t v = sub >> 1;
          if (v >= 1 && !mbar_wait(smem_u32(&acce_bar[buf]), (uint32_t)((v - 1) & 1), &s_abort)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d1 = tmem + (uint32_t)(buf * 2 * ROWS), d2 = d1 + ROWS;
          for (int kc = 0; kc < kchunks; ++kc, ++g) {
            const int s = (int)(g % TSTAGES);
            const int64_t u = g / TSTAGES;
            if ((!RES && !mbar_wait(smem_u32(&copy_bar[s]), (uint32_t)(u & 1), &s_abort)) ||
                !mbar_wait(smem_u32(&full_bar[s]), (uint32_t)(u & 1), &s_abort)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = smem_base + (uint32_t)(L::T_RES + s * L::STAGE);
            const uint32_t th = RES ? smem_base + (uint32_t)(kc * T_CHUNK) : st, tl = th + T_PART;
            const uint32_t xh = st + L::X_OFF, xl = xh + X_PART;
#pragma unroll
            for (int ks = 0; ks < TKC / 8; ++ks) {
              const uint32_t o = (uint32_t)(ks * 2 * CORE_LBO);
              const uint64_t dxh = make_desc(xh + o, CORE_LBO, CHUNK_SBO);
              const uint64_t dxl = make_desc(xl + o, CORE_LBO, CHUNK_SBO);
              const uint64_t dth = make_desc(th + o, CORE_LBO, CHUNK_SBO);
              const uint64_t dtl = make_desc(tl + o, CORE_LBO, CHUNK_SBO);
              const uint32_t more = (kc == 0 && ks == 0) ? 0u : 1u;
              if (unsplit) {
                mma_tf32(d1, dxh, dth, idesc, more);
                continue;
              }
              if (RES) {
                // resident T (a whole row block): the chunk's head and tail rows are
                // contiguous 8-row groups, so one N = 256 product forms [X_hi T_hi |
                // X_hi T_lo] in d1, d2 (measured faster here, not on streamed chunks)
                mma_tf32(d1, dxh, dth, kIdescStack, more);
              } else {
                mma_tf32(d1, dxh, dth, idesc, more);
                mma_tf32(d2, dxh, dtl, idesc, more);
              }
              mma_tf32(d2, dxl, dth, idesc, 1u);
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
    const int q = warp & 3;          // tensor-memory lane quarter this warp may read
    const int r = q * 32 + lane;     // line within the item
    float* racc = reinterpret_cast<float*>(tsm + L::SMEM);  // accumulating launches only
    if (!MANY && P.a.acc)
      for (int m = 0; m < ROWS / 2; ++m) racc[m * LINES + r] = 0.f;
    int64_t sub = 0;
    bool ok = true;
    TcView ev = tc_view<MANY>(P, first);
    for (int64_t it = 0; ok && it < my_items; ++it) {
      if (it > 0) tc_next<MANY>(P, first + it * stride, ev);
      const int64_t inner = ev.inner;
      const bool contiguous = (inner == 1);
      const int nbase = ev.mt * (ROWS / 2);
      const int rows = FULL ? ROWS : row_count(ev.N, ev.mt);  // real rows of this item
      for (int b = 0; b < ev.nb; ++b, ++sub) {
        const int buf = (int)(sub & 1);
        const int64_t v = sub >> 1;
        // warp-uniform outcome: the tensor-memory loads below need the whole warp
        ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&accf_bar[buf]), (uint32_t)(v & 1), &s_abort));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        long long base;
        int br;
        line_ref(ev, ev.ct * LINES + r, b, base, br);
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 2 * ROWS);
#pragma unroll 1
        for (int j0 = 0; j0 < rows; j0 += 16) {
          uint32_t x[16], z[16];
          tmem_ld16(taddr + (uint32_t)j0, x);
          if (!unsplit) tmem_ld16(taddr + (uint32_t)(ROWS + j0), z);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          float y[16];
          if (unsplit) {
#pragma unroll
            for (int m = 0; m < 16; ++m) y[m] = __uint_as_float(x[m]);
          } else {
#pragma unroll
            for (int m = 0; m < 16; ++m) y[m] = __uint_as_float(x[m]) + __uint_as_float(z[m]);
          }
          const int n0 = nbase + j0 / 2;  // complex outputs n0 .. n0 + 7 of this line
          if (ev.acc) {
#pragma unroll
            for (int m = 0; m < 8; ++m)
              racc[(j0 / 2 + m) * LINES + r] += y[2 * m] * y[2 * m] + y[2 * m + 1] * y[2 * m + 1];
          } else if (base >= 0) {
            if (ev.out_c) {
              if (contiguous) {
                float4* o = reinterpret_cast<float4*>(ev.out_c + base + n0);
#pragma unroll
                for (int m = 0; m < 4; ++m) o[m] = make_float4(y[4 * m], y[4 * m + 1], y[4 * m + 2], y[4 * m + 3]);
              } else {
#pragma unroll
                for (int m = 0; m < 8; ++m)
                  ev.out_c[base + (int64_t)(n0 + m) * inner] = make_float2(y[2 * m], y[2 * m + 1]);
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
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(smem_u32(&acce_bar[buf]));
        if (ev.acc && b == ev.nb - 1) {
          if (base >= 0) {
            const int64_t o0 = base - (int64_t)br * ev.M + (int64_t)nbase * inner;
            if (contiguous) {
              float4* o = reinterpret_cast<float4*>(ev.out_d + o0);
#pragma unroll 1
              for (int m = 0; m < rows / 8; ++m) {
                float4 cur = o[m];
                cur.x += racc[(4 * m) * LINES + r];
                cur.y += racc[(4 * m + 1) * LINES + r];
                cur.z += racc[(4 * m + 2) * LINES + r];
                cur.w += racc[(4 * m + 3) * LINES + r];
                o[m] = cur;
              }
            } else {
#pragma unroll 1
              for (int m = 0; m < rows / 2; ++m) ev.out_d[o0 + (int64_t)m * inner] += racc[m * LINES + r];
            }
          }
          for (int m = 0; m < ROWS / 2; ++m) racc[m * LINES + r] = 0.f;
        }
      }
    }
  }

  // the resident T copies have landed before the block can exit
  if (RES && tid == 0) mbar_wait_own(smem_u32(&tres_bar), 0u, &s_abort);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && s_abort) atomicAdd(P.err, 1);
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ACC_COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Lines of NP = 32 or 64 points with T resident (plain forward and adjoint
// passes): the input operand in tensor memory, no pipeline stages.  An item
// is 128 lines x all 2 NP real rows.  Per item every thread has half a line in
// registers (loaded during the previous item), writes its values and tails
// into tensor memory (lane = line), and issues the next item's loads; one
// thread runs 2 NP / 8 K-steps (A from tensor memory, T from shared memory);
// all eight warps read the accumulators back and store.  NP = 64: one block
// per SM (all 512 columns), [X_hi T_hi | X_hi T_lo] in one N = 256 product
// (the row block's head and tail rows are contiguous), then X_lo T_hi.
// NP = 32: 256 columns and 64 KB per block, two blocks per SM (one loads while
// the other multiplies); three N = 64 products per K-step.  Unsplit launches
// write the values rounded to TF32 and run one product per K-step.
// ---------------------------------------------------------------------------
constexpr int TM_THREADS = 256;
constexpr uint32_t kIdescRows = idesc_tf32(LINES, ROWS);

template <int NP>
struct TmLayout {
  static constexpr int R = 2 * NP;                     // real rows = real K
  static constexpr int CHUNKS = R / TKC;               // resident T chunks
  static constexpr int SMEM = CHUNKS * T_CHUNK;        // 128 KB (NP = 64), 64 KB (NP = 32)
  static constexpr int COLS = NP == 64 ? 512 : 256;    // tensor-memory columns per block
  static constexpr int D2 = NP == 64 ? ROWS : R;       // cross-term accumulator
  static constexpr int A_HI = 2 * R, A_LO = A_HI + R;  // the input operand after both accumulators
  static constexpr int BLOCKS = NP == 64 ? 1 : 2;      // per SM
  static constexpr int PER_THREAD = NP;                // floats: half a line
};

template <int NP>
__global__ void __launch_bounds__(TM_THREADS, TmLayout<NP>::BLOCKS)
    dense_tm_kernel(const DenseArgs a, const unsigned char* __restrict__ Tblk, int* err) {
  using L = TmLayout<NP>;
  static_assert(L::A_LO + L::R <= L::COLS, "tensor-memory columns");
  extern __shared__ __align__(1024) unsigned char tsm[];  // T: L::CHUNKS chunks of [head | tail]
  __shared__ __align__(8) uint64_t tbar, mbar, dbar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t items = (a.ncols + LINES - 1) / LINES;
  if ((int64_t)blockIdx.x >= items) return;
  const int64_t my_items = (items - blockIdx.x + gridDim.x - 1) / gridDim.x;
  const bool unsplit = a.unsplit != 0;

  if (warp == 0) tmem_alloc(&tmem_slot, L::COLS);
  if (tid == 0) {
    s_abort = 0;
    mbar_init(smem_u32(&tbar), 1);
    mbar_init(smem_u32(&mbar), 1);
    mbar_init(smem_u32(&dbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(smem_u32(&tbar), (uint32_t)L::SMEM);
    for (int c = 0; c < L::CHUNKS; ++c)
      bulk_g2s(smem_u32(tsm + c * T_CHUNK), Tblk + (size_t)c * T_CHUNK, T_CHUNK, smem_u32(&tbar));
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t smem_base = smem_u32(tsm);

  const int q = warp & 3, h = warp >> 2;  // lanes 32 q .. + 31 (lines), points NP/2 h .. + NP/2 - 1
  const int64_t inner = a.inner;
  const bool contiguous = (inner == 1);
  // line c of the pass: offset of its first point, or -1 past the end
  auto line_base = [&](int64_t c) -> long long {
    if (c >= a.ncols) return -1;
    const int64_t bo = c / inner, i = c - bo * inner;
    return bo * NP * inner + i;
  };
  float x[L::PER_THREAD];
  long long base = line_base((int64_t)blockIdx.x * LINES + 32 * q + lane);
  auto load = [&](long long bs) {
    if (contiguous) {
#pragma unroll
      for (int j = 0; j < NP / 4; ++j) {
        const float4 v = bs >= 0 ? __ldcg(reinterpret_cast<const float4*>(a.in + bs + (NP / 2) * h + 2 * j))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
        x[4 * j] = v.x;
        x[4 * j + 1] = v.y;
        x[4 * j + 2] = v.z;
        x[4 * j + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < NP / 2; ++j) {
        const float2 v = bs >= 0 ? __ldcg(a.in + bs + (int64_t)((NP / 2) * h + j) * inner) : make_float2(0.f, 0.f);
        x[2 * j] = v.x;
        x[2 * j + 1] = v.y;
      }
    }
  };
  load(base);
  uint32_t phase = 0;
  bool slices = false, issued = false;
  const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
  const uint32_t a_hi = trow + L::A_HI + (uint32_t)(NP * h), a_lo = trow + L::A_LO + (uint32_t)(NP * h);
  for (int64_t it = 0; it < my_items && !s_abort; ++it) {
    const int64_t ct = blockIdx.x + it * gridDim.x;
    const long long cur = base;
    // this item's values and tails into tensor memory (the previous item's MMAs are done)
    if (unsplit) {
#pragma unroll
      for (int g = 0; g < NP / 16; ++g) {
        uint32_t hi[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) hi[m] = __float_as_uint(tf32_round(x[16 * g + m]));
        tmem_st16(a_hi + 16 * g, hi);
      }
    } else {
#pragma unroll
      for (int g = 0; g < NP / 16; ++g) {
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const float v = x[16 * g + m];
          hi[m] = __float_as_uint(v);
          lo[m] = __float_as_uint(v - tf32_head(v));
        }
        tmem_st16(a_hi + 16 * g, hi);
        tmem_st16(a_lo + 16 * g, lo);
      }
    }
    tmem_wait_st();
    tc_fence_before();
    __syncthreads();
    // the next item's lines, in flight during this item's product and stores
    if (it + 1 < my_items) {
      base = line_base((ct + gridDim.x) * LINES + 32 * q + lane);
      load(base);
    }
    if (tid == 0 && !slices) slices = mbar_wait(smem_u32(&tbar), 0u, &s_abort);
    if (tid == 0 && slices) {
      tc_fence_after();
#pragma unroll 4
      for (int ks = 0; ks < L::R / 8; ++ks) {
        const uint32_t th = smem_base + (uint32_t)((ks >> 2) * T_CHUNK + (ks & 3) * 2 * CORE_LBO);
        const uint64_t dth = make_desc(th, CORE_LBO, CHUNK_SBO);
        const uint32_t more = ks > 0 ? 1u : 0u;
        const uint32_t xh = tmem + L::A_HI + 8 * ks, xl = tmem + L::A_LO + 8 * ks;
        if constexpr (NP == 64) {
          if (unsplit) {
            mma_tf32_ts(tmem, xh, dth, kIdescRows, more);  // X T, rounded operands
          } else {
            mma_tf32_ts(tmem, xh, dth, kIdescStack, more);           // [X_hi T_hi | X_hi T_lo]
            mma_tf32_ts(tmem + L::D2, xl, dth, kIdescRows, 1u);     // + X_lo T_hi
          }
        } else {
          constexpr uint32_t idesc = idesc_tf32(LINES, 2 * NP);
          const uint64_t dtl = make_desc(th + T_PART, CORE_LBO, CHUNK_SBO);
          mma_tf32_ts(tmem, xh, dth, idesc, more);  // X_hi T_hi (unsplit: X T)
          if (!unsplit) {
            mma_tf32_ts(tmem + L::D2, xh, dtl, idesc, more);  // X_hi T_lo
            mma_tf32_ts(tmem + L::D2, xl, dth, idesc, 1u);    // + X_lo T_hi
          }
        }
      }
      mma_commit(smem_u32(&mbar));
      issued = true;
    }
    const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&mbar), phase, &s_abort));
    phase ^= 1u;
    if (!ok) break;
    tc_fence_after();
    // accumulators: warp (q, h) reads real rows NP h .. NP h + NP - 1 of its 32 lines
#pragma unroll 1
    for (int j0 = 0; j0 < NP; j0 += 16) {
      uint32_t x1[16], x2[16];
      tmem_ld16(trow + (uint32_t)(NP * h + j0), x1);
      if (!unsplit) tmem_ld16(trow + (uint32_t)(L::D2 + NP * h + j0), x2);
      tmem_wait_ld();
      if (cur < 0) continue;
      float y[16];
      if (unsplit) {
#pragma unroll
        for (int m = 0; m < 16; ++m) y[m] = __uint_as_float(x1[m]);
      } else {
#pragma unroll
        for (int m = 0; m < 16; ++m) y[m] = __uint_as_float(x1[m]) + __uint_as_float(x2[m]);
      }
      const int n0 = (NP / 2) * h + j0 / 2;  // complex outputs n0 .. n0 + 7
      if (a.out_c) {
        if (contiguous) {
          float4* o = reinterpret_cast<float4*>(a.out_c + cur + n0);
#pragma unroll
          for (int m = 0; m < 4; ++m) o[m] = make_float4(y[4 * m], y[4 * m + 1], y[4 * m + 2], y[4 * m + 3]);
        } else {
#pragma unroll
          for (int m = 0; m < 8; ++m) a.out_c[cur + (int64_t)(n0 + m) * inner] = make_float2(y[2 * m], y[2 * m + 1]);
        }
      } else {
        float dd[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) dd[m] = y[2 * m] * y[2 * m] + y[2 * m + 1] * y[2 * m + 1];
        if (contiguous) {
          float4* o = reinterpret_cast<float4*>(a.out_d + cur + n0);
          o[0] = make_float4(dd[0], dd[1], dd[2], dd[3]);
          o[1] = make_float4(dd[4], dd[5], dd[6], dd[7]);
        } else {
#pragma unroll
          for (int m = 0; m < 8; ++m) a.out_d[cur + (int64_t)(n0 + m) * inner] = dd[m];
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // accumulators read before the next item's product
  }
  if (tid == 0) {
    if (issued) {
      mma_commit(smem_u32(&dbar));
      mbar_wait_own(smem_u32(&dbar), 0u, &s_abort);
    }
    mbar_wait_own(smem_u32(&tbar), 0u, &s_abort);
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && s_abort && err) atomicAdd(err, 1);
  if (warp == 0) {
    tc_fence_after();
    tmem_free(tmem, L::COLS);
  }
}

// Pre-split T chunks from the complex map T [N][N]: for row block mt and K
// chunk kc, a 32 KB block [head: 128 rows x 32 K][tail] in core-matrix order;
// real (r, k') with r = 2n + p_out, k' = 2k + p_in holds the 2 x 2 block
// entry of T[n][k].
__global__ void tc_build_t_kernel(const float2* __restrict__ T, unsigned char* __restrict__ Tblk, int N) {
  const int R = 2 * N;
  const int RP = (R + ROWS - 1) / ROWS * ROWS;  // rows padded to whole row blocks (zeros past R)
  const int kchunks = R / TKC;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)RP * R;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / R), kp = (int)(idx - (int64_t)r * R);
    const int n = r >> 1, po = r & 1, k = kp >> 1, pi = kp & 1;
    float v = 0.f;
    if (r < R) {
      const float2 t = T[(int64_t)n * N + k];
      if (po == 0)
        v = pi == 0 ? t.x : -t.y;
      else
        v = pi == 0 ? t.y : t.x;
    }
    const float hi = tf32_round(v);
    const int mt = r / ROWS, rr = r % ROWS, kc = kp / TKC, kk = kp % TKC;
    unsigned char* blk = Tblk + ((size_t)mt * kchunks + kc) * T_CHUNK;
    const int off = (rr >> 3) * CHUNK_SBO + (kk >> 2) * CORE_LBO + (rr & 7) * 16 + (kk & 3) * 4;
    *reinterpret_cast<float*>(blk + off) = hi;
    *reinterpret_cast<float*>(blk + T_PART + off) = tf32_round(v - hi);
  }
}

}  // namespace

bool dense_tc_supported(int N) { return N >= 32 && N <= kDenseMaxN && N % 16 == 0; }
cudaError_t dense_tc_prepare() {
  cudaError_t e = cudaFuncSetAttribute(dense_tc_kernel<false, false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, TcLayout<false>::SMEM + EXTRA_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dense_tc_kernel<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TcLayout<false>::SMEM + EXTRA_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dense_tc_kernel<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TcLayout<true>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dense_tm_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmLayout<64>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dense_tm_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmLayout<32>::SMEM);
  return e;
}
size_t dense_tc_t_bytes(int N) {
  return (size_t)((2 * N + ROWS - 1) / ROWS) * ((2 * N) / TKC) * T_CHUNK;  // row blocks x K chunks
}

cudaError_t launch_dense_tc(const DenseArgs& a, const unsigned char* Tblk, int* err, int grid,
                            cudaStream_t stream) {
  TcParams P;
  std::memset(&P, 0, sizeof(P));
  P.a = a;
  P.tblk = Tblk;
  P.err = err;
  const int64_t items = (a.ncols + LINES - 1) / LINES;
  if (a.N == 32 && !a.acc && !a.grad) {
    // two blocks per SM (grid = the SMs when the pass has more items than SMs)
    const int64_t g = items > grid ? std::min<int64_t>(items, 2 * (int64_t)grid) : grid;
    dense_tm_kernel<32><<<(unsigned)g, TM_THREADS, TmLayout<32>::SMEM, stream>>>(a, Tblk, err);
  } else if (a.N == 64 && !a.acc && !a.grad && items <= 4 * (int64_t)grid) {
    // a few items per block: the input operand in tensor memory, no pipeline
    // to fill (measured 7-14% faster at up to ~2 items per SM, 6% slower at 13)
    dense_tm_kernel<64><<<grid, TM_THREADS, TmLayout<64>::SMEM, stream>>>(a, Tblk, err);
  } else if (a.N == 64 && !a.acc && !a.grad) {
    // T (128 KB) stays in shared memory for the whole launch
    dense_tc_kernel<true, false, true><<<grid, NTHREADS, TcLayout<true>::SMEM, stream>>>(P);
  } else {
    const int smem = TcLayout<false>::SMEM + ((a.acc || a.grad) ? EXTRA_SMEM : 0);
    if ((2 * a.N) % ROWS == 0)
      dense_tc_kernel<false, false, true><<<grid, NTHREADS, smem, stream>>>(P);
    else
      dense_tc_kernel<false, false, false><<<grid, NTHREADS, smem, stream>>>(P);
  }
  return cudaGetLastError();
}

int64_t dense_tc_tiles(int N, int64_t ncols) {
  return ((ncols + LINES - 1) / LINES) * ((2 * N + ROWS - 1) / ROWS);
}

cudaError_t launch_tc_build_t(const float2* T, unsigned char* Tblk, int N, cudaStream_t s) {
  tc_build_t_kernel<<<256, 256, 0, s>>>(T, Tblk, N);
  return cudaGetLastError();
}

// ---- many-instance phases ----

const void* many_tc_func() { return (const void*)dense_tc_kernel<false, true, false>; }
int many_tc_threads() { return NTHREADS; }
size_t many_tc_smem() { return (size_t)TcLayout<false>::SMEM + EXTRA_SMEM; }
cudaError_t many_tc_prepare() {
  return cudaFuncSetAttribute(dense_tc_kernel<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)many_tc_smem());
}
int many_tc_lines() { return LINES; }
int many_tc_row_blocks(int N) { return (2 * N + ROWS - 1) / ROWS; }

}  // namespace ffx
