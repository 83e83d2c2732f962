// Dense form on the tensor cores (tcgen05): the per-axis map of lines of
// 64 points as a real 128 x 128 matrix product with split-TF32 operands.
//
// The complex map OUT[n][c] = sum_k T[n][k] IN[k][c] becomes a real product
// with every complex entry t = x + iy of T replaced by the 2 x 2 block
// [[x, -y], [y, x]] and every complex input v = a + ib by the pair (a, b):
// real row 2n is Re OUT[n], row 2n + 1 is Im OUT[n]; real K index 2k + p is
// part p of IN[k].  Each FP32 operand is split into a TF32 head and a TF32
// tail (hi = rna_tf32(x), lo = rna_tf32(x - hi)); the product accumulates
// A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 in tensor memory, which keeps
// ~2^-21 of relative precision (the dropped lo*lo term is below that).
//
// Kernel: one block of 128 threads per SM (persistent), the whole split A
// (2 x 64 KB) resident in shared memory in the tensor cores' K-major
// no-swizzle layout (8-row x 16-byte core matrices; 128 bytes between core
// matrices along K, 4096 bytes between 8-row groups).  Work items are tiles of
// 64 lines (the MMA N dimension) -- times the realizations of the batch when
// summing the ensemble.  The input of a tile arrives in 4 chunks of 32 real K
// (16 complex rows), double-buffered: the threads load, split and lay out
// chunk c + 1 while the tensor cores multiply chunk c (12 MMAs of
// M=128, N=64, K=8, issued by one thread, completion signalled on an
// mbarrier by tcgen05.commit).  The epilogue reads the accumulator from tensor
// memory (tcgen05.ld, one 32-lane quarter per warp), pairs real and imaginary
// rows with a shuffle and stores complex64, |.|^2 or the ensemble sum.
//
// Every wait is bounded: a wait that runs out counts an error in
// a.err (device memory), stops the block's work and frees its tensor memory.
#include <cstring>

#include "ffx_internal.h"

namespace ffx {

namespace {

constexpr int TN = 64;            // complex line length
constexpr int TM = 128;           // real rows (2 TN) = MMA M
constexpr int TK = 128;           // real K (2 TN)
constexpr int TCN = 64;           // lines per tile = MMA N
constexpr int TKC = 32;           // real K per chunk
constexpr int TCHUNKS = TK / TKC;  // 4
constexpr int TSTAGES = 2;
constexpr int A_BYTES = TM * TK * 4;                 // 64 KB per split part
constexpr int A_SBO = (TK / 4) * 128;                // 4096: between 8-row groups
constexpr int B_CHUNK_BYTES = TCN * TKC * 4;         // 8 KB per split part
constexpr int B_SBO = (TKC / 4) * 128;               // 1024
constexpr int CORE_LBO = 128;                        // between core matrices along K
constexpr int TC_SMEM = 2 * A_BYTES + TSTAGES * 2 * B_CHUNK_BYTES + 256;
constexpr long long kSpinLimit = 1ll << 22;  // try_wait polls: a few seconds at most

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// K-major, no swizzle: start >> 4 | LBO >> 4 << 16 | SBO >> 4 << 32 | version 1 << 46
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::tf32, D = F32, A = B = TF32, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TCN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long i = 0; i < kSpinLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc)
      : "memory");
}

// Lines (columns) of one work item.
__device__ __forceinline__ void tc_bases(const DenseArgs& a, int64_t ct, int b, long long* cbase, int* cbr,
                                         int t) {
  const int64_t inner = a.inner;
  const int64_t c = ct * TCN + t;
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
    base = bo * (int64_t)TN * inner + i;
  }
  cbase[t] = base;
  cbr[t] = br;
}

__global__ void __launch_bounds__(128, 1) dense_tc_kernel(const DenseArgs a, const float* __restrict__ Ahi,
                                                          const float* __restrict__ Alo, int* err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sA_hi = tsm;
  unsigned char* sA_lo = tsm + A_BYTES;
  unsigned char* sB = tsm + 2 * A_BYTES;  // [stage][hi, lo][B_CHUNK_BYTES]
  __shared__ __align__(8) uint64_t mbar[TSTAGES];
  __shared__ uint32_t tmem_slot;
  __shared__ long long cbase[TCN];
  __shared__ int cbr[TCN];
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int64_t inner = a.inner;
  const bool contiguous = (inner == 1);
  const int64_t col_tiles = (a.ncols + TCN - 1) / TCN;
  const int nb = a.acc ? (int)a.batch : 1;
  if ((int64_t)blockIdx.x >= col_tiles) return;
  const int64_t my_tiles = (col_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
  const int64_t n_items = my_tiles * nb;

  // tensor memory for the 128 x 64 FP32 accumulator
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TCN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < TSTAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  // the split A, already in core-matrix order in global memory: a straight copy
  {
    const float4* gh = reinterpret_cast<const float4*>(Ahi);
    const float4* gl = reinterpret_cast<const float4*>(Alo);
    float4* sh = reinterpret_cast<float4*>(sA_hi);
    float4* sl = reinterpret_cast<float4*>(sA_lo);
    for (int i = tid; i < A_BYTES / 16; i += 128) {
      sh[i] = __ldg(gh + i);
      sl[i] = __ldg(gl + i);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t a_hi_addr = smem_u32(sA_hi), a_lo_addr = smem_u32(sA_lo), b_addr = smem_u32(sB);

  float racc[TCN];
#pragma unroll
  for (int j = 0; j < TCN; ++j) racc[j] = 0.f;

  int64_t gchunk = 0;  // chunks issued so far (stage = gchunk % 2)
  bool ok = true;
  for (int64_t it = 0; it < n_items && ok; ++it) {
    const int64_t ct = blockIdx.x + (it / nb) * gridDim.x;
    const int b = (int)(it % nb);
    __syncthreads();  // cbase of the previous item no longer read
    if (tid < TCN) tc_bases(a, ct, b, cbase, cbr, tid);
    __syncthreads();
    for (int c = 0; c < TCHUNKS && ok; ++c, ++gchunk) {
      const int stage = (int)(gchunk & 1);
      if (gchunk >= TSTAGES) {
        // the MMAs that last read this stage (chunk gchunk - 2) are done;
        // thread 0 waits, the block follows it through the barrier
        if (tid == 0 && !mbar_wait(smem_u32(&mbar[stage]), (uint32_t)(((gchunk - TSTAGES) >> 1) & 1)))
          s_abort = 1;
        __syncthreads();
        if (s_abort) {
          ok = false;
          break;
        }
      }
      // load 16 complex rows x 64 lines, split, lay out as (line n, real k) K-major
      unsigned char* bh = sB + stage * 2 * B_CHUNK_BYTES;
      unsigned char* bl = bh + B_CHUNK_BYTES;
      for (int idx = tid; idx < 16 * TCN; idx += 128) {
        int kl, n;
        if (contiguous) {
          n = idx >> 4;
          kl = idx & 15;
        } else {
          kl = idx / TCN;
          n = idx - kl * TCN;
        }
        const int k = c * 16 + kl;
        float2 v = make_float2(0.f, 0.f);
        const long long base = cbase[n];
        if (base >= 0) {
          const int64_t addr = base + (int64_t)k * inner;
          v = a.in[addr];  // plain load: passes may run in place
          if (a.grad) {
            const int64_t gaddr = a.grad_shared ? addr - (int64_t)cbr[n] * a.M : addr;
            const float gr = 2.f * __ldg(a.grad + gaddr);
            v.x *= gr;
            v.y *= gr;
          }
        }
        const float2 hi = make_float2(tf32_hi(v.x), tf32_hi(v.y));
        const float2 lo = make_float2(tf32_hi(v.x - hi.x), tf32_hi(v.y - hi.y));
        const int off = (n >> 3) * B_SBO + (kl >> 1) * CORE_LBO + (n & 7) * 16 + (kl & 1) * 8;
        *reinterpret_cast<float2*>(bh + off) = hi;
        *reinterpret_cast<float2*>(bl + off) = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t bh_addr = b_addr + stage * 2 * B_CHUNK_BYTES;
        const uint32_t bl_addr = bh_addr + B_CHUNK_BYTES;
#pragma unroll
        for (int ks = 0; ks < TKC / 8; ++ks) {
          const uint32_t a_off = (uint32_t)((c * (TKC / 8) + ks) * 2 * CORE_LBO);
          const uint32_t b_off = (uint32_t)(ks * 2 * CORE_LBO);
          const uint64_t dah = make_desc(a_hi_addr + a_off, CORE_LBO, A_SBO);
          const uint64_t dal = make_desc(a_lo_addr + a_off, CORE_LBO, A_SBO);
          const uint64_t dbh = make_desc(bh_addr + b_off, CORE_LBO, B_SBO);
          const uint64_t dbl = make_desc(bl_addr + b_off, CORE_LBO, B_SBO);
          const uint32_t first = (c == 0 && ks == 0) ? 0u : 1u;
          mma_tf32(tmem, dah, dbh, first);
          mma_tf32(tmem, dah, dbl, 1u);
          mma_tf32(tmem, dal, dbh, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mbar[stage]))
                     : "memory");
      }
    }
    if (!ok) break;
    // the last commit covers every MMA of this item
    const int64_t last = gchunk - 1;
    if (tid == 0 && !mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1))) s_abort = 1;
    __syncthreads();
    if (s_abort) {
      ok = false;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // accumulator row r = 32 warp + lane: output n = r / 2, part r % 2
    float d[TCN];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int j0 = 0; j0 < TCN; j0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr + (uint32_t)j0));
#pragma unroll
      for (int j = 0; j < 16; ++j) d[j0 + j] = __uint_as_float(r[j]);
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    const int n = (warp * 32 + lane) >> 1;
    const bool re_lane = (lane & 1) == 0;
    const bool tile_done = !a.acc || b == nb - 1;
#pragma unroll
    for (int j = 0; j < TCN; ++j) {
      const float other = __shfl_xor_sync(0xffffffffu, d[j], 1);
      if (re_lane) {
        const float re = d[j], im = other;
        const long long base = cbase[j];
        if (a.acc) {
          racc[j] += re * re + im * im;
        } else if (base >= 0) {
          const int64_t addr = base + (int64_t)n * inner;
          if (a.out_c)
            a.out_c[addr] = make_float2(re, im);
          else
            a.out_d[addr] = re * re + im * im;
        }
      }
    }
    if (a.acc && tile_done && re_lane) {
#pragma unroll
      for (int j = 0; j < TCN; ++j) {
        const long long base = cbase[j];
        if (base >= 0) a.out_d[base - (int64_t)b * a.M + (int64_t)n * inner] += racc[j];
        racc[j] = 0.f;
      }
    }
  }
  if (!ok && tid == 0) atomicAdd(err, 1);
  // all tensor-memory reads are done before the accumulator is freed
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCN) : "memory");
  }
}

// Split A in core-matrix order from the complex map T [64][64]:
// real (r, k') with r = 2n + p_out, k' = 2k + p_in, value = block entry of T[n][k].
__global__ void tc_build_a_kernel(const float2* __restrict__ T, float* __restrict__ Ahi, float* __restrict__ Alo) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < TM * TK; idx += gridDim.x * blockDim.x) {
    const int r = idx / TK, kp = idx - r * TK;
    const int n = r >> 1, po = r & 1, k = kp >> 1, pi = kp & 1;
    const float2 t = T[n * TN + k];
    float v;
    if (po == 0)
      v = pi == 0 ? t.x : -t.y;
    else
      v = pi == 0 ? t.y : t.x;
    const float hi = tf32_hi(v);
    const int off = ((r >> 3) * A_SBO + (kp >> 2) * CORE_LBO + (r & 7) * 16 + (kp & 3) * 4) / 4;
    Ahi[off] = hi;
    Alo[off] = tf32_hi(v - hi);
  }
}

}  // namespace

size_t dense_tc_smem() { return (size_t)TC_SMEM; }
const void* dense_tc_func() { return (const void*)dense_tc_kernel; }
size_t dense_tc_a_floats() { return (size_t)TM * TK; }

cudaError_t launch_dense_tc(const DenseArgs& a, const float* Ahi, const float* Alo, int* err, int grid,
                            cudaStream_t stream) {
  dense_tc_kernel<<<grid, 128, TC_SMEM, stream>>>(a, Ahi, Alo, err);
  return cudaGetLastError();
}

int64_t dense_tc_tiles(int64_t ncols) { return (ncols + TCN - 1) / TCN; }

cudaError_t launch_tc_build_a(const float2* T, float* Ahi, float* Alo, cudaStream_t s) {
  tc_build_a_kernel<<<64, 256, 0, s>>>(T, Ahi, Alo);
  return cudaGetLastError();
}

}  // namespace ffx
