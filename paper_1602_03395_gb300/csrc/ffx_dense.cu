// Dense form of one axis pass: the per-axis map as an N x N matrix.
//
// The d-dimensional map of eq. FF is a tensor product of per-axis maps
// (every phase of eq. FF is exp(i sum_j ...), and n'' is per axis), and each
// per-axis map is linear: Psibar_nb = sum_n T[nb, n] psi_n.  The plan builds
// T once on the GPU by running the FFT-form pass (pre-chirp, FFT, k-space
// phase, fold, inverse FFT) on the N unit vectors, so T is the same map the
// line passes apply, at the same FP32 accuracy.  A pass then is one batched
// complex matrix product per axis: for every (realization, outer) slab,
// OUT[N x inner] = T[N x N] * IN[N x inner]; for the contiguous axis the slab
// is [lines x N] and the product runs on its transpose.  It costs 8N flops per
// point instead of the FFT form's lam (5 log2 N + 14), which is the cheaper
// form when lam is large against N.
//
// Kernel: 256 threads compute a 64 (rows nb) x 32 (columns = lines) tile;
// thread (tx, ty) owns rows ty + 16 i (i < 4) and columns tx + 16 j (j < 2),
// so shared-memory reads of both operands are conflict-free.  K runs in chunks
// of 16 through shared memory.  The epilogue writes complex64, or |.|^2, or
// |.|^2 summed over the batch (the tile then loops over b, deterministic).
#include <cstring>

#include "ffx_dense_tile.cuh"
#include "ffx_internal.h"

namespace ffx {

namespace {

__global__ void __launch_bounds__(256) dense_pass_kernel(const DenseArgs a) {
  __shared__ DenseTileSmem sm;
  const int64_t ntiles = dense_tile_count(a.N, a.ncols);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) dense_tile(a, tile, sm);
}

// Lines of at most 64 points: T stays in shared memory for the whole launch,
// an NM x BN output tile (rows x lines) takes all of K at once, each of 128
// threads owns an (NM/16) x (BN/8) block (rows ty + 16 i, columns tx + 8 j),
// and the next tile's input is loaded into registers while the current one is
// multiplied.  Two shapes: 64 x 32 for lines of 33..64 points, 32 x 64 for
// lines of at most 32 (no rows wasted past N).  Items are (column tile,
// realization) pairs; with ensemble summing a block takes every realization of
// its column tile in order.  Every output is the same FMA sequence (k
// ascending) in either shape.
constexpr int STX = 8, STY = 16, SNMAX = 64;
constexpr int SIMG = SNMAX + 1;  // image row stride (img[k][m] = T[m][k])

struct SmallItem {
  int64_t cbk;
  int b;
};

template <int SBN>
__device__ __forceinline__ void small_bases(const DenseArgs& a, int64_t cbk, int b, long long* cbase,
                                            int* cbr, int t) {
  // column t of column tile cbk, realization b (b only used when summing the ensemble)
  const int64_t inner = a.inner;
  const int64_t c = cbk * SBN + t;
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
    base = bo * (int64_t)a.N * inner + i;
  }
  cbase[t] = base;
  cbr[t] = br;
}

__device__ __forceinline__ uint32_t dsm_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int NM, int SBN>
__global__ void __launch_bounds__(128) dense_small_kernel(const DenseArgs a) {
  constexpr int STM = NM / STY, STN = SBN / STX;
  extern __shared__ __align__(16) unsigned char dsm[];
  float2* As = reinterpret_cast<float2*>(dsm);     // [NM][SIMG], As[k][m] = A[m][k]
  float2* Bs = As + NM * SIMG;                     // [2][NM][SBN + 1]
  constexpr int BSTRIDE = NM * (SBN + 1);
  __shared__ long long cbase[2][SBN];
  __shared__ int cbr[2][SBN];
  __shared__ __align__(8) uint64_t abar;
  __shared__ int s_abort;

  const int N = a.N;
  const int tid = threadIdx.x;
  const int tx = tid % STX, ty = tid / STX;
  const int64_t inner = a.inner;
  const bool contiguous = (inner == 1);
  const int64_t col_tiles = (a.ncols + SBN - 1) / SBN;
  const int nb = a.acc ? (int)a.batch : 1;
  // this block's items: column tiles blockIdx.x, blockIdx.x + gridDim.x, ...; each for nb realizations
  const int64_t my_tiles = (col_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
  const int64_t n_items = (blockIdx.x < col_tiles) ? my_tiles * nb : 0;
  if (n_items == 0) return;

  // T, stored in global memory as the image of As, arrives in one bulk (TMA) copy
  const uint32_t abytes = (uint32_t)(N * SIMG * sizeof(float2));
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(dsm_u32(&abar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(dsm_u32(&abar)), "r"(abytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dsm_u32(As)),
        "l"(a.Aimg), "r"(abytes), "r"(dsm_u32(&abar))
        : "memory");
  }

  auto item_at = [&](int64_t it) {
    SmallItem r;
    r.cbk = blockIdx.x + (it / nb) * gridDim.x;
    r.b = (int)(it % nb);
    return r;
  };
  // input tile of an item: asynchronous 8-byte copies straight into Bs[buf][k][cc]
  // (with the ensemble-gradient factor the values go through registers)
  auto issue_item = [&](int buf) {
    float2* dst = Bs + buf * BSTRIDE;
    for (int idx = tid; idx < NM * SBN; idx += 128) {
      int k, cc;
      if (contiguous) {
        cc = idx / NM;
        k = idx - cc * NM;
      } else {
        k = idx / SBN;
        cc = idx - k * SBN;
      }
      if (k >= N) continue;
      float2* d = dst + k * (SBN + 1) + cc;
      const long long base = cbase[buf][cc];
      if (base < 0) {
        *d = make_float2(0.f, 0.f);
        continue;
      }
      const int64_t addr = base + (int64_t)k * inner;
      if (a.grad) {
        float2 v = a.in[addr];
        const int64_t gaddr = a.grad_shared ? addr - (int64_t)cbr[buf][cc] * a.M : addr;
        const float gr = 2.f * __ldg(a.grad + gaddr);
        v.x *= gr;
        v.y *= gr;
        *d = v;
      } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dsm_u32(d)), "l"(a.in + addr) : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  if (tid < SBN) {
    const SmallItem i0 = item_at(0);
    small_bases<SBN>(a, i0.cbk, i0.b, cbase[0], cbr[0], tid);
  }
  __syncthreads();
  issue_item(0);
  // every thread waits for T (bounded; a timeout abandons the launch)
  {
    bool done = false;
    for (long long i = 0; i < (1ll << 22) && !done; ++i) {
      uint32_t d;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(d)
          : "r"(dsm_u32(&abar))
          : "memory");
      done = d != 0;
    }
    if (!done) s_abort = 1;
  }

  float racc[STM][STN];
#pragma unroll
  for (int i = 0; i < STM; ++i)
#pragma unroll
    for (int j = 0; j < STN; ++j) racc[i][j] = 0.f;

  for (int64_t it = 0; it < n_items; ++it) {
    const int buf = (int)(it & 1);
    const SmallItem cur = item_at(it);
    __syncthreads();  // previous epilogue done with Bs[buf ^ 1] and cbase[buf ^ 1]
    if (s_abort) break;
    const bool more = it + 1 < n_items;
    if (more) {
      if (tid < SBN) {
        const SmallItem nx = item_at(it + 1);
        small_bases<SBN>(a, nx.cbk, nx.b, cbase[buf ^ 1], cbr[buf ^ 1], tid);
      }
      __syncthreads();
      issue_item(buf ^ 1);  // in flight during this item's product
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();  // this item's tile is in Bs[buf]
    const float2* B = Bs + buf * BSTRIDE;

    float2 acc[STM][STN];
#pragma unroll
    for (int i = 0; i < STM; ++i)
#pragma unroll
      for (int j = 0; j < STN; ++j) acc[i][j] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int k = 0; k < N; ++k) {
      float2 av[STM], bv[STN];
#pragma unroll
      for (int i = 0; i < STM; ++i) av[i] = As[k * SIMG + ty + STY * i];
#pragma unroll
      for (int j = 0; j < STN; ++j) bv[j] = B[k * (SBN + 1) + tx + STX * j];
#pragma unroll
      for (int i = 0; i < STM; ++i)
#pragma unroll
        for (int j = 0; j < STN; ++j) dcfma(acc[i][j], av[i], bv[j]);
    }

    const bool tile_done = !a.acc || cur.b == nb - 1;
    if (a.acc) {
#pragma unroll
      for (int i = 0; i < STM; ++i)
#pragma unroll
        for (int j = 0; j < STN; ++j) racc[i][j] += acc[i][j].x * acc[i][j].x + acc[i][j].y * acc[i][j].y;
    }
    if (tile_done) {
      // stage the tile in Bs[buf] (rows m, columns cc) and store it coalesced
      float2* S = Bs + buf * BSTRIDE;
      __syncthreads();
#pragma unroll
      for (int i = 0; i < STM; ++i)
#pragma unroll
        for (int j = 0; j < STN; ++j) {
          float2 v = acc[i][j];
          if (a.acc) v = make_float2(racc[i][j], 0.f);
          S[(ty + STY * i) * (SBN + 1) + tx + STX * j] = v;
        }
      __syncthreads();
      for (int idx = tid; idx < N * SBN; idx += 128) {
        int m, cc;
        if (contiguous) {
          cc = idx / N;
          m = idx - cc * N;
        } else {
          m = idx / SBN;
          cc = idx - m * SBN;
        }
        const long long base = cbase[buf][cc];
        if (base < 0) continue;
        const float2 v = S[m * (SBN + 1) + cc];
        if (a.acc) {
          a.out_d[base - (int64_t)cur.b * a.M + (int64_t)m * inner] += v.x;
        } else {
          const int64_t addr = base + (int64_t)m * inner;
          if (a.out_c)
            a.out_c[addr] = v;
          else
            a.out_d[addr] = v.x * v.x + v.y * v.y;
        }
      }
#pragma unroll
      for (int i = 0; i < STM; ++i)
#pragma unroll
        for (int j = 0; j < STN; ++j) racc[i][j] = 0.f;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (tid == 0 && s_abort && a.err) atomicAdd(a.err, 1);
}

// T's image for the kernel above: img[k][m] = T[m][k], rows of SNMAX + 1.
__global__ void dense_small_image_kernel(const float2* __restrict__ T, float2* __restrict__ img, int N) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N * SIMG; idx += gridDim.x * blockDim.x) {
    const int k = idx / SIMG, m = idx - k * SIMG;
    img[idx] = (m < N) ? T[m * N + k] : make_float2(0.f, 0.f);
  }
}

}  // namespace

// lines of at most 32 points take the 32 x 64 tile, longer ones 64 x 32
const void* dense_small_func(int N) {
  return N <= 32 ? (const void*)dense_small_kernel<32, 64> : (const void*)dense_small_kernel<64, 32>;
}
size_t dense_small_smem(int N) {
  return N <= 32 ? sizeof(float2) * (32 * SIMG + 2 * 32 * 65) : sizeof(float2) * (64 * SIMG + 2 * 64 * 33);
}
size_t dense_small_image_floats2(int N) { return (size_t)N * SIMG; }
cudaError_t launch_dense_small_image(const float2* T, float2* img, int N, cudaStream_t s) {
  dense_small_image_kernel<<<16, 256, 0, s>>>(T, img, N);
  return cudaGetLastError();
}

cudaError_t launch_dense_small(const DenseArgs& a, int grid, cudaStream_t stream) {
  if (a.N <= 32)
    dense_small_kernel<32, 64><<<grid, 128, dense_small_smem(a.N), stream>>>(a);
  else
    dense_small_kernel<64, 32><<<grid, 128, dense_small_smem(a.N), stream>>>(a);
  return cudaGetLastError();
}

int64_t dense_small_tiles(int N, int64_t ncols) {
  const int bn = N <= 32 ? 64 : 32;
  return (ncols + bn - 1) / bn;
}

const void* dense_kernel_func() { return (const void*)dense_pass_kernel; }

cudaError_t launch_dense(const DenseArgs& a, int grid, cudaStream_t stream) {
  dense_pass_kernel<<<grid, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

int64_t dense_tiles(int N, int64_t ncols) { return dense_tile_count(N, ncols); }

}  // namespace ffx

namespace ffx {

namespace {

// O[b][nb] = (T e_b)[nb] (the map applied to the unit vectors) -> T[nb][b] = O[b][nb]
// and T^H[b][nb] = conj(T[nb][b]) = conj(O[b][nb]).
__global__ void dense_build_kernel(const float2* __restrict__ O, float2* __restrict__ T,
                                   float2* __restrict__ TH, int N) {
  const int64_t total = (int64_t)N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx / N, nb = idx - b * N;
    const float2 o = O[idx];
    T[nb * N + b] = o;
    TH[idx] = make_float2(o.x, -o.y);
  }
}

__global__ void identity_kernel(float2* __restrict__ I, int N) {
  const int64_t total = (int64_t)N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx / N, n = idx - b * N;
    I[idx] = make_float2(b == n ? 1.f : 0.f, 0.f);
  }
}

}  // namespace

cudaError_t launch_identity(float2* I, int N, cudaStream_t s) {
  const int64_t total = (int64_t)N * N;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  identity_kernel<<<blocks, 256, 0, s>>>(I, N);
  return cudaGetLastError();
}

cudaError_t launch_dense_build(const float2* O, float2* T, float2* TH, int N, cudaStream_t s) {
  const int64_t total = (int64_t)N * N;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  dense_build_kernel<<<blocks, 256, 0, s>>>(O, T, TH, N);
  return cudaGetLastError();
}

}  // namespace ffx
