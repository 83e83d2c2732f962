// FFT-form passes at magnification lam = 1 on lines of N = R^2 points
// (R = 4, 8, 16): the per-axis map is then a single term (q = 0, whose
// pre-chirp is 1), a convolution
//   fold form (eq. FFaux with the presf factor folded in):  out = IFFT(Kf_0 . FFT(psi))
//   paper form (eqs. presA, presB, presf):                  out = F_0 . IFFT(K_0 . FFT(psi))
//   adjoint of the fold form:                               out = IFFT(conj(Kf_0) . FFT(g))
// with unnormalised DFTs (the tables carry the scale).  Each line is
// transformed by R threads holding R points each, in registers:
//
//   with n = t + R e (thread t, register e) and k = k1 + R k2,
//   X[k1 + R k2] = sum_t w_R^(t k2) w_N^(t k1) sum_e w_R^(e k1) x[t + R e],
//
// so a transform is an R-point DFT over the thread's own registers, the
// twiddle w_N^(t k1), a transpose through the line's shared-memory block
// (row k1, column t; padded rows, conflict free) and a second R-point DFT
// over the registers: thread t then holds X[t + R e] -- the same layout
// as its input, so the inverse transform takes the product as it is and
// returns the natural order.  The thread's twiddles and K or Kf entries (at
// t + R e) sit in registers (R <= 8) or in shared memory (R = 16) for the
// whole launch.  Lines move between HBM and registers
// directly: along a contiguous line the R threads of a line read consecutive
// points (line-major lanes, warp barriers); across strided lines neighbouring
// threads take neighbouring lines of the tile (the block's barriers around
// the transposes), so a warp reads 16 or more lines' neighbouring points at a
// time.  Loads of the next tile are issued before the current tile is
// transformed.
#include "ffx_fft.cuh"
#include "ffx_internal.h"

namespace ffx {

namespace {

constexpr int kConvThreads = 256;

// A thread's place: line slot l of the block's tile, thread t of the line.
// Contiguous lines: a line's R threads are neighbours in a warp (its points
// are neighbours in memory).  Strided lines: neighbouring threads take
// neighbouring lines of the tile (their points are neighbours in memory), so
// a line's threads spread over the block.
template <int R, bool CONTIG>
__device__ __forceinline__ void conv_place(int tid, int& l, int& t) {
  constexpr int LB = kConvThreads / R;
  if (CONTIG) {
    l = tid / R;
    t = tid - l * R;
  } else {
    t = tid / LB;
    l = tid - t * LB;
  }
}

// Shared-memory block of one line: R rows of R + 1 points; with strided
// lines (a half-warp's 16 lanes are 16 lines at the same offset) an odd line
// stride keeps them on distinct banks.
template <int R, bool CONTIG>
struct ConvLayout {
  static constexpr int RS = R + 1;
  static constexpr int LS = R * RS + (CONTIG ? 0 : 1);
  static constexpr int LB = kConvThreads / R;  // lines per tile
  static constexpr bool REG = R <= 8;          // per-thread tables in registers
  // [line blocks][twiddles w_N^(t e) as [e][t]][K as [e][t]][F as [e][t]]
  static constexpr size_t tab_off = sizeof(float2) * LB * LS;
  static constexpr size_t bytes = tab_off + (REG ? 0 : 3 * sizeof(float2) * R * R);
};

// Every thread of the line (contiguous lines: one warp; strided: the block).
template <bool CONTIG>
__device__ __forceinline__ void line_barrier() {
  if (CONTIG)
    __syncwarp();
  else
    __syncthreads();
}

// One line transform (forward or inverse) on the thread's registers.
template <int R, bool INV, bool CONTIG>
__device__ __forceinline__ void conv_fft(float2 (&v)[R], const float2 (&tw)[R], float2* xl, int t) {
  constexpr int RS = R + 1;
  dft<R, INV>(v);
#pragma unroll
  for (int e = 1; e < R; ++e) v[e] = INV ? cmulc(v[e], tw[e]) : cmul(v[e], tw[e]);
  line_barrier<CONTIG>();  // the line's earlier readers of its block are done
#pragma unroll
  for (int e = 0; e < R; ++e) xl[e * RS + t] = v[e];
  line_barrier<CONTIG>();
#pragma unroll
  for (int e = 0; e < R; ++e) v[e] = xl[t * RS + e];
  dft<R, INV>(v);
}

template <int R, bool CONTIG>
__global__ void __launch_bounds__(kConvThreads, 2) conv_kernel(const PassArgs a, const int kind) {
  using L = ConvLayout<R, CONTIG>;
  constexpr int N = R * R, LB = L::LB;
  extern __shared__ __align__(16) unsigned char csm[];
  float2* const blocks = reinterpret_cast<float2*>(csm);
  float2* const tabs = reinterpret_cast<float2*>(csm + L::tab_off);
  const int tid = threadIdx.x;
  int l, t;
  conv_place<R, CONTIG>(tid, l, t);
  float2* const xl = blocks + l * L::LS;

  // the spectral table of the kind (K_0 for the paper form, Kf_0 otherwise;
  // conjugated for the adjoint), and the paper form's post-chirp F_0
  const float2* __restrict__ ktab = kind == KIND_FWD_PAPER ? a.tab.K : a.tab.Kf;
  const bool conj_k = kind == KIND_ADJ_FOLD, post = kind == KIND_FWD_PAPER;
  float2 tw[R], kk[R];
  if constexpr (L::REG) {
#pragma unroll
    for (int e = 0; e < R; ++e) {
      tw[e] = __ldg(a.tab.tw + (t * e) % N);
      kk[e] = __ldg(ktab + t + R * e);
      if (conj_k) kk[e].y = -kk[e].y;
    }
  } else {
    for (int i = tid; i < N; i += kConvThreads) {
      const int e = i / R, tt = i - e * R;
      tabs[i] = __ldg(a.tab.tw + (tt * e) % N);
      float2 k = __ldg(ktab + tt + R * e);
      if (conj_k) k.y = -k.y;
      tabs[N + i] = k;
      tabs[2 * N + i] = post ? __ldg(a.tab.F + tt + R * e) : make_float2(1.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < R; ++e) tw[e] = tabs[e * R + t];
  }

  const int64_t inner = a.inner;
  const int64_t per_real = a.outer * inner;
  const int64_t ntiles = (a.nlines + LB - 1) / LB;
  // line c's first point, or -1 past the end
  auto line_base = [&](int64_t c) -> long long {
    if (c >= a.nlines) return -1;
    const int64_t bo = c / inner;
    return bo * (int64_t)N * inner + (c - bo * inner);
  };
  auto load = [&](long long base, float2 (&v)[R]) {
#pragma unroll
    for (int e = 0; e < R; ++e)
      v[e] = base >= 0 ? __ldcs(a.in + base + (int64_t)(t + R * e) * inner) : make_float2(0.f, 0.f);
  };

  int64_t tile = blockIdx.x;
  long long base = line_base(tile * LB + l);
  float2 v[R];
  load(base, v);
  for (; tile < ntiles; tile += gridDim.x) {
    // the next tile's loads go out before this one is transformed
    const int64_t next = tile + gridDim.x;
    const long long nbase = next < ntiles ? line_base(next * LB + l) : -1;
    float2 nv[R];
    load(nbase, nv);
    if (a.grad && base >= 0) {
      // backward passes: the input element is 2 grad * psi
      const int64_t c = tile * LB + l;
      const int64_t goff = a.grad_shared ? base - (c / per_real) * a.M : base;
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const float gr = 2.f * __ldg(a.grad + goff + (int64_t)(t + R * e) * inner);
        v[e] = make_float2(v[e].x * gr, v[e].y * gr);
      }
    }
    conv_fft<R, false, CONTIG>(v, tw, xl, t);
#pragma unroll
    for (int e = 0; e < R; ++e) v[e] = cmul(v[e], L::REG ? kk[e] : tabs[N + e * R + t]);
    conv_fft<R, true, CONTIG>(v, tw, xl, t);
    if (post) {
#pragma unroll
      for (int e = 0; e < R; ++e) v[e] = cmul(v[e], L::REG ? __ldg(a.tab.F + t + R * e) : tabs[2 * N + e * R + t]);
    }
    if (base >= 0) {
      if (a.out_c) {
#pragma unroll
        for (int e = 0; e < R; ++e) __stcs(a.out_c + base + (int64_t)(t + R * e) * inner, v[e]);
      } else {
#pragma unroll
        for (int e = 0; e < R; ++e)
          __stcs(a.out_d + base + (int64_t)(t + R * e) * inner, v[e].x * v[e].x + v[e].y * v[e].y);
      }
    }
    base = nbase;
#pragma unroll
    for (int e = 0; e < R; ++e) v[e] = nv[e];
  }
}

template <int R, bool CONTIG>
cudaError_t launch_conv_r(const PassArgs& a, int kind, int sms, cudaStream_t s) {
  using L = ConvLayout<R, CONTIG>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(conv_kernel<R, CONTIG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L::bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_kernel<R, CONTIG>, kConvThreads, L::bytes) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int64_t ntiles = (a.nlines + L::LB - 1) / L::LB;
  int64_t grid = (int64_t)per_sm * sms;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  conv_kernel<R, CONTIG><<<(int)grid, kConvThreads, L::bytes, s>>>(a, kind);
  return cudaGetLastError();
}

}  // namespace

bool conv_supported(int N, int lam, int acc) { return lam == 1 && !acc && (N == 16 || N == 64 || N == 256); }

cudaError_t launch_conv(const PassArgs& a, int kind, int N, int sms, cudaStream_t s) {
  const bool contig = a.inner == 1;
  switch (N) {
    case 16: return contig ? launch_conv_r<4, true>(a, kind, sms, s) : launch_conv_r<4, false>(a, kind, sms, s);
    case 64: return contig ? launch_conv_r<8, true>(a, kind, sms, s) : launch_conv_r<8, false>(a, kind, sms, s);
    case 256: return contig ? launch_conv_r<16, true>(a, kind, sms, s) : launch_conv_r<16, false>(a, kind, sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ffx
