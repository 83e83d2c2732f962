// FFT-form passes with one or two terms, on lines of N = R^2 points
// (R = 4, 8, 16, 32).  At magnification lam = 1 the per-axis map is a single
// term (q = 0, whose pre-chirp is 1), a convolution:
//   fold form (eq. FFaux with the presf factor folded in):  out = IFFT(Kf_0 . FFT(psi))
//   paper form (eqs. presA, presB, presf):                  out = F_0 . IFFT(K_0 . FFT(psi))
//   adjoint of the fold form:                               out = IFFT(conj(Kf_0) . FFT(g))
// At lam = 2 the fold form sums two terms into one spectrum before its
// inverse transform:
//   D[(2 m + q) mod N] += Kf_q[m] . FFT(P_q . psi)[m],  q = 0, 1;  out = IFFT(D).
// DFTs are unnormalised (the tables carry the scale).  Each line is
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
// returns the natural order.  For lam = 2 the two frequencies that fold onto
// one point, m and m + N/2, are registers e and e + R/2 of the same thread:
// their sum goes to the line's block at 2 m + q, and every thread then reads
// its spectrum D[t + R e] back.  Per-thread twiddles and table entries sit in
// registers (lam = 1, R <= 8; twiddles also for R = 16) or in shared memory.
// Lines move between HBM and registers directly: along a contiguous line the
// R threads of a line read consecutive points (line-major lanes, warp
// barriers); across strided lines neighbouring threads take neighbouring
// lines of the tile (the block's barriers around the exchanges), so a warp
// reads 8 or more lines' neighbouring points at a time.  Where the registers
// allow it (lam = 1 and R <= 16, lam = 2 and R <= 8) the loads of the next
// tile are issued before the current tile is transformed.
#include "ffx_fft.cuh"
#include "ffx_internal.h"

namespace ffx {

namespace {

constexpr int kConvThreads = 256;

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int R, bool CONTIG, int LAM>
struct ConvCfg {
  static constexpr int N = R * R;
  static constexpr int RS = R + 1;
  static constexpr int LB = kConvThreads / R;  // lines per tile
  // a line's block: the transposes' R rows of R + 1, and for lam = 2 the
  // folded spectrum at pad(j); odd for strided lines (16 lines at one offset
  // then fall on distinct banks)
  static constexpr int LS0 = cmax(R * RS, LAM == 2 ? N + (N - 1) / 16 + 1 : 0);
  static constexpr int LS = CONTIG ? LS0 : (LS0 | 1);
  static constexpr bool TWREG = R <= 16;               // twiddles in registers
  static constexpr bool TABREG = LAM == 1 && R <= 8;   // K (or Kf) in registers
  static constexpr bool PREFETCH = (LAM == 1 && R <= 16) || (LAM == 2 && R <= 8);
  // shared tables, each [e][t] (entry t + R e of the natural-order row):
  // twiddles w_N^(t e), K_0 or Kf_0, F_0 (paper form) or Kf_1 (lam = 2), P_1
  static constexpr int NTAB = 4;
  static constexpr size_t tab_off = sizeof(float2) * LB * LS;
  static constexpr size_t bytes = tab_off + (TABREG ? 0 : NTAB * sizeof(float2) * N);
};

// A thread's place: line slot l of the block's tile, thread t of the line.
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

// Every thread of the line (contiguous lines: one warp; strided: the block).
template <bool CONTIG>
__device__ __forceinline__ void line_barrier() {
  if (CONTIG)
    __syncwarp();
  else
    __syncthreads();
}

// One line transform (forward or inverse) on the thread's registers; the
// twiddles from registers (tw) or from the shared table (tws, [e][t]).
template <int R, bool INV, bool CONTIG, bool TWREG>
__device__ __forceinline__ void conv_fft(float2 (&v)[R], const float2 (&tw)[R], const float2* tws, float2* xl,
                                         int t) {
  constexpr int RS = R + 1;
  dft<R, INV>(v);
#pragma unroll
  for (int e = 1; e < R; ++e) {
    const float2 w = TWREG ? tw[e] : tws[e * R + t];
    v[e] = INV ? cmulc(v[e], w) : cmul(v[e], w);
  }
  line_barrier<CONTIG>();  // the line's earlier readers of its block are done
#pragma unroll
  for (int e = 0; e < R; ++e) xl[e * RS + t] = v[e];
  line_barrier<CONTIG>();
#pragma unroll
  for (int e = 0; e < R; ++e) v[e] = xl[t * RS + e];
  dft<R, INV>(v);
}

// two blocks per SM, one for the two 32-point spectra of lam = 2 (their registers)
template <int R, bool CONTIG, int LAM>
__global__ void __launch_bounds__(kConvThreads, (R == 32 && LAM == 2) ? 1 : 2)
    conv_kernel(const PassArgs a, const int kind) {
  using C = ConvCfg<R, CONTIG, LAM>;
  constexpr int N = C::N, LB = C::LB;
  extern __shared__ __align__(16) unsigned char csm[];
  float2* const blocks = reinterpret_cast<float2*>(csm);
  float2* const tabs = reinterpret_cast<float2*>(csm + C::tab_off);
  const float2* const tw_s = tabs;
  const float2* const k0_s = tabs + N;
  const float2* const t2_s = tabs + 2 * N;  // F_0 (paper form) or Kf_1 (lam = 2)
  const float2* const p1_s = tabs + 3 * N;
  const int tid = threadIdx.x;
  int l, t;
  conv_place<R, CONTIG>(tid, l, t);
  float2* const xl = blocks + l * C::LS;

  // K_0 for the paper form, Kf_0 otherwise (conjugated for the adjoint); the
  // paper form's post-chirp F_0; lam = 2: Kf_1 and the pre-chirp P_1
  const float2* __restrict__ ktab = kind == KIND_FWD_PAPER ? a.tab.K : a.tab.Kf;
  const bool conj_k = kind == KIND_ADJ_FOLD, post = kind == KIND_FWD_PAPER;
  float2 tw[R], kk[R];
  if constexpr (C::TABREG) {
#pragma unroll
    for (int e = 0; e < R; ++e) {
      tw[e] = __ldg(a.tab.tw + (t * e) % N);
      kk[e] = __ldg(ktab + t + R * e);
      if (conj_k) kk[e].y = -kk[e].y;
    }
  } else {
    for (int i = tid; i < N; i += kConvThreads) {
      const int e = i / R, tt = i - e * R, n = tt + R * e;
      tabs[i] = __ldg(a.tab.tw + (tt * e) % N);
      float2 k = __ldg(ktab + n);
      if (conj_k) k.y = -k.y;
      tabs[N + i] = k;
      if (LAM == 2) {
        tabs[2 * N + i] = __ldg(a.tab.Kf + N + n);
        tabs[3 * N + i] = __ldg(a.tab.P + N + n);
      } else {
        tabs[2 * N + i] = post ? __ldg(a.tab.F + n) : make_float2(1.f, 0.f);
      }
    }
    __syncthreads();
    if constexpr (C::TWREG) {
#pragma unroll
      for (int e = 0; e < R; ++e) tw[e] = tw_s[e * R + t];
    }
  }

  const int64_t inner = CONTIG ? 1 : a.inner;  // contiguous lines: the stride is 1
  const int64_t per_real = a.outer * inner;
  // offset of the thread's register e from its line's first point
  auto off = [&](int e) -> int64_t { return CONTIG ? (int64_t)(t + R * e) : (int64_t)(t + R * e) * inner; };
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
      v[e] = base >= 0 ? __ldcs(a.in + base + off(e)) : make_float2(0.f, 0.f);
  };

  int64_t tile = blockIdx.x;
  long long base = line_base(tile * LB + l);
  float2 v[R];
  if constexpr (C::PREFETCH) load(base, v);
  for (; tile < ntiles; tile += gridDim.x) {
    const int64_t next = tile + gridDim.x;
    long long nbase = -1;
    float2 nv[C::PREFETCH ? R : 1];
    if constexpr (C::PREFETCH) {
      // the next tile's loads go out before this one is transformed
      nbase = next < ntiles ? line_base(next * LB + l) : -1;
      load(nbase, nv);
    } else {
      load(base, v);
    }
    if (a.grad && base >= 0) {
      // backward passes: the input element is 2 grad * psi
      const int64_t c = tile * LB + l;
      const int64_t goff = a.grad_shared ? base - (c / per_real) * a.M : base;
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const float gr = 2.f * __ldg(a.grad + goff + off(e));
        v[e] = make_float2(v[e].x * gr, v[e].y * gr);
      }
    }
    if constexpr (LAM == 1) {
      conv_fft<R, false, CONTIG, C::TWREG>(v, tw, tw_s, xl, t);
#pragma unroll
      for (int e = 0; e < R; ++e) v[e] = cmul(v[e], C::TABREG ? kk[e] : k0_s[e * R + t]);
    } else {
      // the q = 1 term's input (pre-chirp P_1); both spectra; the fold
      float2 u[R];
#pragma unroll
      for (int e = 0; e < R; ++e) u[e] = cmul(v[e], p1_s[e * R + t]);
      conv_fft<R, false, CONTIG, C::TWREG>(v, tw, tw_s, xl, t);
      conv_fft<R, false, CONTIG, C::TWREG>(u, tw, tw_s, xl, t);
      line_barrier<CONTIG>();  // the line's block is free again
#pragma unroll
      for (int e = 0; e < R / 2; ++e) {
        const int j = 2 * (t + R * e);  // 2 m for m = t + R e < N / 2; m + N / 2 is register e + R / 2
        xl[pad(j)] = cadd(cmul(v[e], k0_s[e * R + t]), cmul(v[e + R / 2], k0_s[(e + R / 2) * R + t]));
        xl[pad(j + 1)] = cadd(cmul(u[e], t2_s[e * R + t]), cmul(u[e + R / 2], t2_s[(e + R / 2) * R + t]));
      }
      line_barrier<CONTIG>();
#pragma unroll
      for (int e = 0; e < R; ++e) v[e] = xl[pad(t + R * e)];
    }
    conv_fft<R, true, CONTIG, C::TWREG>(v, tw, tw_s, xl, t);
    if (LAM == 1 && post) {
#pragma unroll
      for (int e = 0; e < R; ++e) v[e] = cmul(v[e], C::TABREG ? __ldg(a.tab.F + t + R * e) : t2_s[e * R + t]);
    }
    if (base >= 0) {
      if (a.out_c) {
#pragma unroll
        for (int e = 0; e < R; ++e) __stcs(a.out_c + base + off(e), v[e]);
      } else {
#pragma unroll
        for (int e = 0; e < R; ++e)
          __stcs(a.out_d + base + off(e), v[e].x * v[e].x + v[e].y * v[e].y);
      }
    }
    if constexpr (C::PREFETCH) {
      base = nbase;
#pragma unroll
      for (int e = 0; e < R; ++e) v[e] = nv[e];
    } else {
      base = next < ntiles ? line_base(next * LB + l) : -1;
    }
  }
}

template <int R, bool CONTIG, int LAM>
cudaError_t launch_conv_r(const PassArgs& a, int kind, int sms, cudaStream_t s) {
  using C = ConvCfg<R, CONTIG, LAM>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(conv_kernel<R, CONTIG, LAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_kernel<R, CONTIG, LAM>, kConvThreads, C::bytes) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int64_t ntiles = (a.nlines + C::LB - 1) / C::LB;
  int64_t grid = (int64_t)per_sm * sms;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  conv_kernel<R, CONTIG, LAM><<<(int)grid, kConvThreads, C::bytes, s>>>(a, kind);
  return cudaGetLastError();
}

template <int R, int LAM>
cudaError_t launch_conv_c(const PassArgs& a, int kind, int sms, cudaStream_t s) {
  return a.inner == 1 ? launch_conv_r<R, true, LAM>(a, kind, sms, s) : launch_conv_r<R, false, LAM>(a, kind, sms, s);
}

}  // namespace

bool conv_supported(int N, int lam, int acc, int kind) {
  if (acc || !(N == 16 || N == 64 || N == 256 || N == 1024)) return false;
  return lam == 1 || (lam == 2 && kind == KIND_FWD_FOLD);
}

cudaError_t launch_conv(const PassArgs& a, int kind, int N, int sms, cudaStream_t s) {
  if (a.lam == 2) {
    switch (N) {
      case 16: return launch_conv_c<4, 2>(a, kind, sms, s);
      case 64: return launch_conv_c<8, 2>(a, kind, sms, s);
      case 256: return launch_conv_c<16, 2>(a, kind, sms, s);
      case 1024: return launch_conv_c<32, 2>(a, kind, sms, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (N) {
    case 16: return launch_conv_c<4, 1>(a, kind, sms, s);
    case 64: return launch_conv_c<8, 1>(a, kind, sms, s);
    case 256: return launch_conv_c<16, 1>(a, kind, sms, s);
    case 1024: return launch_conv_c<32, 1>(a, kind, sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ffx
