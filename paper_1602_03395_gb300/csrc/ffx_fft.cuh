// Line FFTs held in registers, with the butterflies across threads done by
// warp shuffles.
//
// A line of N = E * T complex points is transformed by T threads, each holding
// E points: thread t owns the positions t + e T, e = 0..E-1 (natural order,
// the layout of the forward input and of the inverse output).  With
// n = t + T e and k = k_e + E k_t the DFT factorises as
//   X[k_e + E k_t] = sum_t w_T^(t k_t) [ w_N^(t k_e) sum_e w_E^(e k_e) x[t + T e] ],
// so the forward transform is
//   1. an E-point DFT over the thread's own registers (radix 4, 8, 12 or 16),
//   2. the twiddle w_N^(t k_e), read from a [k_e][t] table (conflict free),
//   3. a T-point DFT across the threads for every k_e: log2 T radix-2
//      decimation-in-frequency stages, partner t ^ d, by __shfl_xor_sync
//      within a warp and through shared memory for the stages that cross
//      warps (lines of more than 32 threads).
// Its output is in the spectral layout: thread t's register e holds frequency
// spec(t, e) = e + E * rev_T(t), rev_T the bit reversal of log2 T bits.  The
// inverse transform takes the spectral layout (decimation in time across the
// threads, the conjugate twiddles, the inverse E-point DFTs) and returns the
// natural layout, so no reordering pass is needed; callers index k-space
// tables and folds by spec(t, e).
//
// Every DFT here is unnormalised: forward sum x_n e^{-2 pi i m n / N},
// inverse sum x_m e^{+2 pi i m n / N}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ffx {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// acc + a*b
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// multiply by exp(-+ i pi/4) = (1 -+ i)/sqrt(2)
template <bool INV>
__device__ __forceinline__ float2 rot45(float2 a) {
  const float h = 0.70710678118654752f;
  return INV ? make_float2(h * (a.x - a.y), h * (a.x + a.y))
             : make_float2(h * (a.x + a.y), h * (a.y - a.x));
}
// multiply by exp(-+ 3 i pi/4) = (-1 -+ i)/sqrt(2)
template <bool INV>
__device__ __forceinline__ float2 rot135(float2 a) {
  const float h = 0.70710678118654752f;
  return INV ? make_float2(-h * (a.x + a.y), h * (a.x - a.y))
             : make_float2(h * (a.y - a.x), -h * (a.x + a.y));
}

// ---- radix-R DFTs on a local array, natural order in and out ------------------

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2* x) {
  // y1 = x0 - (x1+x2)/2 -+ i (sqrt3/2)(x1 - x2), y2 = conjugate pairing
  const float s = 0.86602540378443865f;
  float2 t1 = cadd(x[1], x[2]);
  float2 t2 = make_float2(x[0].x - 0.5f * t1.x, x[0].y - 0.5f * t1.y);
  float2 d = csub(x[1], x[2]);
  float2 t3 = rot90<INV>(make_float2(s * d.x, s * d.y));
  x[0] = cadd(x[0], t1);
  x[1] = cadd(t2, t3);
  x[2] = csub(t2, t3);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2* x) {
  float2 a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
  float2 a2 = cadd(x[1], x[3]), a3 = rot90<INV>(csub(x[1], x[3]));
  x[0] = cadd(a0, a2);
  x[2] = csub(a0, a2);
  x[1] = cadd(a1, a3);
  x[3] = csub(a1, a3);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* x) {
  float2 e[4] = {x[0], x[2], x[4], x[6]};
  float2 o[4] = {x[1], x[3], x[5], x[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  o[1] = rot45<INV>(o[1]);
  o[2] = rot90<INV>(o[2]);
  o[3] = rot135<INV>(o[3]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    x[k] = cadd(e[k], o[k]);
    x[k + 4] = csub(e[k], o[k]);
  }
}

template <bool INV>
__device__ __forceinline__ void dft16(float2* x) {
  float2 e[8], o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    e[k] = x[2 * k];
    o[k] = x[2 * k + 1];
  }
  dft8<INV>(e);
  dft8<INV>(o);
  // o[k] *= exp(-+ 2 pi i k / 16)
  const float c1 = 0.92387953251128676f, s1 = 0.38268343236508977f;
  const float sg = INV ? 1.f : -1.f;
  o[1] = cmul(o[1], make_float2(c1, sg * s1));
  o[2] = rot45<INV>(o[2]);
  o[3] = cmul(o[3], make_float2(s1, sg * c1));
  o[4] = rot90<INV>(o[4]);
  o[5] = cmul(o[5], make_float2(-s1, sg * c1));
  o[6] = rot135<INV>(o[6]);
  o[7] = cmul(o[7], make_float2(-c1, sg * s1));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    x[k] = cadd(e[k], o[k]);
    x[k + 8] = csub(e[k], o[k]);
  }
}

template <bool INV>
__device__ __forceinline__ void dft32(float2* x) {
  float2 e[16], o[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    e[k] = x[2 * k];
    o[k] = x[2 * k + 1];
  }
  dft16<INV>(e);
  dft16<INV>(o);
  // o[k] *= exp(-+ 2 pi i k / 32) = cos(pi k / 16) -+ i sin(pi k / 16)
  const float c[8] = {1.f, 0.98078528040323043f, 0.92387953251128674f, 0.83146961230254524f,
                      0.70710678118654752f, 0.55557023301960218f, 0.38268343236508978f, 0.19509032201612825f};
  const float sg = INV ? 1.f : -1.f;
#pragma unroll
  for (int k = 1; k < 16; ++k) {
    // c[j] = cos(pi j / 16), j = 0..7: cos(pi k / 16) is c[k], 0 (k = 8) or
    // -c[16 - k]; sin(pi k / 16) is c[8 - k] (k <= 8) or c[k - 8]
    const float cs = k < 8 ? c[k] : (k == 8 ? 0.f : -c[16 - k]);
    const float sn = k <= 8 ? c[8 - k] : c[k - 8];
    o[k] = cmul(o[k], make_float2(cs, sg * sn));
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    x[k] = cadd(e[k], o[k]);
    x[k + 16] = csub(e[k], o[k]);
  }
}

// 12 = 4 x 3: with n = n1 + 4 n2 and k = 3 k1 + k2,
// X[3 k1 + k2] = sum_n1 w_4^(n1 k1) w_12^(n1 k2) sum_n2 w_3^(n2 k2) x[n1 + 4 n2].
template <bool INV>
__device__ __forceinline__ void dft12(float2* x) {
  float2 y[4][3];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    float2 z[3] = {x[n1], x[n1 + 4], x[n1 + 8]};
    dft3<INV>(z);
    y[n1][0] = z[0];
    y[n1][1] = z[1];
    y[n1][2] = z[2];
  }
  // w_12^(n1 k2) for n1 = 1..3, k2 = 1..2: angles pi/6 (n1 k2 = 1), pi/3 (2),
  // pi/2 (3), 2 pi/3 (4), pi (6)
  const float c30 = 0.86602540378443865f, s30 = 0.5f;
  const float sg = INV ? 1.f : -1.f;
  y[1][1] = cmul(y[1][1], make_float2(c30, sg * s30));
  y[1][2] = cmul(y[1][2], make_float2(s30, sg * c30));
  y[2][1] = cmul(y[2][1], make_float2(s30, sg * c30));
  y[2][2] = cmul(y[2][2], make_float2(-s30, sg * c30));
  y[3][1] = rot90<INV>(y[3][1]);
  y[3][2] = make_float2(-y[3][2].x, -y[3][2].y);
#pragma unroll
  for (int k2 = 0; k2 < 3; ++k2) {
    float2 z[4] = {y[0][k2], y[1][k2], y[2][k2], y[3][k2]};
    dft4<INV>(z);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) x[3 * k1 + k2] = z[k1];
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* x) {
  if constexpr (R == 2) {
    dft2<INV>(x[0], x[1]);
  } else if constexpr (R == 3) {
    dft3<INV>(x);
  } else if constexpr (R == 4) {
    dft4<INV>(x);
  } else if constexpr (R == 8) {
    dft8<INV>(x);
  } else if constexpr (R == 12) {
    dft12<INV>(x);
  } else if constexpr (R == 16) {
    dft16<INV>(x);
  } else if constexpr (R == 32) {
    dft32<INV>(x);
  } else {
    static_assert(R == 2, "unsupported radix");
  }
}

// ---- line plans ---------------------------------------------------------------

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// N = E * T points per line, T threads per line (a power of two), E points per
// thread (4, 8, 12 or 16).
template <int N_, int E_>
struct LinePlan {
  static constexpr int N = N_;
  static constexpr int E = E_;
  static constexpr int T = N_ / E_;
  static_assert(N_ % E_ == 0 && (T & (T - 1)) == 0, "T = N / E must be a power of two");
  static_assert(E_ == 4 || E_ == 8 || E_ == 12 || E_ == 16, "E must be 4, 8, 12 or 16");
  static constexpr int LOG_T = ilog2(T);
};

// Padded shared-memory index: one spare slot every 16 points spreads
// stride-16 accesses over the banks.
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
template <int N>
struct Padded {
  static constexpr int value = N + N / 16 + 1;
};

// Synchronise the T threads of one line-group.  Groups of <= 32 threads sit
// inside a warp on consecutive lanes (T is a power of two dividing 32, blocks
// are laid out group-major) and synchronise with their own lane mask, so other
// groups of the warp may be elsewhere; longer groups use a named barrier per
// group (ids 1..15; id 0 is __syncthreads).  `key` comes from line_sync_key.
template <int T>
__device__ __forceinline__ unsigned line_sync_key(int group_in_block, int tid) {
  static_assert((T & (T - 1)) == 0, "threads per line must be a power of two");
  if constexpr (T >= 32) {
    return T == 32 ? 0xffffffffu : 1u + (unsigned)group_in_block;
  } else {
    return ((1u << T) - 1u) << ((tid & 31) & ~(T - 1));
  }
}

template <int T>
__device__ __forceinline__ void line_sync(unsigned key) {
  if constexpr (T <= 32) {
    __syncwarp(key);
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(key), "r"(T) : "memory");
  }
}

template <int T>
__device__ __forceinline__ int bitrev(int t) {
  if constexpr (T <= 1) {
    return 0;
  } else {
    return (int)(__brev((unsigned)t) >> (32 - ilog2(T)));
  }
}

// Frequency held by thread t's register e after a forward transform (and
// expected there by an inverse one).
template <class P>
__device__ __forceinline__ int spec_index(int t, int e) {
  return e + P::E * bitrev<P::T>(t);
}

// Per-thread constants of a line transform: the shuffle mask of the thread's
// line-group, and the cross-thread stage twiddles w_(2d)^j = e^{-i pi j / d},
// j < d, of every distance d = 1, 2, .., T/2 in a block-shared table at
// d + j (forward sign; the inverse takes their conjugates).
template <class P>
struct LineFftCtx {
  const float2* stw;
  unsigned mask;
  __device__ __forceinline__ void init(const float2* stage_tw, unsigned key) {
    stw = stage_tw;
    mask = P::T >= 32 ? 0xffffffffu : key;
  }
};

// Twiddle tables of a line transform, filled by a whole block (NT threads):
// tw2[k_e * T + t] = w_N^(t k_e) (the step between the local and the
// cross-thread DFTs, from the length-N table tw[i] = w_N^i), and the stage
// table stw[d + j] = w_(2d)^j (T entries; entry 0 unused).
template <class P>
__device__ __forceinline__ void fill_line_twiddles(float2* tw2, float2* stw, const float2* __restrict__ tw, int tid,
                                                   int NT) {
  for (int i = tid; i < P::N; i += NT) {
    const int ke = i / P::T, t = i - ke * P::T;
    tw2[i] = tw[(t * ke) % P::N];
  }
  for (int i = tid; i < P::T; i += NT) {
    const int d = i > 0 ? 1 << (31 - __clz(i)) : 1;  // the power of two below or at i
    float sn, cs;
    sincospif((float)(i - d) / (float)d, &sn, &cs);
    stw[i] = make_float2(cs, -sn);
  }
}

// One radix-2 stage across threads at distance d (a power of two below T),
// partner p = the value of thread t ^ d, w = w_(2d)^(t mod d):
//  DIF (forward): bit clear: v + p; bit set: (p - v) w, i.e. (s v + p) w'
//                 with s = -+1, w' = w or 1;
//  DIT (inverse): bit clear: v + w* p; bit set: p - w* v, i.e. A v + B p
//                 with (A, B) = (1, w*) or (-w*, 1).
template <class P, bool INV>
__device__ __forceinline__ void cross_stage(float2 (&v)[P::E], int t, int s, const LineFftCtx<P>& c, float2* line,
                                            unsigned key) {
  const int d = 1 << s;
  const bool up = (t & d) != 0;
  float2 w = c.stw[d + (t & (d - 1))];
  if (INV) w.y = -w.y;
  const float sg = up ? -1.f : 1.f;
  const float2 wp = up ? w : make_float2(1.f, 0.f);                         // DIF
  const float2 A = up ? make_float2(-w.x, -w.y) : make_float2(1.f, 0.f);    // DIT
  const float2 B = up ? make_float2(1.f, 0.f) : w;
  auto combine = [&](float2 x, float2 p) -> float2 {
    if (!INV) return cmul(make_float2(fmaf(sg, x.x, p.x), fmaf(sg, x.y, p.y)), wp);
    return cfma(B, p, cmul(A, x));
  };
  if (d < 32) {
#pragma unroll
    for (int e = 0; e < P::E; ++e) {
      float2 p;
      p.x = __shfl_xor_sync(c.mask, v[e].x, d);
      p.y = __shfl_xor_sync(c.mask, v[e].y, d);
      v[e] = combine(v[e], p);
    }
  } else {
    // partner in another warp: through the line's exchange buffer, thread t's
    // register e at e * T + t (consecutive threads, consecutive slots)
    line_sync<P::T>(key);  // earlier readers of `line` are done
#pragma unroll
    for (int e = 0; e < P::E; ++e) line[pad(e * P::T + t)] = v[e];
    line_sync<P::T>(key);
#pragma unroll
    for (int e = 0; e < P::E; ++e) v[e] = combine(v[e], line[pad(e * P::T + (t ^ d))]);
  }
}

// Forward line transform: natural layout in, spectral layout out.  `line` is
// the line's exchange buffer (used only by lines of more than 32 threads);
// tw2 is the step-twiddle table (fill_step_twiddles).  Threads may still read
// `line` on return: callers line_sync before writing it again.
template <class P>
__device__ __forceinline__ void fft_fwd(float2 (&v)[P::E], float2* line, const float2* tw2, int t, unsigned key,
                                        const LineFftCtx<P>& c) {
  dft<P::E, false>(v);
#pragma unroll
  for (int e = 1; e < P::E; ++e) v[e] = cmul(v[e], tw2[e * P::T + t]);
#pragma unroll
  for (int s = P::LOG_T - 1; s >= 0; --s) cross_stage<P, false>(v, t, s, c, line, key);
}

// Inverse line transform: spectral layout in, natural layout out.
template <class P>
__device__ __forceinline__ void fft_inv(float2 (&v)[P::E], float2* line, const float2* tw2, int t, unsigned key,
                                        const LineFftCtx<P>& c) {
#pragma unroll
  for (int s = 0; s < P::LOG_T; ++s) cross_stage<P, true>(v, t, s, c, line, key);
#pragma unroll
  for (int e = 1; e < P::E; ++e) v[e] = cmulc(v[e], tw2[e * P::T + t]);
  dft<P::E, true>(v);
}

template <class P>
__device__ __forceinline__ void load_owned(float2 (&v)[P::E], const float2* __restrict__ line, int t) {
#pragma unroll
  for (int e = 0; e < P::E; ++e) v[e] = line[pad(t + e * P::T)];
}

template <class P>
__device__ __forceinline__ void store_owned(const float2 (&v)[P::E], float2* __restrict__ line, int t) {
#pragma unroll
  for (int e = 0; e < P::E; ++e) line[pad(t + e * P::T)] = v[e];
}

// A spectral-layout line into natural order in shared memory.
template <class P>
__device__ __forceinline__ void store_spectral(const float2 (&v)[P::E], float2* __restrict__ line, int t) {
  const int base = P::E * bitrev<P::T>(t);
#pragma unroll
  for (int e = 0; e < P::E; ++e) line[pad(base + e)] = v[e];
}

}  // namespace ffx
