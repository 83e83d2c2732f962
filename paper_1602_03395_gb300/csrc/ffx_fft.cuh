// Line FFTs held in registers and exchanged through shared memory.
//
// A line of N complex points is transformed by T = N/E threads, each holding
// E points.  Thread t "owns" the positions t + e*T, e = 0..E-1.  The transform
// is a mixed-radix Stockham sequence (radices R_0 ... R_{S-1}, product N):
// stage s with span Ns (product of the earlier radices) runs N/R_s butterflies
// j = 0..N/R_s-1; butterfly j reads the points j + r*N/R_s, multiplies point
// r by W_N^{r (j mod Ns) N/(Ns R_s)}, applies a radix-R_s DFT and writes
// its outputs to (j div Ns)*Ns*R_s + (j mod Ns) + r*Ns.  The output is in
// natural order.  Thread t runs the butterflies j = t + b*T, b < E/R_s; their
// inputs are its owned positions (e = b + r*E/R_s), and so are the last
// stage's outputs.  Only the stages in between go through shared memory.
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
  } else if constexpr (R == 16) {
    dft16<INV>(x);
  } else {
    static_assert(R == 2, "unsupported radix");
  }
}

// ---- line plans ---------------------------------------------------------------

template <int N_, int E_, int R0, int R1 = 1, int R2 = 1, int R3 = 1, int R4 = 1>
struct LinePlan {
  static constexpr int N = N_;
  static constexpr int E = E_;
  static constexpr int T = N_ / E_;
  static constexpr int S = (R1 > 1) + (R2 > 1) + (R3 > 1) + (R4 > 1) + 1;
  static_assert(R0 * R1 * R2 * R3 * R4 == N_, "radices must multiply to N");
  static_assert(E_ % R0 == 0 && E_ % R1 == 0 && E_ % R2 == 0 && E_ % R3 == 0 && E_ % R4 == 0,
                "each radix must divide E");
  static_assert(N_ % E_ == 0, "E must divide N");
  static __host__ __device__ constexpr int radix(int s) {
    return s == 0 ? R0 : s == 1 ? R1 : s == 2 ? R2 : s == 3 ? R3 : R4;
  }
  static __host__ __device__ constexpr int span(int s) {  // product of radices before s
    return s == 0 ? 1 : span(s - 1) * radix(s - 1);
  }
};

// Padded shared-memory index: one spare slot every 16 points spreads the
// stride-R stores of the Stockham stages over the banks.
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

// Twiddles of the last stage, which depend only on the thread: kept in
// registers when there are few of them (forward and inverse share them).
template <class P>
struct LastStageTw {
  static constexpr int STAGE = P::S - 1;
  static constexpr int R = P::radix(STAGE);
  static constexpr int NB = P::E / R;
  static constexpr int COUNT = NB * (R - 1);
  static constexpr bool enabled = (P::S > 1) && COUNT <= 8;
  float2 w[enabled ? COUNT : 1];
  __device__ __forceinline__ void load(const float2* __restrict__ tw, int t) {
    if constexpr (enabled) {
      constexpr int Ns = P::span(STAGE);
      constexpr int step = P::N / (Ns * R);
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int k = (t + b * P::T) % Ns;
#pragma unroll
        for (int r = 1; r < R; ++r) w[b * (R - 1) + r - 1] = tw[r * k * step];
      }
    }
  }
};

// One butterfly stage on the registers (inputs at owned positions).
template <class P, int STAGE, bool INV>
__device__ __forceinline__ void stage_compute(float2 (&v)[P::E], const float2* __restrict__ tw, int t,
                                              const LastStageTw<P>& twc) {
  constexpr int R = P::radix(STAGE);
  constexpr int Ns = P::span(STAGE);
  constexpr int NB = P::E / R;
  constexpr bool cached = (STAGE == P::S - 1) && LastStageTw<P>::enabled;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = v[b + r * NB];
    if constexpr (Ns > 1) {
      const int j = t + b * P::T;
      const int k = j % Ns;
      constexpr int step = P::N / (Ns * R);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w;
        if constexpr (cached) {
          w = twc.w[b * (R - 1) + r - 1];
        } else {
          w = tw[r * k * step];
        }
        if (INV) w.y = -w.y;
        x[r] = cmul(x[r], w);
      }
    }
    dft<R, INV>(x);
#pragma unroll
    for (int r = 0; r < R; ++r) v[b + r * NB] = x[r];
  }
}

// Store the outputs of stage STAGE to their Stockham positions.
template <class P, int STAGE>
__device__ __forceinline__ void stage_store(const float2 (&v)[P::E], float2* __restrict__ line, int t) {
  constexpr int R = P::radix(STAGE);
  constexpr int Ns = P::span(STAGE);
  constexpr int NB = P::E / R;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = t + b * P::T;
    const int base = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
    for (int r = 0; r < R; ++r) line[pad(base + r * Ns)] = v[b + r * NB];
  }
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

template <class P, int STAGE, bool INV>
__device__ __forceinline__ void fft_from(float2 (&v)[P::E], float2* line, const float2* tw, int t,
                                         unsigned key, const LastStageTw<P>& twc) {
  stage_compute<P, STAGE, INV>(v, tw, t, twc);
  if constexpr (STAGE + 1 < P::S) {
    line_sync<P::T>(key);  // earlier readers of `line` are done
    stage_store<P, STAGE>(v, line, t);
    line_sync<P::T>(key);
    load_owned<P>(v, line, t);
    fft_from<P, STAGE + 1, INV>(v, line, tw, t, key, twc);
  }
}

// Full line transform: v holds the input at owned positions and receives the
// output at owned positions.  `line` is this line's shared exchange buffer.
// It is written only after a line_sync, so earlier readers are safe; threads
// may still be reading it on return, so the caller line_syncs before writing
// it again.
template <class P, bool INV>
__device__ __forceinline__ void fft_line(float2 (&v)[P::E], float2* line, const float2* tw, int t,
                                         unsigned key, const LastStageTw<P>& twc) {
  fft_from<P, 0, INV>(v, line, tw, t, key, twc);
}

}  // namespace ffx
