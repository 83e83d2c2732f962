// One pass of the per-axis free-flight map (eq. FF restricted to one axis),
// or of its adjoint, over every line of a [B][outer][N][inner] complex64 array.
//
// A block holds G line-groups of T = N/E threads.  qg groups share one line
// and split its sum over the fine momentum index q (group r takes
// q = r, r + qg, ...; the paper notes the terms are independent, Sec. 7.1),
// so a tile is G/qg lines.  The tile is loaded into shared memory with
// coalesced accesses; each group transforms its line in registers (see
// ffx_fft.cuh); the groups' partial sums are added in shared memory in group
// order (deterministic); the result is staged back through shared memory and
// stored coalesced: complex64, or |.|^2 as float32, or |.|^2 summed over the
// realizations of the batch (tiles then loop over b in order, so the sum is
// deterministic and needs no atomics).
//
// Kinds:
//  FWD_PAPER: acc += F_q * IFFT(K_q * FFT(P_q * psi))[(lam nb) mod N]
//             -- eqs. presA, presB, presf, FFaux and the term sum FFpsi.
//  FWD_FOLD : D[(lam m + q) mod N] += Kf_q[m] * FFT(P_q * psi)[m]; out = IFFT(D)
//             -- the same sum with the presf factor's n-dependence merged into
//             the inverse-DFT kernel (one inverse FFT per line).
//  ADJ_FOLD : the adjoint of FWD_FOLD: D = FFT(g); out = sum_q conj(P_q) *
//             IFFT(conj(Kf_q[m]) * D[(lam m + q) mod N]).
#pragma once

#include <stdint.h>

#include "ffx_fft.cuh"
#include "ffx_internal.h"

#ifndef FFX_PASS_MIN_BLOCKS
#define FFX_PASS_MIN_BLOCKS 3  // resident 256-thread blocks per SM the register budget aims for
#endif

namespace ffx {

template <class P, int G>
struct PassSmem {
  static constexpr int NP = Padded<P::N>::value;
  static constexpr size_t tw_off = 0;
  static constexpr size_t fold_off = tw_off + sizeof(float2) * P::N;
  static constexpr size_t base_off = (fold_off + sizeof(int) * P::N + 15) & ~size_t(15);
  static constexpr size_t b_off = base_off + sizeof(long long) * G;
  static constexpr size_t psi_off = (b_off + sizeof(int) * G + 15) & ~size_t(15);
  static constexpr size_t work_off = psi_off + sizeof(float2) * G * NP;
  static constexpr size_t bytes = work_off + sizeof(float2) * G * NP;
};

// Element idx of a tile copy -> (line l, point n): along n for contiguous
// lines, along the line index for strided ones (neighbouring lines are
// neighbours in memory), so either way the copy is coalesced.
__device__ __forceinline__ void tile_coords(int idx, int N, int lines, bool contiguous, int& l, int& n) {
  if (contiguous) {
    l = idx / N;
    n = idx - l * N;
  } else {
    n = idx / lines;
    l = idx - n * lines;
  }
}

// Tiles first, first + step, ... (below min(last, number of tiles)) of one
// pass.  Called by a whole block; uses `smem` (PassSmem<P, G>::bytes).
template <class P, int KIND, int G>
__device__ __forceinline__ void pass_tiles(const PassArgs& a, int64_t first, int64_t last, int64_t step,
                                           unsigned char* smem) {
  constexpr int N = P::N, E = P::E, T = P::T;
  using SM = PassSmem<P, G>;
  constexpr int NP = SM::NP;
  float2* tw_s = reinterpret_cast<float2*>(smem + SM::tw_off);
  int* fold_s = reinterpret_cast<int*>(smem + SM::fold_off);
  long long* base_s = reinterpret_cast<long long*>(smem + SM::base_off);
  int* b_s = reinterpret_cast<int*>(smem + SM::b_off);
  float2* psi_s = reinterpret_cast<float2*>(smem + SM::psi_off);
  float2* work_s = reinterpret_cast<float2*>(smem + SM::work_off);

  if (a.acc && a.batch <= 0) return;  // nothing to sum (the host never launches this)
  const int QG = a.qg > 1 ? a.qg : 1;
  const int LINES = G / QG;
  const int NT = LINES * QG * T;  // == blockDim.x
  const int tid = threadIdx.x;
  // Line-groups are laid out group-major: the groups in one warp work on the
  // same q (different lines) and read the same phase-row segments.  Group r of
  // line l has index r * LINES + l; group 0 of line l is index l.
  const int lg = tid / T;
  const int t = tid - lg * T;
  const int grp = lg / LINES;
  const int line = lg - grp * LINES;
  const unsigned key = line_sync_key<T>(lg, tid);

  __syncthreads();  // an earlier call on this block may still read shared memory
  for (int i = tid; i < N; i += NT) {
    tw_s[i] = a.tab.tw[i];
    if constexpr (KIND == KIND_FWD_FOLD) fold_s[i] = a.tab.fold[i];
  }

  __syncthreads();  // twiddles are in shared memory
  LastStageTw<P> twc;
  twc.load(tw_s, t);

  const int lam = a.lam;
  const int64_t inner = a.inner;
  const bool contiguous = (inner == 1);
  const int64_t per_real_lines = a.outer * inner;
  int64_t ntiles = (a.nlines + LINES - 1) / LINES;
  if (last < ntiles) ntiles = last;
  const int nb_loop = a.acc ? (int)a.batch : 1;

  float2* psi_line = psi_s + line * NP;
  float2* wl = work_s + lg * NP;

  // per-thread index helper (q-independent): (lam * (t + e T)) mod N
  int nii[E];
  {
    const int lmod = lam % N;
    const int step = (lmod * T) % N;
    int v = (lmod * t) % N;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      nii[e] = v;
      v += step;
      if (v >= N) v -= N;
    }
  }

  for (int64_t tile = first; tile < ntiles; tile += step) {
    float racc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) racc[e] = 0.f;

    for (int bl = 0; bl < nb_loop; ++bl) {
      __syncthreads();  // previous users of base_s / psi_s / work_s are done
      if (tid < LINES) {
        const int64_t gline = tile * LINES + tid;
        long long base = -1;
        int b = 0;
        if (gline < a.nlines) {
          int64_t bo = gline / inner;
          const int64_t i = gline - bo * inner;
          if (a.acc) {
            b = bl;
            bo += (int64_t)bl * a.outer;
          } else {
            b = (int)(gline / per_real_lines);
          }
          base = bo * (int64_t)N * inner + i;
        }
        base_s[tid] = base;
        b_s[tid] = b;
      }
      __syncthreads();
      // the tile's loads go out U at a time per thread, then their stores (same values)
      constexpr int U = 8;
      for (int idx0 = tid; idx0 < LINES * N; idx0 += U * NT) {
        float2 v[U];
        float gr[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = idx0 + u * NT;
          v[u] = make_float2(0.f, 0.f);
          gr[u] = 1.f;
          if (idx < LINES * N) {
            int l, n;
            tile_coords(idx, N, LINES, contiguous, l, n);
            const long long base = base_s[l];
            if (base >= 0) {
              const int64_t addr = base + (int64_t)n * inner;
              v[u] = a.in[addr];  // plain load: passes may run in place
              if (a.grad) {
                const int64_t b = b_s[l];
                const int64_t gaddr = a.grad_shared ? addr - b * a.M : addr;
                gr[u] = 2.f * __ldg(a.grad + gaddr);
              }
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = idx0 + u * NT;
          if (idx < LINES * N) {
            int l, n;
            tile_coords(idx, N, LINES, contiguous, l, n);
            psi_s[l * NP + pad(n)] = a.grad ? make_float2(v[u].x * gr[u], v[u].y * gr[u]) : v[u];
          }
        }
      }
      __syncthreads();

      float2 res[E];
#pragma unroll
      for (int e = 0; e < E; ++e) res[e] = make_float2(0.f, 0.f);

      if constexpr (KIND == KIND_FWD_PAPER) {
        for (int q = grp; q < lam; q += QG) {
          const float2* Pq = a.tab.P + (size_t)q * N;
          const float2* Kq = a.tab.K + (size_t)q * N;
          const float2* Fq = a.tab.F + (size_t)q * N;
          float2 v[E];
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = cmul(psi_line[pad(t + e * T)], __ldg(Pq + t + e * T));
          fft_line<P, false>(v, wl, tw_s, t, key, twc);
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = cmul(v[e], __ldg(Kq + t + e * T));
          fft_line<P, true>(v, wl, tw_s, t, key, twc);
          line_sync<T>(key);
          store_owned<P>(v, wl, t);
          line_sync<T>(key);
#pragma unroll
          for (int e = 0; e < E; ++e) res[e] = cfma(__ldg(Fq + t + e * T), wl[pad(nii[e])], res[e]);
        }
      } else if constexpr (KIND == KIND_FWD_FOLD) {
        const int g = a.g, Np = a.Np;
        int qN = grp % N;  // q mod N
        const int qstep = QG % N;
        for (int q = grp; q < lam; q += QG) {
          const float2* Pq = a.tab.P + (size_t)q * N;
          const float2* Kq = a.tab.Kf + (size_t)q * N;
          float2 v[E];
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = cmul(psi_line[pad(t + e * T)], __ldg(Pq + t + e * T));
          fft_line<P, false>(v, wl, tw_s, t, key, twc);
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = cmul(v[e], __ldg(Kq + t + e * T));
          line_sync<T>(key);
          store_owned<P>(v, wl, t);
          line_sync<T>(key);
          if (g == 1) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              int jq = t + e * T - qN;
              if (jq < 0) jq += N;
              res[e] = cadd(res[e], wl[pad(fold_s[jq])]);
            }
          } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              int jq = t + e * T - qN;
              if (jq < 0) jq += N;
              const int m0 = fold_s[jq];
              if (m0 >= 0) {
                for (int r = 0; r < g; ++r) res[e] = cadd(res[e], wl[pad(m0 + r * Np)]);
              }
            }
          }
          qN += qstep;
          if (qN >= N) qN -= N;
        }
      } else {  // KIND_ADJ_FOLD
        // D = FFT(g) once per line (group 0), kept in the line's input buffer
        if (grp == 0) {
          float2 v[E];
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = psi_line[pad(t + e * T)];
          fft_line<P, false>(v, wl, tw_s, t, key, twc);
          line_sync<T>(key);
          store_owned<P>(v, psi_line, t);
        }
        __syncthreads();
        int qN = grp % N;
        const int qstep = QG % N;
        for (int q = grp; q < lam; q += QG) {
          const float2* Pq = a.tab.P + (size_t)q * N;
          const float2* Kq = a.tab.Kf + (size_t)q * N;
          float2 v[E];
#pragma unroll
          for (int e = 0; e < E; ++e) {
            int idx = nii[e] + qN;
            if (idx >= N) idx -= N;
            v[e] = cmulc(psi_line[pad(idx)], __ldg(Kq + t + e * T));
          }
          fft_line<P, true>(v, wl, tw_s, t, key, twc);
#pragma unroll
          for (int e = 0; e < E; ++e) res[e] = cadd(res[e], cmulc(v[e], __ldg(Pq + t + e * T)));
          qN += qstep;
          if (qN >= N) qN -= N;
        }
      }

      // add the groups' partial sums in group order (group 0 ends with the line's sum)
      if (QG > 1) {
        __syncthreads();  // every group is done with its exchange buffer
        store_owned<P>(res, wl, t);
        __syncthreads();
        if (grp == 0) {
          for (int r = 1; r < QG; ++r) {
            const float2* other = work_s + (r * LINES + line) * NP;
#pragma unroll
            for (int e = 0; e < E; ++e) res[e] = cadd(res[e], other[pad(t + e * T)]);
          }
        }
      }
      if constexpr (KIND == KIND_FWD_FOLD) {
        if (QG > 1) __syncthreads();  // the other groups' buffers are read; wl is free again
        if (grp == 0) fft_line<P, true>(res, wl, tw_s, t, key, twc);
      }

      if (a.acc) {
        if (grp == 0) {
#pragma unroll
          for (int e = 0; e < E; ++e) racc[e] += res[e].x * res[e].x + res[e].y * res[e].y;
        }
      } else {
        // stage each line (group 0's buffer) in shared memory, then store the tile coalesced
        __syncthreads();
        if (grp == 0) store_owned<P>(res, wl, t);
        __syncthreads();
        for (int idx = tid; idx < LINES * N; idx += NT) {
          int l, n;
          tile_coords(idx, N, LINES, contiguous, l, n);
          const long long base = base_s[l];
          if (base < 0) continue;
          const int64_t addr = base + (int64_t)n * inner;
          const float2 v = work_s[l * NP + pad(n)];
          if (a.out_c) {
            a.out_c[addr] = v;
          } else {
            a.out_d[addr] = v.x * v.x + v.y * v.y;
          }
        }
      }
    }  // batch loop

    if (a.acc) {
      __syncthreads();
      if (grp == 0) {
        float2 tmp[E];
#pragma unroll
        for (int e = 0; e < E; ++e) tmp[e] = make_float2(racc[e], 0.f);
        store_owned<P>(tmp, wl, t);
      }
      __syncthreads();
      for (int idx = tid; idx < LINES * N; idx += NT) {
        int l, n;
        tile_coords(idx, N, LINES, contiguous, l, n);
        const long long base = base_s[l];
        if (base < 0) continue;
        // base_s holds the last realization's line; remove its batch offset
        const int64_t addr = base - (int64_t)(nb_loop - 1) * a.M + (int64_t)n * inner;
        a.out_d[addr] += work_s[l * NP + pad(n)].x;
      }
    }
  }
}

template <class P, int KIND, int G>
__global__ void __launch_bounds__(P::T * G, FFX_PASS_MIN_BLOCKS) pass_kernel(const PassArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  pass_tiles<P, KIND, G>(a, blockIdx.x, INT64_MAX, gridDim.x, smem);
}

template <class P, int KIND, int G>
cudaError_t launch_pass(const PassArgs& a, int grid, cudaStream_t stream) {
  using SM = PassSmem<P, G>;
  const int qg = a.qg > 1 ? a.qg : 1;
  const int threads = (G / qg) * qg * P::T;
  pass_kernel<P, KIND, G><<<grid, threads, SM::bytes, stream>>>(a);
  return cudaGetLastError();
}

template <class P, int KIND, int G>
PassKernelInfo pass_info() {
  using SM = PassSmem<P, G>;
  PassKernelInfo info;
  info.launch = &launch_pass<P, KIND, G>;
  info.func = reinterpret_cast<const void*>(&pass_kernel<P, KIND, G>);
  info.threads = P::T * G;
  info.lines = G;
  info.T = P::T;
  info.max_qg = (P::T <= 32) ? (G < 8 ? G : 8) : 1;
  info.smem = SM::bytes;
  return info;
}

}  // namespace ffx
