// One pass of the per-axis free-flight map (eq. FF restricted to one axis),
// or of its adjoint, over every line of a [B][outer][N][inner] complex64 array.
//
// A block handles LINES lines at a time (a tile), LINES * T threads, T = N/E
// threads per line.  The tile is loaded into shared memory with coalesced
// accesses, each line is transformed by its T threads in registers (see
// ffx_fft.cuh), and the result is staged back through shared memory and
// stored coalesced: complex64, or |.|^2 as float32, or |.|^2 summed over the
// realizations of the batch (tiles then loop over b in order, so the sum is
// deterministic and needs no atomics).
//
// Kinds (q runs over the fine momentum index 0..lam-1 of eq. FF):
//  FWD_PAPER: acc += F_q * IFFT(K_q * FFT(P_q * psi))[(lam nb) mod N]
//             -- eqs. presA, presB, presf, FFaux and the term sum FFpsi.
//  FWD_FOLD : D[(lam m + q) mod N] += Kf_q[m] * FFT(P_q * psi)[m]; out = IFFT(D)
//             -- the same sum with the presf factor's n-dependence merged into
//             the inverse-DFT kernel (one inverse FFT per line).
//  ADJ_FOLD : the adjoint of FWD_FOLD: D = FFT(g); out = sum_q conj(P_q) *
//             IFFT(conj(Kf_q[m]) * D[(lam m + q) mod N]).
#pragma once

#include "ffx_fft.cuh"
#include "ffx_internal.h"

namespace ffx {

template <class P, int LINES>
struct PassSmem {
  static constexpr int NP = Padded<P::N>::value;
  static constexpr size_t tw_off = 0;
  static constexpr size_t fold_off = tw_off + sizeof(float2) * P::N;
  static constexpr size_t base_off = (fold_off + sizeof(int) * P::N + 15) & ~size_t(15);
  static constexpr size_t b_off = base_off + sizeof(long long) * LINES;
  static constexpr size_t psi_off = (b_off + sizeof(int) * LINES + 15) & ~size_t(15);
  static constexpr size_t work_off = psi_off + sizeof(float2) * LINES * NP;
  static constexpr size_t bytes = work_off + sizeof(float2) * LINES * NP;
};

template <class P, int KIND, int LINES>
__global__ void __launch_bounds__(P::T * LINES)
    pass_kernel(const PassArgs a) {
  constexpr int N = P::N, E = P::E, T = P::T;
  using SM = PassSmem<P, LINES>;
  constexpr int NP = SM::NP;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tw_s = reinterpret_cast<float2*>(smem + SM::tw_off);
  int* fold_s = reinterpret_cast<int*>(smem + SM::fold_off);
  long long* base_s = reinterpret_cast<long long*>(smem + SM::base_off);
  int* b_s = reinterpret_cast<int*>(smem + SM::b_off);
  float2* psi_s = reinterpret_cast<float2*>(smem + SM::psi_off);
  float2* work_s = reinterpret_cast<float2*>(smem + SM::work_off);

  if (a.acc && a.batch <= 0) return;  // nothing to sum (the host never launches this)
  const int tid = threadIdx.x;
  const int lib = tid / T;  // line in block
  const int t = tid - lib * T;
  constexpr int NT = T * LINES;

  for (int i = tid; i < N; i += NT) {
    tw_s[i] = a.tab.tw[i];
    if constexpr (KIND == KIND_FWD_FOLD) fold_s[i] = a.tab.fold[i];
  }

  const int lam = a.lam;
  const int64_t inner = a.inner;
  const int64_t per_real_lines = a.outer * inner;
  const int64_t ntiles = (a.nlines + LINES - 1) / LINES;
  const int nb_loop = a.acc ? (int)a.batch : 1;

  float2* psi_line = psi_s + lib * NP;
  float2* wl = work_s + lib * NP;

  // per-thread index helpers (q-independent)
  int nii[E];  // (lam * (t + e T)) mod N
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

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    float racc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) racc[e] = 0.f;

    for (int bl = 0; bl < nb_loop; ++bl) {
      __syncthreads();  // previous tile's users of base_s / psi_s / work_s are done
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
      // coalesced load of the tile: contiguous lines along n, strided lines along the line index
      for (int idx = tid; idx < LINES * N; idx += NT) {
        int l, n;
        if (inner == 1) {
          l = idx / N;
          n = idx - l * N;
        } else {
          n = idx / LINES;
          l = idx - n * LINES;
        }
        const long long base = base_s[l];
        float2 v = make_float2(0.f, 0.f);
        if (base >= 0) {
          const int64_t addr = base + (int64_t)n * inner;
          v = a.in[addr];  // plain load: passes may run in place
          if (a.grad) {
            const int64_t b = b_s[l];
            const int64_t gaddr = a.grad_shared ? addr - b * a.M : addr;
            const float gr = 2.f * __ldg(a.grad + gaddr);
            v.x *= gr;
            v.y *= gr;
          }
        }
        psi_s[l * NP + pad(n)] = v;
      }
      __syncthreads();

      float2 res[E];
      if constexpr (KIND == KIND_FWD_PAPER) {
#pragma unroll
        for (int e = 0; e < E; ++e) res[e] = make_float2(0.f, 0.f);
        for (int q = 0; q < lam; ++q) {
          const float2* Pq = a.tab.P + (size_t)q * N;
          const float2* Kq = a.tab.K + (size_t)q * N;
          const float2* Fq = a.tab.F + (size_t)q * N;
          float2 v[E];
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = cmul(psi_line[pad(t + e * T)], __ldg(Pq + t + e * T));
          fft_line<P, false>(v, wl, tw_s, t, lib);
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = cmul(v[e], __ldg(Kq + t + e * T));
          fft_line<P, true>(v, wl, tw_s, t, lib);
          line_sync<T>(lib);
          store_owned<P>(v, wl, t);
          line_sync<T>(lib);
#pragma unroll
          for (int e = 0; e < E; ++e) res[e] = cfma(__ldg(Fq + t + e * T), wl[pad(nii[e])], res[e]);
        }
      } else if constexpr (KIND == KIND_FWD_FOLD) {
        float2 D[E];
#pragma unroll
        for (int e = 0; e < E; ++e) D[e] = make_float2(0.f, 0.f);
        const int g = a.g, Np = a.Np;
        int qN = 0;  // q mod N
        for (int q = 0; q < lam; ++q) {
          const float2* Pq = a.tab.P + (size_t)q * N;
          const float2* Kq = a.tab.Kf + (size_t)q * N;
          float2 v[E];
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = cmul(psi_line[pad(t + e * T)], __ldg(Pq + t + e * T));
          fft_line<P, false>(v, wl, tw_s, t, lib);
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = cmul(v[e], __ldg(Kq + t + e * T));
          line_sync<T>(lib);
          store_owned<P>(v, wl, t);
          line_sync<T>(lib);
#pragma unroll
          for (int e = 0; e < E; ++e) {
            int jq = t + e * T - qN;
            if (jq < 0) jq += N;
            const int m0 = fold_s[jq];
            if (m0 >= 0) {
              for (int r = 0; r < g; ++r) D[e] = cadd(D[e], wl[pad(m0 + r * Np)]);
            }
          }
          if (++qN == N) qN = 0;
        }
        fft_line<P, true>(D, wl, tw_s, t, lib);
#pragma unroll
        for (int e = 0; e < E; ++e) res[e] = D[e];
      } else {  // KIND_ADJ_FOLD
        float2 v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = psi_line[pad(t + e * T)];
        fft_line<P, false>(v, wl, tw_s, t, lib);
        line_sync<T>(lib);
        store_owned<P>(v, psi_line, t);  // D = FFT(g) replaces g in the line buffer
        line_sync<T>(lib);
#pragma unroll
        for (int e = 0; e < E; ++e) res[e] = make_float2(0.f, 0.f);
        int qN = 0;
        for (int q = 0; q < lam; ++q) {
          const float2* Pq = a.tab.P + (size_t)q * N;
          const float2* Kq = a.tab.Kf + (size_t)q * N;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            int idx = nii[e] + qN;
            if (idx >= N) idx -= N;
            v[e] = cmulc(psi_line[pad(idx)], __ldg(Kq + t + e * T));
          }
          fft_line<P, true>(v, wl, tw_s, t, lib);
#pragma unroll
          for (int e = 0; e < E; ++e) res[e] = cadd(res[e], cmulc(v[e], __ldg(Pq + t + e * T)));
          if (++qN == N) qN = 0;
        }
      }

      if (a.acc) {
#pragma unroll
        for (int e = 0; e < E; ++e) racc[e] += res[e].x * res[e].x + res[e].y * res[e].y;
      } else {
        // stage the line in shared memory, then store the tile coalesced
        line_sync<T>(lib);
        store_owned<P>(res, wl, t);
        __syncthreads();
        for (int idx = tid; idx < LINES * N; idx += NT) {
          int l, n;
          if (inner == 1) {
            l = idx / N;
            n = idx - l * N;
          } else {
            n = idx / LINES;
            l = idx - n * LINES;
          }
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
      line_sync<T>(lib);
      float2 tmp[E];
#pragma unroll
      for (int e = 0; e < E; ++e) tmp[e] = make_float2(racc[e], 0.f);
      store_owned<P>(tmp, wl, t);
      __syncthreads();
      for (int idx = tid; idx < LINES * N; idx += NT) {
        int l, n;
        if (inner == 1) {
          l = idx / N;
          n = idx - l * N;
        } else {
          n = idx / LINES;
          l = idx - n * LINES;
        }
        const long long base = base_s[l];
        if (base < 0) continue;
        // base_s holds the last realization's line; remove its batch offset
        const int64_t addr = base - (int64_t)(nb_loop - 1) * a.M + (int64_t)n * inner;
        a.out_d[addr] += work_s[l * NP + pad(n)].x;
      }
    }
  }
}

template <class P, int KIND, int LINES>
cudaError_t launch_pass(const PassArgs& a, int grid, cudaStream_t stream) {
  using SM = PassSmem<P, LINES>;
  pass_kernel<P, KIND, LINES><<<grid, P::T * LINES, SM::bytes, stream>>>(a);
  return cudaGetLastError();
}

template <class P, int KIND, int LINES>
PassKernelInfo pass_info() {
  using SM = PassSmem<P, LINES>;
  PassKernelInfo info;
  info.launch = &launch_pass<P, KIND, LINES>;
  info.func = reinterpret_cast<const void*>(&pass_kernel<P, KIND, LINES>);
  info.threads = P::T * LINES;
  info.lines = LINES;
  info.smem = SM::bytes;
  return info;
}

}  // namespace ffx
