// One pass of the per-axis free-flight map (eq. FF restricted to one axis),
// or of its adjoint, over every line of a [B][outer][N][inner] complex64 array.
//
// A block holds G line-groups of T = N/E threads.  qg groups share one line
// and split its sum over the fine momentum index q (group r takes
// q = r, r + qg, ...; the paper notes the terms are independent, Sec. 7.1),
// so a tile is G/qg lines.  Tiles are loaded into shared memory by cp.async,
// coalesced (along a contiguous line, or across neighbouring strided lines),
// one tile ahead of the one being transformed; each group transforms its line
// in registers, exchanging across its threads by warp shuffles (see
// ffx_fft.cuh), and indexes the k-space phases and the fold by the spectral
// position spec(t, e) of each register; the groups' partial sums are added in
// shared memory in group order (deterministic); the result is staged back
// through shared memory and
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
  static constexpr size_t tw_off = 0;                                   // w_N^(t k_e) as [k_e][t]
  static constexpr size_t stw_off = tw_off + sizeof(float2) * P::N;     // stage twiddles (T)
  static constexpr size_t fold_off = stw_off + sizeof(float2) * P::T;
  // line offsets of three units (the one being stored, the one being
  // transformed, the one in flight: a slot is rewritten only two units after
  // its last reader), and tiles of two (transformed, in flight)
  static constexpr size_t base_off = (fold_off + sizeof(int) * P::N + 15) & ~size_t(15);
  static constexpr size_t b_off = base_off + 3 * sizeof(long long) * G;
  static constexpr size_t psi_off = (b_off + 3 * sizeof(int) * G + 15) & ~size_t(15);
  static constexpr size_t work_off = psi_off + 2 * sizeof(float2) * G * NP;
  static constexpr size_t bytes = work_off + sizeof(float2) * G * NP;
};

// A thread's walk over the elements idx = tid, tid + NT, ... of a tile copy,
// element idx being (line l, point n) along n for contiguous lines and along
// the line index for strided ones (neighbouring lines are neighbours in
// memory), so either way the copy is coalesced; no division per element:
// contiguous lines advance along n, strided ones along the line index (which
// stays put when NT is a multiple of the tile's line count).
template <int N>
struct TileWalk {
  int l, n, dl, dn;
  bool contiguous;
  int lines;
  __device__ __forceinline__ TileWalk(int tid, int NT, bool contig, int LINES) : contiguous(contig), lines(LINES) {
    if (contiguous) {
      l = tid / N;
      n = tid - l * N;
      dl = NT / N;
      dn = NT - dl * N;
    } else {
      l = tid % LINES;
      n = tid / LINES;
      dl = NT % LINES;
      dn = NT / LINES;
    }
  }
  __device__ __forceinline__ bool ok() const { return l < lines && n < N; }
  __device__ __forceinline__ void next() {
    l += dl;
    n += dn;
    if (contiguous) {
      if (n >= N) {
        n -= N;
        ++l;
      }
    } else if (l >= lines) {
      l -= lines;
      ++n;
    }
  }
};

// Tiles first, first + step, ... (below min(last, number of tiles)) of one
// pass.  Called by a whole block; uses `smem` (PassSmem<P, G>::bytes).
template <class P, int KIND, int G>
__device__ __forceinline__ void pass_tiles(const PassArgs& a, int64_t first, int64_t last, int64_t step,
                                           unsigned char* smem) {
  constexpr int N = P::N, E = P::E, T = P::T;
  using SM = PassSmem<P, G>;
  constexpr int NP = SM::NP;
  float2* tw_s = reinterpret_cast<float2*>(smem + SM::tw_off);
  float2* stw_s = reinterpret_cast<float2*>(smem + SM::stw_off);
  int* fold_s = reinterpret_cast<int*>(smem + SM::fold_off);
  long long* const base_all = reinterpret_cast<long long*>(smem + SM::base_off);
  int* const b_all = reinterpret_cast<int*>(smem + SM::b_off);
  float2* const psi_all = reinterpret_cast<float2*>(smem + SM::psi_off);
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
  fill_line_twiddles<P>(tw_s, stw_s, a.tab.tw, tid, NT);
  if constexpr (KIND == KIND_FWD_FOLD)
    for (int i = tid; i < N; i += NT) fold_s[i] = a.tab.fold[i];

  __syncthreads();  // twiddles are in shared memory
  LineFftCtx<P> fc;
  fc.init(stw_s, key);

  const int lam = a.lam;
  const int64_t inner = a.inner;
  const bool contiguous = (inner == 1);
  const int64_t per_real_lines = a.outer * inner;
  int64_t ntiles = (a.nlines + LINES - 1) / LINES;
  if (last < ntiles) ntiles = last;
  const int nb_loop = a.acc ? (int)a.batch : 1;

  float2* wl = work_s + lg * NP;

  // per-thread index helper (q-independent): (lam * j) mod N for the
  // register's position j: the natural one t + e T (post-chirp gather of the
  // paper form) or the spectral one spec(t, e) (the adjoint's fold gather)
  int nii[E];
  {
    const int lmod = lam % N;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = KIND == KIND_ADJ_FOLD ? spec_index<P>(t, e) : t + e * T;
      nii[e] = (int)(((long long)lmod * j) % N);
    }
  }
  // spectral position of register e: sbase + e (k-space tables, the fold)
  const int sbase = spec_index<P>(t, 0);

  // The block's units -- (tile, realization) pairs, realizations innermost --
  // run as a two-stage pipeline: while unit k is transformed and stored, the
  // copies of unit k + 1 (cp.async, 8 bytes per point, coalesced along the
  // line or across neighbouring strided lines) land in the other buffer.
  const int64_t my_tiles = first < ntiles ? (ntiles - first + step - 1) / step : 0;
  const int64_t units = my_tiles * nb_loop;
  // lines' offsets of unit u into slot `slot` (threads below LINES)
  auto unit_bases = [&](int64_t u, int slot) {
    if (tid < LINES) {
      const int64_t tile = first + (u / nb_loop) * step;
      const int bl = (int)(u % nb_loop);
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
      base_all[slot * G + tid] = base;
      b_all[slot * G + tid] = b;
    }
  };
  // the copies of a unit whose offsets are in slot `slot` into tile buffer
  // `buf` (one commit group)
  auto unit_loads = [&](int slot, int buf) {
    const long long* bs = base_all + slot * G;
    const uint32_t dst0 = (uint32_t)__cvta_generic_to_shared(psi_all + buf * G * NP);
    for (TileWalk<N> w(tid, NT, contiguous, LINES); w.ok(); w.next()) {
      const int l = w.l, n = w.n;
      const long long base = bs[l];
      const bool valid = base >= 0;
      const float2* src = a.in + (valid ? base + (int64_t)n * inner : 0);
      // invalid lines read nothing and land as zeros (source size 0)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst0 + (uint32_t)(l * NP + pad(n)) * 8u),
                   "l"(src), "r"(valid ? 8 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (units > 0) {
    unit_bases(0, 0);
    __syncthreads();
    unit_loads(0, 0);
  }
  float racc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) racc[e] = 0.f;
  for (int64_t k = 0; k < units; ++k) {
    const int buf = (int)(k & 1);
    const int slot = (int)(k % 3), next_slot = slot == 2 ? 0 : slot + 1;
    const int bl = (int)(k % nb_loop);
    if (bl == 0) {
#pragma unroll
      for (int e = 0; e < E; ++e) racc[e] = 0.f;
    }
    // unit k + 1's offsets (a slot last read by unit k - 2) and copies;
    // after the barrier everyone is past unit k - 1, the last reader of the
    // other tile buffer and of work_s
    if (k + 1 < units) unit_bases(k + 1, next_slot);
    __syncthreads();
    if (k + 1 < units) {
      unit_loads(next_slot, buf ^ 1);
    } else {
      asm volatile("cp.async.commit_group;" ::: "memory");  // an empty group keeps the count
    }
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // this thread's copies of unit k
    __syncthreads();                                       // ... and everyone's
    const long long* base_s = base_all + slot * G;
    const int* b_s = b_all + slot * G;
    float2* const psi_s = psi_all + buf * G * NP;
    float2* const psi_line = psi_s + line * NP;
    if (a.grad) {
      // backward passes: the input element is 2 grad * psi
      for (TileWalk<N> w(tid, NT, contiguous, LINES); w.ok(); w.next()) {
        const int l = w.l, n = w.n;
        const long long base = base_s[l];
        if (base < 0) continue;
        const int64_t addr = base + (int64_t)n * inner;
        const int64_t gaddr = a.grad_shared ? addr - (int64_t)b_s[l] * a.M : addr;
        const float gr = 2.f * __ldg(a.grad + gaddr);
        float2& x = psi_s[l * NP + pad(n)];
        x = make_float2(x.x * gr, x.y * gr);
      }
      __syncthreads();
    }

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
          for (int e = 0; e < E; ++e)  // the q = 0 pre-chirp is 1
            v[e] = q == 0 ? psi_line[pad(t + e * T)] : cmul(psi_line[pad(t + e * T)], __ldg(Pq + t + e * T));
          fft_fwd<P>(v, wl, tw_s, t, key, fc);
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = cmul(v[e], __ldg(Kq + (sbase + e)));
          fft_inv<P>(v, wl, tw_s, t, key, fc);
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
          for (int e = 0; e < E; ++e)  // the q = 0 pre-chirp is 1
            v[e] = q == 0 ? psi_line[pad(t + e * T)] : cmul(psi_line[pad(t + e * T)], __ldg(Pq + t + e * T));
          fft_fwd<P>(v, wl, tw_s, t, key, fc);
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = cmul(v[e], __ldg(Kq + (sbase + e)));
          if (lam == 1) {
            // the fold is the identity: D = Kf_0 * FFT(psi), in place
#pragma unroll
            for (int e = 0; e < E; ++e) res[e] = cadd(res[e], v[e]);
            continue;
          }
          line_sync<T>(key);
          store_spectral<P>(v, wl, t);
          line_sync<T>(key);
          // D[j] at the register's spectral position j (the layout the inverse takes)
          if (g == 1) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              int jq = (sbase + e) - qN;
              if (jq < 0) jq += N;
              res[e] = cadd(res[e], wl[pad(fold_s[jq])]);
            }
          } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              int jq = (sbase + e) - qN;
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
          fft_fwd<P>(v, wl, tw_s, t, key, fc);
          line_sync<T>(key);
          store_spectral<P>(v, psi_line, t);  // D in natural order
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
            v[e] = cmulc(psi_line[pad(idx)], __ldg(Kq + (sbase + e)));
          }
          fft_inv<P>(v, wl, tw_s, t, key, fc);
#pragma unroll
          for (int e = 0; e < E; ++e)  // the q = 0 pre-chirp is 1
            res[e] = cadd(res[e], q == 0 ? v[e] : cmulc(v[e], __ldg(Pq + t + e * T)));
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
        if (grp == 0) fft_inv<P>(res, wl, tw_s, t, key, fc);
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
        for (TileWalk<N> w(tid, NT, contiguous, LINES); w.ok(); w.next()) {
          const int l = w.l, n = w.n;
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

    if (a.acc && bl == nb_loop - 1) {
      __syncthreads();
      if (grp == 0) {
        float2 tmp[E];
#pragma unroll
        for (int e = 0; e < E; ++e) tmp[e] = make_float2(racc[e], 0.f);
        store_owned<P>(tmp, wl, t);
      }
      __syncthreads();
      for (TileWalk<N> w(tid, NT, contiguous, LINES); w.ok(); w.next()) {
        const int l = w.l, n = w.n;
        const long long base = base_s[l];
        if (base < 0) continue;
        // base_s holds the last realization's line; remove its batch offset
        const int64_t addr = base - (int64_t)(nb_loop - 1) * a.M + (int64_t)n * inner;
        a.out_d[addr] += work_s[l * NP + pad(n)].x;
      }
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
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
