// Plan-time phase tables for one axis (see AxisTables in ffx_internal.h).
//
// Every phase of eq. FF (Sec. 5.2) on one axis is 2 pi times a sum of terms
// (real constant) x (integer polynomial in q, n, l).  The host reduces each
// constant to its fractional part as a 64-bit fixed-point number of turns
// (c = frac(constant) * 2^64); here the integer polynomial multiplies it with
// wrapping 64-bit arithmetic, which is exact modulo one turn.  The reduced
// turn in [-1/2, 1/2) then goes through double-precision sincospi and is
// rounded once to float.  Arguments of 10^4..10^6 rad therefore cost no
// precision.
//
// Other spectra (Sec. 7): with a dispersion table (disp != null) the phase
// -t omega(k) of the huge-lattice wavevector k = 2 pi (lam l + q) / (lam L)
// replaces the free-particle terms -tau (l + q/lam)^2.  It depends on q and m
// together, so all of it goes into K (and Kf); F keeps only the shift terms.
// The host passes the table as fixed-point turns frac(-t omega / 2 pi) per
// huge-lattice index u, and zero for the tau constants.
#include "ffx_internal.h"

namespace ffx {

__device__ __forceinline__ float2 turn_to_unit(uint64_t fx, double scale) {
  const double turn = (double)(long long)fx * 0x1p-64;  // [-1/2, 1/2)
  double s, c;
  sincospi(2.0 * turn, &s, &c);
  return make_float2((float)(c * scale), (float)(s * scale));
}

struct TableArgs {
  int N, lam;
  uint64_t c_sN, c_tau, c_2tl, c_slN, c_tl2, c_N, c_lamN;
  const uint64_t* disp;  // [lam N] fixed-point turns of -t omega(k_u), or null (free particle)
  float2 *P, *K, *Kf, *F, *tw;
};

__global__ void fill_tables_kernel(const TableArgs a) {
  const int64_t total = (int64_t)a.lam * a.N;
  const int N = a.N;
  const double inv_lamN = 1.0 / ((double)a.lam * (double)N);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx / N;
    const int64_t n = idx - q * N;  // n for P, m for K/Kf, nbar for F
    // pre-chirp: -q n / (lam N)
    const uint64_t rqn = (uint64_t)((q * n) % ((int64_t)a.lam * N));
    a.P[idx] = turn_to_unit(0ull - rqn * a.c_lamN, 1.0);
    // k-space phase with the symmetric index and the odd-N umklapp
    int64_t l = (2 * n < N) ? n : n - N;
    if ((N & 1) && n == (N - 1) / 2 && 2 * q >= a.lam) l = -(int64_t)(N + 1) / 2;
    uint64_t fk = (uint64_t)l * a.c_sN - (uint64_t)(l * l) * a.c_tau - (uint64_t)(l * q) * a.c_2tl;
    if (a.disp) {
      // huge-lattice index of k = 2 pi (lam l + q) / (lam L)
      const int64_t lamN = (int64_t)a.lam * N;
      const int64_t u = (((int64_t)a.lam * l + q) % lamN + lamN) % lamN;
      fk += a.disp[u];
    }
    a.K[idx] = turn_to_unit(fk, 1.0);
    const uint64_t fq = (uint64_t)q * a.c_slN - (uint64_t)(q * q) * a.c_tl2;
    a.Kf[idx] = turn_to_unit(fk + fq, inv_lamN);
    // post-chirp: q s/(lam N) + q nbar / N - tau q^2 / lam^2, with 1/(lam N)
    const uint64_t rqnb = (uint64_t)((q * n) % N);
    a.F[idx] = turn_to_unit(fq + rqnb * a.c_N, inv_lamN);
    if (q == 0) a.tw[n] = turn_to_unit(0ull - (uint64_t)n * a.c_N, 1.0);
  }
}

cudaError_t launch_fill_tables(int N, int lam, uint64_t c_sN, uint64_t c_tau, uint64_t c_2tl,
                               uint64_t c_slN, uint64_t c_tl2, const uint64_t* disp, float2* P, float2* K,
                               float2* Kf, float2* F, float2* tw, cudaStream_t stream) {
  TableArgs a;
  a.disp = disp;
  a.N = N;
  a.lam = lam;
  a.c_sN = c_sN;
  a.c_tau = c_tau;
  a.c_2tl = c_2tl;
  a.c_slN = c_slN;
  a.c_tl2 = c_tl2;
  // exact reciprocals as 64-bit fixed point (rounded): 2^64 / N, 2^64 / (lam N)
  a.c_N = (uint64_t)((((unsigned __int128)1 << 64) + N / 2) / (unsigned)N);
  const uint64_t lamN = (uint64_t)lam * (uint64_t)N;
  a.c_lamN = (uint64_t)((((unsigned __int128)1 << 64) + lamN / 2) / lamN);
  a.P = P;
  a.K = K;
  a.Kf = Kf;
  a.F = F;
  a.tw = tw;
  const int64_t total = (int64_t)lam * N;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  fill_tables_kernel<<<blocks, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace ffx
