// ffx_expand_noalloc: the density expansion without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc once they are running --
// for instance a host framework that has already reserved almost all device
// memory for its own pool (a raw cudaMalloc then fails or fragments that
// pool), or a real-time loop that forbids allocations, and the device-wide
// synchronisation cudaMalloc/cudaFree imply, after start-up.  ffx_plan
// allocates its phase tables and ffx_expand its workspace, so neither fits
// them.  This entry point keeps everything it needs beyond the caller's input
// and output in file-scope __device__ arrays of fixed size, which every GPU
// that loads the library holds until the process exits.
//
// The map is that of ffx_plan + ffx_expand, and the kernels are those of the
// fold form (FFX_FORM_FOLD) on every axis, whatever form ffx_plan's automatic
// choice would take: the phase tables are rebuilt into the static arrays on
// every call, on the caller's stream, and the intermediate field between axis
// passes lives in the static field array.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/ffx.h"
#include "ffx_internal.h"

namespace ffx {
namespace {

// Scratch (sizes also stated in include/ffx.h):
//   field  : FFX_NOALLOC_MAX_FIELD complex64 (8 MiB), the field between passes
//   tables : FFX_NOALLOC_MAX_TABLE complex64 (2 MiB), phase tables of all axes
//   fold   : FFX_NOALLOC_MAX_FOLD ints (32 KiB), fold lookup of all axes
static __device__ __align__(256) float2 g_noalloc_field[FFX_NOALLOC_MAX_FIELD];
static __device__ __align__(256) float2 g_noalloc_tables[FFX_NOALLOC_MAX_TABLE];
static __device__ __align__(256) int g_noalloc_fold[FFX_NOALLOC_MAX_FOLD];

constexpr int kMaxDevices = 64;

struct DeviceScratch {
  bool ready = false;
  float2* field = nullptr;
  float2* tables = nullptr;
  int* fold = nullptr;
  int sms = 1;
};

std::mutex g_setup_mutex;
DeviceScratch g_dev[kMaxDevices];
// The message goes where ffx_last_error() reads it.
int nfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error_message(buf);
  return code;
}

// Once per device, with that device current: the device addresses of the
// static arrays (their names in host code are host-side stand-ins, not device
// addresses), and the kernels' shared-memory limits.
int setup_device(int dev, DeviceScratch** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceScratch& d = g_dev[dev];
  if (!d.ready) {
    cudaError_t e = cudaGetSymbolAddress((void**)&d.field, g_noalloc_field);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d.tables, g_noalloc_tables);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d.fold, g_noalloc_fold);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return nfail(FFX_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    d.sms = sms > 0 ? sms : 1;
    d.ready = true;
  }
  *out = &d;
  return FFX_OK;
}

uint64_t frac_turns(double x) {
  double f = x - std::floor(x);
  if (!(f >= 0.0) || f >= 1.0) f = 0.0;
  return (uint64_t)std::ldexp(f, 64);
}

int64_t gcd_i64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

int64_t inverse_mod(int64_t a, int64_t m) {
  if (m == 1) return 0;
  int64_t t = 0, nt = 1, r = m, nr = a % m;
  while (nr) {
    int64_t qq = r / nr, tmp = t - qq * nt;
    t = nt;
    nt = tmp;
    tmp = r - qq * nr;
    r = nr;
    nr = tmp;
  }
  return t < 0 ? t + m : t;
}

// fold[r] = m0 with (lam/g) m0 = r/g (mod N/g) when g | r, else -1
__global__ void noalloc_fold_kernel(int* fold, int N, int g, int Np, long long inv) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x)
    fold[r] = (r % g == 0) ? (int)(((long long)(r / g) * inv) % Np) : -1;
}

struct AxisState {
  int N, lam, g, Np;
  AxisTables tab;
  PassKernelInfo info;
  int grid;
};

}  // namespace
}  // namespace ffx

using namespace ffx;

extern "C" int ffx_expand_noalloc(int ndim, const int64_t* dims, const double* spacing, double t,
                                  const int32_t* magnification, const double* a,
                                  const double* abar, const void* psi0, int64_t batch,
                                  float* out_density, void* stream) {
  set_last_error_message("");
  if (ndim < 1 || ndim > 3) return nfail(FFX_EINVAL, "ndim must be 1..3, got %d", ndim);
  if (!dims || !spacing || !magnification) return nfail(FFX_EINVAL, "dims/spacing/magnification is NULL");
  if (!std::isfinite(t)) return nfail(FFX_EINVAL, "t must be finite");
  if (batch < 0) return nfail(FFX_EINVAL, "batch < 0");
  int64_t M = 1, table_need = 0, fold_need = 0;
  for (int j = 0; j < ndim; ++j) {
    if (dims[j] < 1 || !ffx_supported_length(dims[j]))
      return nfail(FFX_EUNSUPPORTED, "no line kernel for length %lld (axis %d)", (long long)dims[j], j);
    if (!(spacing[j] > 0) || !std::isfinite(spacing[j]))
      return nfail(FFX_EINVAL, "spacing[%d] must be positive and finite", j);
    if (magnification[j] < 1 || magnification[j] > 65536)
      return nfail(FFX_EINVAL, "magnification[%d] must be an integer in 1..65536", j);
    if ((a && !std::isfinite(a[j])) || (abar && !std::isfinite(abar[j])))
      return nfail(FFX_EINVAL, "offsets must be finite");
    M *= dims[j];
    table_need += 4 * (int64_t)magnification[j] * dims[j] + dims[j];
    fold_need += dims[j];
  }
  if (table_need > FFX_NOALLOC_MAX_TABLE)
    return nfail(FFX_EINVAL, "phase tables need %lld complex entries, the static limit is %d "
                 "(sum over axes of 4*lam*M + M)", (long long)table_need, FFX_NOALLOC_MAX_TABLE);
  if (fold_need > FFX_NOALLOC_MAX_FOLD)
    return nfail(FFX_EINVAL, "lattice too long for the static fold table (%lld > %d)",
                 (long long)fold_need, FFX_NOALLOC_MAX_FOLD);
  if (ndim > 1 && batch * M > FFX_NOALLOC_MAX_FIELD)
    return nfail(FFX_EINVAL, "batch * M = %lld exceeds the static field limit %d",
                 (long long)(batch * M), FFX_NOALLOC_MAX_FIELD);
  if (batch == 0) return FFX_OK;
  if (!psi0 || ((uintptr_t)psi0 & 7)) return nfail(FFX_EINVAL, "psi0 is NULL or not 8-byte aligned");
  if (!out_density || ((uintptr_t)out_density & 7))
    return nfail(FFX_EINVAL, "out_density is NULL or not 8-byte aligned");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(FFX_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return nfail(FFX_EINVAL, "device index %d out of range", dev);
  DeviceScratch* ds = nullptr;
  int rc = setup_device(dev, &ds);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  AxisState ax[3];
  float2* tcur = ds->tables;
  int* fcur = ds->fold;
  for (int j = 0; j < ndim; ++j) {
    AxisState& A = ax[j];
    A.N = (int)dims[j];
    A.lam = magnification[j];
    A.g = (int)gcd_i64(A.lam, A.N);
    A.Np = A.N / A.g;
    const double dx = spacing[j], L = A.N * dx;
    const double aj = a ? a[j] : -0.5 * L;
    const double abj = abar ? abar[j] : aj + (double)(-(((int64_t)(A.lam - 1) * A.N) / 2)) * dx;
    const size_t lN = (size_t)A.lam * A.N;
    float2 *P = tcur, *K = tcur + lN, *Kf = tcur + 2 * lN, *F = tcur + 3 * lN, *tw = tcur + 4 * lN;
    tcur += 4 * lN + A.N;
    const double sv = (abj - aj) / dx, tau = M_PI * t / (L * L);
    e = launch_fill_tables(A.N, A.lam, frac_turns(sv / A.N), frac_turns(tau), frac_turns(2.0 * tau / A.lam),
                           frac_turns(sv / ((double)A.lam * A.N)), frac_turns(tau / ((double)A.lam * A.lam)),
                           nullptr, P, K, Kf, F, tw, s);
    if (e != cudaSuccess) return nfail(FFX_ECUDA, "table fill: %s", cudaGetErrorString(e));
    const int64_t inv = inverse_mod((A.lam / A.g) % A.Np, A.Np);
    noalloc_fold_kernel<<<(A.N + 255) / 256, 256, 0, s>>>(fcur, A.N, A.g, A.Np, (long long)inv);
    e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(FFX_ECUDA, "fold table: %s", cudaGetErrorString(e));
    A.tab.P = P;
    A.tab.K = K;
    A.tab.Kf = Kf;
    A.tab.F = F;
    A.tab.tw = tw;
    A.tab.fold = fcur;
    fcur += A.N;
    if (!find_pass_kernel(A.N, KIND_FWD_FOLD, &A.info))
      return nfail(FFX_EUNSUPPORTED, "no kernel for length %d", A.N);
    e = cudaFuncSetAttribute(A.info.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)A.info.smem);
    if (e != cudaSuccess) return nfail(FFX_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, A.info.func, A.info.threads, A.info.smem) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    A.grid = per_sm * ds->sms;
  }

  // pass order: longest lines first (as ffx_plan)
  int order[3] = {0, 1, 2};
  for (int i = 0; i < ndim; ++i)
    for (int k = i + 1; k < ndim; ++k)
      if (dims[order[k]] > dims[order[i]]) {
        int tmp = order[i];
        order[i] = order[k];
        order[k] = tmp;
      }

  for (int k = 0; k < ndim; ++k) {
    const int j = order[k];
    const AxisState& A = ax[j];
    const bool first = (k == 0), last = (k == ndim - 1);
    PassArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    int64_t outer = 1, inner = 1;
    for (int i = 0; i < j; ++i) outer *= dims[i];
    for (int i = j + 1; i < ndim; ++i) inner *= dims[i];
    pa.in = first ? (const float2*)psi0 : ds->field;
    pa.out_c = last ? nullptr : ds->field;
    pa.out_d = last ? out_density : nullptr;
    pa.outer = outer;
    pa.inner = inner;
    pa.M = M;
    pa.batch = batch;
    pa.acc = 0;
    pa.nlines = batch * outer * inner;
    pa.lam = A.lam;
    pa.g = A.g;
    pa.Np = A.Np;
    pa.tab = A.tab;
    const int64_t ntiles = (pa.nlines + pass_lines_per_tile(A.info, pa.qg) - 1) /
                           pass_lines_per_tile(A.info, pa.qg);
    int64_t grid = A.grid < ntiles ? A.grid : ntiles;
    if (grid < 1) grid = 1;
    e = A.info.launch(pa, (int)grid, s);
    if (e != cudaSuccess) return nfail(FFX_ECUDA, "pass launch: %s", cudaGetErrorString(e));
  }
  return FFX_OK;
}
