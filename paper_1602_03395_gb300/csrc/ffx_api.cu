// C ABI of the free-flight expansion library: plans, argument checks,
// workspace, and the sequence of per-axis passes.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "../../include/ffx.h"
#include "ffx_internal.h"

namespace ffx {
bool pass_kernel_16(int, PassKernelInfo*);
bool pass_kernel_32(int, PassKernelInfo*);
bool pass_kernel_48(int, PassKernelInfo*);
bool pass_kernel_64(int, PassKernelInfo*);
bool pass_kernel_96(int, PassKernelInfo*);
bool pass_kernel_128(int, PassKernelInfo*);
bool pass_kernel_192(int, PassKernelInfo*);
bool pass_kernel_256(int, PassKernelInfo*);
bool pass_kernel_384(int, PassKernelInfo*);
bool pass_kernel_512(int, PassKernelInfo*);
bool pass_kernel_768(int, PassKernelInfo*);
bool pass_kernel_1024(int, PassKernelInfo*);
bool pass_kernel_2048(int, PassKernelInfo*);

bool find_pass_kernel(int N, int kind, PassKernelInfo* out) {
  switch (N) {
    case 16: return pass_kernel_16(kind, out);
    case 32: return pass_kernel_32(kind, out);
    case 48: return pass_kernel_48(kind, out);
    case 64: return pass_kernel_64(kind, out);
    case 96: return pass_kernel_96(kind, out);
    case 128: return pass_kernel_128(kind, out);
    case 192: return pass_kernel_192(kind, out);
    case 256: return pass_kernel_256(kind, out);
    case 384: return pass_kernel_384(kind, out);
    case 512: return pass_kernel_512(kind, out);
    case 768: return pass_kernel_768(kind, out);
    case 1024: return pass_kernel_1024(kind, out);
    case 2048: return pass_kernel_2048(kind, out);
    default: return false;
  }
}

bool supported_length(int64_t N) {
  PassKernelInfo info;
  return N > 0 && N <= 2048 && find_pass_kernel((int)N, KIND_FWD_FOLD, &info);
}

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(FFX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// frac(x) as a 64-bit fixed-point number of turns.
uint64_t frac_fx(double x) {
  double f = x - std::floor(x);
  if (!(f >= 0.0) || f >= 1.0) f = 0.0;
  return (uint64_t)std::ldexp(f, 64);
}

int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// inverse of a modulo m (gcd(a, m) = 1), m >= 1
int64_t inv_mod(int64_t a, int64_t m) {
  if (m == 1) return 0;
  int64_t t = 0, nt = 1, r = m, nr = a % m;
  while (nr) {
    int64_t qq = r / nr;
    int64_t tmp = t - qq * nt;
    t = nt;
    nt = tmp;
    tmp = r - qq * nr;
    r = nr;
    nr = tmp;
  }
  if (t < 0) t += m;
  return t;
}

struct Axis {
  int N = 0, lam = 1, g = 1, Np = 1;
  double dx = 0, a = 0, abar = 0;
  float2 *P = nullptr, *K = nullptr, *Kf = nullptr, *F = nullptr, *tw = nullptr;
  int* fold = nullptr;
  PassKernelInfo fwd{}, adj{};
  int grid_fwd = 0, grid_adj = 0;
};

}  // namespace

void set_last_error_message(const char* msg) { g_last_error = msg ? msg : ""; }

}  // namespace ffx

using namespace ffx;

struct ffx_plan_s {
  int ndim = 0;
  int64_t dims[3] = {1, 1, 1};
  int64_t M = 1;
  double t = 0;
  uint32_t flags = 0;
  int form = FFX_FORM_FOLD;
  int acc = 0;
  int device = 0;
  Axis axis[3];
  int order[3] = {0, 1, 2};  // forward pass order
  void* tables = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  ManyPlan* many = nullptr;        // set for plans over many instances
  void* const* trace = nullptr;  // caller's cudaEvent_t array (profiling)
  int64_t trace_n = 0;
  int64_t trace_i = 0;
};

namespace {

int axis_outer_inner(const ffx_plan_s* p, int j, int64_t* outer, int64_t* inner) {
  int64_t o = 1, in = 1;
  for (int i = 0; i < j; ++i) o *= p->dims[i];
  for (int i = j + 1; i < p->ndim; ++i) in *= p->dims[i];
  *outer = o;
  *inner = in;
  return 0;
}

int grid_for(const PassKernelInfo& info, int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, info.func, info.threads, info.smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * sms;
}

// Thread groups per line (qg): split a line's q-sum over qg groups when the
// lines alone cannot fill the GPU.  Cost model: waves of resident blocks times
// the q-terms each group runs (plus one for the epilogue); ties keep fewer groups.
int choose_qg(const PassKernelInfo& k, int64_t nlines, int lam, int capacity) {
  int best = 1;
  double best_cost = 1e300;
  const int qmax = k.max_qg < lam ? k.max_qg : lam;
  for (int qg = 1; qg <= qmax; ++qg) {
    const int lines = pass_lines_per_tile(k, qg);
    if (lines < 1) break;
    const int64_t tiles = (nlines + lines - 1) / lines;
    const int64_t waves = (tiles + capacity - 1) / capacity;
    const double cost = (double)waves * ((lam + qg - 1) / qg + 1);
    if (cost < best_cost * (1.0 - 1e-9)) {
      best_cost = cost;
      best = qg;
    }
  }
  return best;
}

int prepare_kernel(PassKernelInfo& info) {
  cudaError_t e = cudaFuncSetAttribute(info.func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)info.smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  return FFX_OK;
}

int check_ptr(const void* p, const char* name) {
  if (!p) return fail(FFX_EINVAL, "%s is NULL", name);
  if (((uintptr_t)p) & 7) return fail(FFX_EINVAL, "%s is not 8-byte aligned", name);
  return FFX_OK;
}

int ensure_ws(ffx_plan_s* p, int64_t batch) {
  const size_t need = (size_t)batch * (size_t)p->M * sizeof(float2);
  if (need <= p->ws_bytes) return FFX_OK;
  if (p->ws) {
    cudaFree(p->ws);  // synchronizes the device: queued users of the old buffer finish first
    p->ws = nullptr;
    p->ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&p->ws, need);
  if (e != cudaSuccess) {
    p->ws = nullptr;
    cudaGetLastError();
    return fail(FFX_ENOMEM, "workspace of %zu bytes: %s", need, cudaGetErrorString(e));
  }
  p->ws_bytes = need;
  return FFX_OK;
}

// Launch one pass of axis j.
int run_pass(ffx_plan_s* p, int j, bool adjoint, const float2* in, const float* grad,
             int grad_shared, float2* out_c, float* out_d, int acc, int64_t batch,
             cudaStream_t stream) {
  const Axis& ax = p->axis[j];
  PassArgs a;
  std::memset(&a, 0, sizeof(a));
  int64_t outer, inner;
  axis_outer_inner(p, j, &outer, &inner);
  a.in = in;
  a.grad = grad;
  a.grad_shared = grad_shared;
  a.out_c = out_c;
  a.out_d = out_d;
  a.outer = outer;
  a.inner = inner;
  a.M = p->M;
  a.batch = batch;
  a.acc = acc;
  a.nlines = acc ? outer * inner : batch * outer * inner;
  a.lam = ax.lam;
  a.g = ax.g;
  a.Np = ax.Np;
  a.tab.P = ax.P;
  a.tab.K = ax.K;
  a.tab.Kf = ax.Kf;
  a.tab.F = ax.F;
  a.tab.tw = ax.tw;
  a.tab.fold = ax.fold;
  const PassKernelInfo& info = adjoint ? ax.adj : ax.fwd;
  const int capacity = adjoint ? ax.grid_adj : ax.grid_fwd;
  // The split depends on one realization's lines only, so a realization's
  // result does not depend on the batch it came in (bitwise).
  a.qg = choose_qg(info, outer * inner, ax.lam, capacity);
  const int lines = pass_lines_per_tile(info, a.qg);
  const int64_t ntiles = (a.nlines + lines - 1) / lines;
  int64_t grid = capacity;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  const bool traced = p->trace && p->trace_i + 2 <= p->trace_n;
  if (traced) cudaEventRecord((cudaEvent_t)p->trace[p->trace_i], stream);
  cudaError_t e = info.launch(a, (int)grid, stream);
  if (e != cudaSuccess) return cuda_fail(e, "pass launch");
  if (traced) {
    cudaEventRecord((cudaEvent_t)p->trace[p->trace_i + 1], stream);
    p->trace_i += 2;
  }
  return FFX_OK;
}

// Forward map into a complex field (out may equal in).
int forward_field(ffx_plan_s* p, const float2* psi0, int64_t batch, float2* out,
                  cudaStream_t s) {
  const float2* cur = psi0;
  for (int k = 0; k < p->ndim; ++k) {
    int rc = run_pass(p, p->order[k], false, cur, nullptr, 0, out, nullptr, 0, batch, s);
    if (rc) return rc;
    cur = out;
  }
  return FFX_OK;
}

}  // namespace

extern "C" {

const char* ffx_error_string(int code) {
  switch (code) {
    case FFX_OK: return "ok";
    case FFX_EINVAL: return "invalid argument";
    case FFX_ENOMEM: return "out of device memory";
    case FFX_ECUDA: return "CUDA error";
    case FFX_EUNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
  }
}

const char* ffx_last_error(void) { return g_last_error.c_str(); }

int ffx_supported_length(int64_t n) { return supported_length(n) ? 1 : 0; }

int ffx_plan(ffx_plan_t* out, int ndim, const int64_t* dims, const double* spacing, double t,
             const int32_t* magnification, const double* a, const double* abar, uint32_t flags) {
  g_last_error.clear();
  if (!out) return fail(FFX_EINVAL, "out is NULL");
  *out = nullptr;
  if (ndim < 1 || ndim > 3) return fail(FFX_EINVAL, "ndim must be 1..3, got %d", ndim);
  if (!dims || !spacing || !magnification) return fail(FFX_EINVAL, "dims/spacing/magnification is NULL");
  if (!std::isfinite(t)) return fail(FFX_EINVAL, "t must be finite");
  const uint32_t known = FFX_FORM_MASK | FFX_ACCUMULATE;
  if (flags & ~known) return fail(FFX_EINVAL, "unknown flag bits 0x%x", flags & ~known);
  const uint32_t form = flags & FFX_FORM_MASK;
  if (form != FFX_FORM_AUTO && form != FFX_FORM_PAPER && form != FFX_FORM_FOLD)
    return fail(FFX_EINVAL, "unknown form %u", form);
  int64_t M = 1;
  for (int j = 0; j < ndim; ++j) {
    if (dims[j] < 1) return fail(FFX_EINVAL, "dims[%d] = %lld < 1", j, (long long)dims[j]);
    if (!(spacing[j] > 0) || !std::isfinite(spacing[j]))
      return fail(FFX_EINVAL, "spacing[%d] must be positive and finite", j);
    if (magnification[j] < 1 || magnification[j] > 65536)
      return fail(FFX_EINVAL, "magnification[%d] = %d must be an integer in 1..65536", j,
                  (int)magnification[j]);
    if ((int64_t)magnification[j] * dims[j] > (int64_t(1) << 24))
      return fail(FFX_EINVAL, "magnification[%d] * dims[%d] exceeds 2^24", j, j);
    if ((a && !std::isfinite(a[j])) || (abar && !std::isfinite(abar[j])))
      return fail(FFX_EINVAL, "offsets must be finite");
    if (!supported_length(dims[j]))
      return fail(FFX_EUNSUPPORTED, "no line kernel for length %lld (axis %d)", (long long)dims[j], j);
    M *= dims[j];
  }

  ffx_plan_s* p = new (std::nothrow) ffx_plan_s();
  if (!p) return fail(FFX_ENOMEM, "host allocation failed");
  p->ndim = ndim;
  p->t = t;
  p->flags = flags;
  p->form = (form == FFX_FORM_PAPER) ? FFX_FORM_PAPER : FFX_FORM_FOLD;
  p->acc = (flags & FFX_ACCUMULATE) ? 1 : 0;
  p->M = M;
  cudaGetDevice(&p->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  if (sms < 1) sms = 1;

  // table memory: per axis 4 lam*N complex tables + N twiddles + N fold ints
  size_t bytes = 0;
  for (int j = 0; j < ndim; ++j) {
    const size_t N = (size_t)dims[j], lam = (size_t)magnification[j];
    bytes += (4 * lam * N + N) * sizeof(float2) + ((N * sizeof(int) + 255) & ~size_t(255));
  }
  cudaError_t e = cudaMalloc(&p->tables, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return fail(FFX_ENOMEM, "phase tables (%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  cudaStream_t s;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(p->tables);
    delete p;
    return cuda_fail(e, "cudaStreamCreate");
  }
  char* cur = (char*)p->tables;
  int rc = FFX_OK;
  for (int j = 0; j < ndim && rc == FFX_OK; ++j) {
    Axis& ax = p->axis[j];
    const int N = (int)dims[j];
    const int lam = magnification[j];
    p->dims[j] = dims[j];
    ax.N = N;
    ax.lam = lam;
    ax.dx = spacing[j];
    const double L = N * ax.dx;
    ax.a = a ? a[j] : -0.5 * L;
    if (abar) {
      ax.abar = abar[j];
    } else {
      const int64_t sdef = -(((int64_t)(lam - 1) * N) / 2);
      ax.abar = ax.a + (double)sdef * ax.dx;
    }
    ax.g = (int)gcd64(lam, N);
    ax.Np = N / ax.g;
    const size_t lN = (size_t)lam * N;
    ax.P = (float2*)cur;
    cur += lN * sizeof(float2);
    ax.K = (float2*)cur;
    cur += lN * sizeof(float2);
    ax.Kf = (float2*)cur;
    cur += lN * sizeof(float2);
    ax.F = (float2*)cur;
    cur += lN * sizeof(float2);
    ax.tw = (float2*)cur;
    cur += (size_t)N * sizeof(float2);
    ax.fold = (int*)cur;
    cur += ((size_t)N * sizeof(int) + 255) & ~size_t(255);

    // phase constants in turns (hbar = m = 1): s = (abar - a)/dx, tau = pi t / L^2
    const double sv = (ax.abar - ax.a) / ax.dx;
    const double tau = M_PI * t / (L * L);
    const uint64_t c_sN = frac_fx(sv / N);
    const uint64_t c_tau = frac_fx(tau);
    const uint64_t c_2tl = frac_fx(2.0 * tau / lam);
    const uint64_t c_slN = frac_fx(sv / ((double)lam * N));
    const uint64_t c_tl2 = frac_fx(tau / ((double)lam * lam));
    e = launch_fill_tables(N, lam, c_sN, c_tau, c_2tl, c_slN, c_tl2, ax.P, ax.K, ax.Kf, ax.F, ax.tw, s);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "table fill");
      break;
    }
    // fold table: m0 with (lam/g) m0 = r/g (mod N/g) for g | r, else -1
    int* fold_h = (int*)std::malloc(sizeof(int) * N);
    if (!fold_h) {
      rc = fail(FFX_ENOMEM, "host allocation failed");
      break;
    }
    const int64_t inv = inv_mod((lam / ax.g) % ax.Np, ax.Np);
    for (int r = 0; r < N; ++r)
      fold_h[r] = (r % ax.g == 0) ? (int)(((int64_t)(r / ax.g) * inv) % ax.Np) : -1;
    e = cudaMemcpyAsync(ax.fold, fold_h, sizeof(int) * N, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    std::free(fold_h);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "fold table upload");
      break;
    }
    const int kind = (p->form == FFX_FORM_PAPER) ? KIND_FWD_PAPER : KIND_FWD_FOLD;
    if (!find_pass_kernel(N, kind, &ax.fwd) || !find_pass_kernel(N, KIND_ADJ_FOLD, &ax.adj)) {
      rc = fail(FFX_EUNSUPPORTED, "no kernel for length %d", N);
      break;
    }
    if ((rc = prepare_kernel(ax.fwd)) != FFX_OK) break;
    if ((rc = prepare_kernel(ax.adj)) != FFX_OK) break;
    ax.grid_fwd = grid_for(ax.fwd, sms);
    ax.grid_adj = grid_for(ax.adj, sms);
  }
  if (rc == FFX_OK) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "table fill");
  }
  cudaStreamDestroy(s);
  if (rc != FFX_OK) {
    cudaFree(p->tables);
    delete p;
    return rc;
  }
  // Forward order: longest lines first, so the last pass (which may sum the
  // ensemble and then has only one realization's lines to spread over the
  // GPU) runs on the axis with the most lines.
  for (int j = 0; j < ndim; ++j) p->order[j] = j;
  for (int i = 0; i < ndim; ++i)
    for (int k = i + 1; k < ndim; ++k)
      if (p->dims[p->order[k]] > p->dims[p->order[i]]) {
        int tmp = p->order[i];
        p->order[i] = p->order[k];
        p->order[k] = tmp;
      }
  *out = p;
  return FFX_OK;
}

int ffx_plan_many(ffx_plan_t* out, int n_instances, const ffx_instance_desc* descs, uint32_t flags) {
  g_last_error.clear();
  if (!out) return fail(FFX_EINVAL, "out is NULL");
  *out = nullptr;
  std::string err;
  ManyPlan* mp = nullptr;
  int rc = many_create(&mp, n_instances, descs, flags, &err);
  if (rc) return fail(rc, "%s", err.c_str());
  ffx_plan_s* p = new (std::nothrow) ffx_plan_s();
  if (!p) {
    many_destroy(mp);
    return fail(FFX_ENOMEM, "host allocation failed");
  }
  p->many = mp;
  p->ndim = many_max_dim(mp);
  p->form = many_form(mp);
  p->M = many_total(mp);
  *out = p;
  return FFX_OK;
}

int64_t ffx_plan_many_offset(ffx_plan_t p, int i) {
  if (!p || !p->many) return -1;
  return many_offset(p->many, i);
}

int64_t ffx_plan_points(ffx_plan_t p) { return p ? p->M : -1; }

int ffx_plan_destroy(ffx_plan_t p) {
  if (!p) return FFX_OK;
  cudaDeviceSynchronize();
  if (p->many) {
    many_destroy(p->many);
    delete p;
    return FFX_OK;
  }
  if (p->ws) cudaFree(p->ws);
  if (p->tables) cudaFree(p->tables);
  delete p;
  return FFX_OK;
}

int ffx_plan_form(ffx_plan_t p) { return p ? p->form : -1; }

int ffx_plan_pass_order(ffx_plan_t p, int32_t* order) {
  if (!p || !order) return fail(FFX_EINVAL, "plan or order is NULL");
  for (int k = 0; k < p->ndim; ++k) order[k] = p->order[k];
  return FFX_OK;
}

int ffx_plan_trace(ffx_plan_t p, void* const* events, int64_t n_events) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (n_events < 0) return fail(FFX_EINVAL, "n_events < 0");
  p->trace = (events && n_events > 0) ? events : nullptr;
  p->trace_n = p->trace ? n_events : 0;
  p->trace_i = 0;
  return FFX_OK;
}

int64_t ffx_plan_trace_count(ffx_plan_t p) { return p ? p->trace_i : -1; }

int64_t ffx_workspace_bytes(ffx_plan_t p, int64_t batch) {
  if (!p || batch < 0) return -1;
  return batch * p->M * (int64_t)sizeof(float2);
}

int ffx_launches_per_call(ffx_plan_t p, int backward) {
  if (!p) return -1;
  if (p->many) return backward ? 2 * p->ndim : p->ndim;  // one persistent kernel per phase
  return backward ? 2 * p->ndim : p->ndim;
}

int ffx_expand(ffx_plan_t p, const void* psi0, int64_t batch, float* out_density, void* stream) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (batch < 0) return fail(FFX_EINVAL, "batch < 0");
  if (batch == 0) return FFX_OK;
  int rc;
  if ((rc = check_ptr(psi0, "psi0")) || (rc = check_ptr(out_density, "out_density"))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->many) {
    if (batch != 1) return fail(FFX_EINVAL, "a many-instance plan takes batch = 1");
    std::string err;
    rc = many_expand(p->many, psi0, out_density, nullptr, s, &err);
    return rc ? fail(rc, "%s", err.c_str()) : FFX_OK;
  }
  const float2* in = (const float2*)psi0;
  const int d = p->ndim;
  if (d > 1 && (rc = ensure_ws(p, batch))) return rc;
  float2* ws = (float2*)p->ws;
  for (int k = 0; k < d; ++k) {
    const int j = p->order[k];
    const bool last = (k == d - 1);
    rc = run_pass(p, j, false, k == 0 ? in : ws, nullptr, 0, last ? nullptr : ws,
                  last ? out_density : nullptr, last ? p->acc : 0, batch, s);
    if (rc) return rc;
  }
  return FFX_OK;
}

int ffx_expand_field(ffx_plan_t p, const void* psi0, int64_t batch, void* out_field, void* stream) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (batch < 0) return fail(FFX_EINVAL, "batch < 0");
  if (batch == 0) return FFX_OK;
  int rc;
  if ((rc = check_ptr(psi0, "psi0")) || (rc = check_ptr(out_field, "out_field"))) return rc;
  if (p->many) {
    if (batch != 1) return fail(FFX_EINVAL, "a many-instance plan takes batch = 1");
    std::string err;
    rc = many_expand(p->many, psi0, nullptr, out_field, (cudaStream_t)stream, &err);
    return rc ? fail(rc, "%s", err.c_str()) : FFX_OK;
  }
  return forward_field(p, (const float2*)psi0, batch, (float2*)out_field, (cudaStream_t)stream);
}

int ffx_expand_adjoint(ffx_plan_t p, const void* g_in, int64_t batch, void* g_out, void* stream) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (batch < 0) return fail(FFX_EINVAL, "batch < 0");
  if (batch == 0) return FFX_OK;
  int rc;
  if ((rc = check_ptr(g_in, "g_in")) || (rc = check_ptr(g_out, "g_out"))) return rc;
  if (p->many) return fail(FFX_EUNSUPPORTED, "ffx_expand_adjoint does not take a many-instance plan");
  const float2* cur = (const float2*)g_in;
  for (int k = p->ndim - 1; k >= 0; --k) {
    rc = run_pass(p, p->order[k], true, cur, nullptr, 0, (float2*)g_out, nullptr, 0, batch,
                  (cudaStream_t)stream);
    if (rc) return rc;
    cur = (const float2*)g_out;
  }
  return FFX_OK;
}

int ffx_expand_backward(ffx_plan_t p, const void* psi0, const float* grad_density, int64_t batch,
                        void* grad_psi0, void* stream) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (batch < 0) return fail(FFX_EINVAL, "batch < 0");
  if (batch == 0) return FFX_OK;
  int rc;
  if ((rc = check_ptr(psi0, "psi0")) || (rc = check_ptr(grad_density, "grad_density")) ||
      (rc = check_ptr(grad_psi0, "grad_psi0")))
    return rc;
  if (p->many) {
    if (batch != 1) return fail(FFX_EINVAL, "a many-instance plan takes batch = 1");
    std::string err;
    rc = many_backward(p->many, psi0, grad_density, grad_psi0, (cudaStream_t)stream, &err);
    return rc ? fail(rc, "%s", err.c_str()) : FFX_OK;
  }
  if ((rc = ensure_ws(p, batch))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  float2* ws = (float2*)p->ws;
  if ((rc = forward_field(p, (const float2*)psi0, batch, ws, s))) return rc;
  const float2* cur = ws;
  for (int k = p->ndim - 1; k >= 0; --k) {
    const bool first = (k == p->ndim - 1);
    rc = run_pass(p, p->order[k], true, cur, first ? grad_density : nullptr, first ? p->acc : 0,
                  (float2*)grad_psi0, nullptr, 0, batch, s);
    if (rc) return rc;
    cur = (const float2*)grad_psi0;
  }
  return FFX_OK;
}

}  // extern "C"
