// C ABI of the free-flight expansion library: plans, argument checks, the
// per-axis choice of form (paper / fold / dense, by cost model or by timing
// with an on-disk cache), workspace, and the sequence of per-axis passes.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/ffx.h"
#include "ffx_dense_lines.h"
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
  int form = FFX_FORM_FOLD;  // PAPER, FOLD or DENSE
  bool few = false;          // automatic dense form taken for fewer than kDenseFewLines lines per realization
  PassKernelInfo paper{}, foldk{}, adj{};
  int grid_paper = 0, grid_fold = 0, grid_adj = 0;
  float2* T = nullptr;   // dense map [N][N] (N <= kDenseMaxN)
  float2* TH = nullptr;  // its adjoint
  int grid_dense = 0, grid_dense_small = 0;
  unsigned char* tc_t[2] = {nullptr, nullptr};  // split tensor-core operands of T, T^H (ffx_tc.cu)
  unsigned char* bf_t[2] = {nullptr, nullptr};  // FFX_TC_BF16: the BF16 operand blocks (ffx_tc16.cu)
  unsigned char* ft_ts = nullptr;                 // N = 64: T's row-block slices for the fused tensor-core launch
  float2* img[2] = {nullptr, nullptr};                      // lines <= 64: shared-memory images of T, T^H
};

}  // namespace

void set_last_error_message(const char* msg) { g_last_error = msg ? msg : ""; }

}  // namespace ffx

using namespace ffx;

// Head of a plan's tensor-core allocation: device error counter (+0), the
// fused launch's grid-barrier counters (+64), its tile counters (+1024).
constexpr size_t kTcHeader = 1024 + kFusedTileFlags * sizeof(unsigned);

constexpr int kWs = 5, kWsSplit = 4;

struct ffx_plan_s {
  int ndim = 0;
  int64_t dims[3] = {1, 1, 1};
  int64_t M = 1;
  double t = 0;
  uint32_t flags = 0;
  int acc = 0;
  int device = 0;
  int sms = 1;
  Axis axis[3];
  int order[3] = {0, 1, 2};  // forward pass order
  // every axis has BF16 operand blocks and the driver makes TMA maps: large
  // forward calls may run as a BF16 chain (ffx_tc16.cu), whose order -- the
  // last axis first -- is then the plan's forward order
  int chain_bf16 = 0;
  void* tables = nullptr;
  void* dense_mem = nullptr;
  void* tc_mem = nullptr;    // split tensor-core operands + the fused launch's counters
  int* dev_err = nullptr;    // kernels that gave up on a bounded wait (device address)
  // the same counter in mapped page-locked host memory where the device has
  // native atomics to host memory (else NULL and dev_err is device memory):
  // the host reads it without a synchronization to report FFX_ETIMEOUT
  int* host_err = nullptr;
  int err_seen = 0;          // timeouts already reported through FFX_ETIMEOUT
  long long wait_limit = kCrossBlockSpin;  // polls of a wait on other blocks
  unsigned* grid_bar = nullptr;  // arrival counter of the fused kernel's grid barriers
  unsigned* tile_done = nullptr;  // per line tile: row blocks of the fused kernel's previous pass written
  int64_t fused = 0;             // largest batch whose forward calls run as one launch (ffx_fused.cu)
  int fused_grid = 0;
  int fused_tc = 0;              // ... on the tensor cores (every axis 64 points, automatic or tc form)
  int fused_tc_grid = 0;
  size_t fused_smem_bytes = 0;
  // workspace buffers, grown on demand: [0], [1] the passes' fields; [2] the
  // detector densities, or a positive-P pair's first field; [3] its second;
  // [4] the BF16 planes a per-axis BF16 pass splits its FP32 input into
  void* ws[kWs] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t ws_bytes[kWs] = {0, 0, 0, 0, 0};
  int64_t launches = 0;  // kernels the plan's calls have launched (ffx_plan_launch_count)
  void* stage[2] = {nullptr, nullptr};  // ffx_expand_host: device copies of the input and the densities
  size_t stage_bytes[2] = {0, 0};
  ManyPlan* many = nullptr;       // set for plans over many instances
  void* const* trace = nullptr;   // caller's cudaEvent_t array (profiling)
  int64_t trace_n = 0;
  int64_t trace_i = 0;
};

namespace {

// FFX_ETIMEOUT once per new timeout: the kernels count waits that ran out in
// the mapped word, which the host reads here without synchronizing (a launch
// that has not finished yet is seen by a later call).
int check_timeout(ffx_plan_s* p) {
  if (!p->host_err) return FFX_OK;
  const int now = *(volatile int*)p->host_err;
  if (now <= p->err_seen) return FFX_OK;
  p->err_seen = now;
  return fail(FFX_ETIMEOUT, "a kernel of this plan gave up on a bounded wait (%d so far): its output is not valid",
              now);
}

void axis_outer_inner(const ffx_plan_s* p, int j, int64_t* outer, int64_t* inner) {
  int64_t o = 1, in = 1;
  for (int i = 0; i < j; ++i) o *= p->dims[i];
  for (int i = j + 1; i < p->ndim; ++i) in *= p->dims[i];
  *outer = o;
  *inner = in;
}

int grid_for(const void* func, int threads, size_t smem, int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
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

// Device staging buffer k of ffx_expand_host, at least `need` bytes (grown
// like the workspace: cudaMalloc synchronizes the device the first time).
int ensure_stage(ffx_plan_s* p, int k, size_t need) {
  if (need <= p->stage_bytes[k]) return FFX_OK;
  if (p->stage[k]) {
    cudaFree(p->stage[k]);
    p->stage[k] = nullptr;
    p->stage_bytes[k] = 0;
  }
  cudaError_t e = cudaMalloc(&p->stage[k], need);
  if (e != cudaSuccess) {
    p->stage[k] = nullptr;
    cudaGetLastError();
    return fail(FFX_ENOMEM, "staging buffer of %zu bytes: %s", need, cudaGetErrorString(e));
  }
  p->stage_bytes[k] = need;
  return FFX_OK;
}

int ensure_ws(ffx_plan_s* p, int which, int64_t batch) {
  const size_t need = (size_t)batch * (size_t)p->M * sizeof(float2);
  if (need <= p->ws_bytes[which]) return FFX_OK;
  if (p->ws[which]) {
    cudaFree(p->ws[which]);  // synchronizes the device: queued users of the old buffer finish first
    p->ws[which] = nullptr;
    p->ws_bytes[which] = 0;
  }
  cudaError_t e = cudaMalloc(&p->ws[which], need);
  if (e != cudaSuccess) {
    p->ws[which] = nullptr;
    cudaGetLastError();
    return fail(FFX_ENOMEM, "workspace of %zu bytes: %s", need, cudaGetErrorString(e));
  }
  p->ws_bytes[which] = need;
  return FFX_OK;
}

bool inplace_ok(const Axis& ax) {
  return !((ax.form == FFX_FORM_DENSE || ax.form == FFX_FORM_TC) && ax.N > kDenseInPlaceMaxN);
}

bool tc_capable(const Axis& ax) { return dense_tc_supported(ax.N) && ax.tc_t[0] != nullptr; }

// The form whose kernel a pass over `lines` lines runs (explicit forms keep
// theirs).  An axis the plan's automatic choice gave the FP32 dense form
// moves to the tensor cores when the pass leaves the few-lines kernel and
// either its lines have at least 96 points (the FP32 tile kernel's K loop is
// the slower one there, measured down to a single 128-line tile) or it has at
// least 64 tensor-core items.  An axis that took the dense form only for its
// handful of lines per realization (a 1-D field) takes an FFT form instead
// when a call over many lines makes that cheaper (small lam).
double model_cost(const Axis& ax, int form, int64_t lines);
int call_form(const ffx_plan_s* p, const Axis& ax, int64_t lines);

// The tensor-core kernel moves 16-byte vectors; other pointers take the SIMT dense kernels.
bool tc_aligned(const void* in, const void* out_c, const void* out_d) {
  return ((uintptr_t)in & 15) == 0 && ((uintptr_t)out_c & 15) == 0 && ((uintptr_t)out_d & 15) == 0;
}

// Profiling: with a trace set (ffx_plan_trace), each launch sits between a
// pair of the caller's events; under stream capture they become event-record
// nodes of the graph.  trace_begin returns the record flags, ~0u when the
// trace is off or full.
unsigned trace_begin(ffx_plan_s* p, cudaStream_t stream) {
  if (!(p->trace && p->trace_i + 2 <= p->trace_n)) return ~0u;
  unsigned rec_flags = cudaEventRecordDefault;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    rec_flags = cudaEventRecordExternal;
  cudaEventRecordWithFlags((cudaEvent_t)p->trace[p->trace_i], stream, rec_flags);
  return rec_flags;
}
void trace_end(ffx_plan_s* p, cudaStream_t stream, unsigned rec_flags) {
  if (rec_flags == ~0u) return;
  cudaEventRecordWithFlags((cudaEvent_t)p->trace[p->trace_i + 1], stream, rec_flags);
  p->trace_i += 2;
}

// A pass of a BF16 chain (forward only): its lines are contiguous (the
// previous pass wrote them transposed, or the axis is the last one), read
// from BF16 planes (in_bf) or the FP32 field `in`; its output goes to BF16
// planes (out_bf) or the caller's buffers, transposed: point n' of line rho
// at n' (M / N) + rho of its realization.  plane: points per plane.
struct ChainIo {
  const uint32_t* in_bf;
  uint32_t* out_bf;
  int64_t plane;
};

// Launch one pass of axis j (forward or adjoint) with the axis's form, or,
// with `io`, a pass of a BF16 chain.
int run_axis(ffx_plan_s* p, int j, bool adjoint, const float2* in, const float* grad, int grad_shared,
             float2* out_c, float* out_d, int acc, int64_t batch, cudaStream_t stream, const ChainIo* io = nullptr) {
  const Axis& ax = p->axis[j];
  int64_t outer, inner;
  axis_outer_inner(p, j, &outer, &inner);
  if (io) {
    outer = p->M / ax.N;
    inner = 1;
  }
  const unsigned rec_flags = trace_begin(p, stream);
  cudaError_t e;
  const int64_t lines = acc ? outer * inner : batch * outer * inner;
  const int cform = call_form(p, ax, lines);  // this call's form
  if (cform == FFX_FORM_TC && tc_aligned(in, out_c, out_d)) {
    DenseArgs d;
    std::memset(&d, 0, sizeof(d));
    d.in = in;
    d.grad = grad;
    d.grad_shared = grad_shared;
    d.out_c = out_c;
    d.out_d = out_d;
    d.outer = outer;
    d.inner = inner;
    d.M = p->M;
    d.batch = batch;
    d.acc = acc;
    d.unsplit = (p->flags & FFX_TC_UNSPLIT) ? 1 : 0;
    d.ncols = acc ? outer * inner : batch * outer * inner;
    d.N = ax.N;
    const int64_t items = dense_tc_tiles(ax.N, d.ncols);
    int64_t grid = items;
    if (grid > p->sms) grid = p->sms;
    if (grid < 1) grid = 1;
    // BF16 operands on the streaming kernel's passes; the tensor-memory
    // kernels (64-point plain passes with at most four items per block) keep
    // split TF32
    const bool tm64 = ax.N == 64 && !acc && !grad && items <= 4 * grid;
    if (io) {
      if (!ax.bf_t[adjoint ? 1 : 0] || tm64 || grad)
        return fail(FFX_EUNSUPPORTED, "internal: a BF16 chain pass of axis %d without the BF16 kernel", j);
      d.in_bf = io->in_bf;
      d.out_bf = io->out_bf;
      d.bf_plane = io->plane;
      d.oouter = 1;
      d.oinner = outer;
    } else if (ax.bf_t[0] && !tm64 && !grad && inner == 1) {
      // contiguous FP32 lines: split into BF16 planes first (an HBM-bound
      // pass), so that the pass loads its operands straight into the tensor
      // cores' layout instead of converting them on the way
      int rc = ensure_ws(p, kWsSplit, batch);
      if (rc) return rc;
      const int64_t plane = batch * p->M;
      e = launch_bf16_split(in, (uint32_t*)p->ws[kWsSplit], plane, plane, d.unsplit, p->sms, stream);
      if (e != cudaSuccess) return cuda_fail(e, "BF16 split of a pass input");
      ++p->launches;
      d.in_bf = (const uint32_t*)p->ws[kWsSplit];
      d.bf_plane = plane;
      d.in = nullptr;
    }
    if (ax.bf_t[0] && !tm64)
      e = launch_dense_bf16(d, ax.bf_t[adjoint ? 1 : 0], p->dev_err, (int)grid, stream);
    else
      e = launch_dense_tc(d, ax.tc_t[adjoint ? 1 : 0], p->dev_err, (int)grid, stream);
  } else if (io) {
    return fail(FFX_EUNSUPPORTED, "internal: a BF16 chain pass of axis %d off the tensor cores", j);
  } else if (cform == FFX_FORM_DENSE || cform == FFX_FORM_TC) {
    DenseArgs d;
    std::memset(&d, 0, sizeof(d));
    d.A = adjoint ? ax.TH : ax.T;
    d.in = in;
    d.grad = grad;
    d.grad_shared = grad_shared;
    d.out_c = out_c;
    d.out_d = out_d;
    d.outer = outer;
    d.inner = inner;
    d.M = p->M;
    d.batch = batch;
    d.acc = acc;
    d.ncols = acc ? outer * inner : batch * outer * inner;
    d.N = ax.N;
    d.Aimg = adjoint ? ax.img[1] : ax.img[0];
    d.err = p->dev_err;
    const bool in_place = (const void*)in == (const void*)out_c;
    if (batch * outer * inner < kDenseFewLines && !in_place) {
      e = launch_dense_lines(d, stream);
    } else if (ax.N <= kDenseInPlaceMaxN) {
      int64_t grid = dense_small_tiles(ax.N, d.ncols);
      if (grid > ax.grid_dense_small) grid = ax.grid_dense_small;
      if (grid < 1) grid = 1;
      e = launch_dense_small(d, (int)grid, stream);
    } else {
      int64_t grid = dense_tiles(ax.N, d.ncols);
      if (grid > ax.grid_dense) grid = ax.grid_dense;
      if (grid < 1) grid = 1;
      e = launch_dense(d, (int)grid, stream);
    }
  } else {
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
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
    const int kind = adjoint ? KIND_ADJ_FOLD : (cform == FFX_FORM_PAPER ? KIND_FWD_PAPER : KIND_FWD_FOLD);
    if (conv_supported(ax.N, ax.lam, acc, kind)) {
      // one or two terms on lines of 16, 64, 256 or 1024 points: the kernel
      // with four-step line transforms in registers
      e = launch_conv(a, kind, ax.N, p->sms, stream);
    } else {
      const PassKernelInfo& info = adjoint ? ax.adj : (cform == FFX_FORM_PAPER ? ax.paper : ax.foldk);
      const int capacity = adjoint ? ax.grid_adj : (cform == FFX_FORM_PAPER ? ax.grid_paper : ax.grid_fold);
      // The split depends on one realization's lines only, so a realization's
      // result does not depend on the batch it came in (bitwise).
      a.qg = choose_qg(info, outer * inner, ax.lam, capacity);
      const int lines = pass_lines_per_tile(info, a.qg);
      const int64_t ntiles = (a.nlines + lines - 1) / lines;
      int64_t grid = capacity;
      if (grid > ntiles) grid = ntiles;
      if (grid < 1) grid = 1;
      e = info.launch(a, (int)grid, stream);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "pass launch");
  ++p->launches;
  trace_end(p, stream, rec_flags);
  return FFX_OK;
}

// Output buffers of a chain of passes (axes[0..n-1]) whose last pass must
// write `final`: a pass that cannot run in place writes the other buffer of
// the pair (final, alt).  outs[0] is where the first pass writes.  Returns
// whether `alt` is used.
bool plan_chain(const ffx_plan_s* p, const int* axes, int n, float2* final, float2* alt, float2** outs) {
  bool uses_alt = false;
  float2* cur = final;
  for (int k = n - 1; k >= 0; --k) {
    outs[k] = cur;
    if (cur == alt) uses_alt = true;
    if (k > 0 && !inplace_ok(p->axis[axes[k]])) cur = (cur == final) ? alt : final;
  }
  return uses_alt;
}

// Whether a forward call over `batch` realizations runs as a BF16 chain:
// the plan allows it, and every pass takes the BF16 streaming kernel in this
// call (the per-axis passes' choice: tensor-core form, not the 64-point
// tensor-memory kernel) with 16-byte aligned pointers.
bool bf16_chain_ok(const ffx_plan_s* p, int64_t batch, const void* in, const void* out_c, const void* out_d) {
  if (!p->chain_bf16 || p->many || !tc_aligned(in, out_c, out_d)) return false;
  for (int r = 0; r < p->ndim; ++r) {
    const Axis& ax = p->axis[p->order[r]];
    const bool acc = r == p->ndim - 1 && out_d && p->acc;
    const int64_t lines = (acc ? 1 : batch) * (p->M / ax.N);
    if (call_form(p, ax, lines) != FFX_FORM_TC) return false;
    const int64_t items = dense_tc_tiles(ax.N, lines);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(items, p->sms));
    if (ax.N == 64 && !acc && items <= 4 * grid) return false;
  }
  return true;
}

// Every axis has the BF16 blocks of T_j^H too (adjoint chains).
bool bf16_adjoint_ok(const ffx_plan_s* p) {
  for (int r = 0; r < p->ndim; ++r)
    if (!p->axis[r].bf_t[1]) return false;
  return true;
}

// The forward map of a batch as a BF16 chain: the input split into BF16
// planes in ws[1] (head plane, then tail plane: 8 bytes a point, the size of
// a complex64 field), then the passes in the plan's order (the last axis
// first), each reading planes and writing planes (ws[0], ws[1], ...), the
// last one the caller's field (out_c) or densities (out_d, summed over the
// batch with FFX_ACCUMULATE).  `in` is read by the split alone, so out_c may
// equal it; it must not be ws[1].
int chain_bf16(ffx_plan_s* p, const float2* in, int64_t batch, float2* out_c, float* out_d, cudaStream_t s) {
  const int d = p->ndim;
  int rc;
  if ((rc = ensure_ws(p, 0, batch)) || (rc = ensure_ws(p, 1, batch))) return rc;
  const int64_t plane = batch * p->M;
  const int unsplit = (p->flags & FFX_TC_UNSPLIT) ? 1 : 0;
  const unsigned rec = trace_begin(p, s);
  cudaError_t e = launch_bf16_split(in, (uint32_t*)p->ws[1], plane, plane, unsplit, p->sms, s);
  if (e != cudaSuccess) return cuda_fail(e, "BF16 split of the input");
  ++p->launches;
  trace_end(p, s, rec);
  const uint32_t* cur_bf = (const uint32_t*)p->ws[1];
  for (int r = 0; r < d; ++r) {
    const bool last = r == d - 1;
    ChainIo io;
    io.in_bf = cur_bf;
    io.out_bf = last ? nullptr : (uint32_t*)p->ws[r & 1];
    io.plane = plane;
    rc = run_axis(p, p->order[r], false, nullptr, nullptr, 0, last ? out_c : nullptr, last ? out_d : nullptr,
                  last && out_d ? p->acc : 0, batch, s, &io);
    if (rc) return rc;
    cur_bf = io.out_bf;
  }
  return FFX_OK;
}

// The adjoint half of a backward call as a BF16 chain: 2 grad * field split
// into BF16 planes in ws[1], then the adjoint passes in the chain's order
// (T_j^H along the last axis first; the axes' factors commute), planes
// between them in ws[0] and ws[1] as in chain_bf16, the last pass writing
// `out`.  `field` is read by the split alone (it may be ws[0]).
int chain_bf16_adjoint(ffx_plan_s* p, const float2* field, const float* grad, int grad_shared, int64_t batch,
                       float2* out, cudaStream_t s) {
  const int d = p->ndim;
  int rc;
  if ((rc = ensure_ws(p, 0, batch)) || (rc = ensure_ws(p, 1, batch))) return rc;
  const int64_t plane = batch * p->M;
  const int unsplit = (p->flags & FFX_TC_UNSPLIT) ? 1 : 0;
  const unsigned rec = trace_begin(p, s);
  cudaError_t e = launch_bf16_split_grad(field, grad, grad_shared, p->M, (uint32_t*)p->ws[1], plane, plane, unsplit,
                                         p->sms, s);
  if (e != cudaSuccess) return cuda_fail(e, "BF16 split of the gradient factors");
  ++p->launches;
  trace_end(p, s, rec);
  const uint32_t* cur_bf = (const uint32_t*)p->ws[1];
  for (int r = 0; r < d; ++r) {
    const bool last = r == d - 1;
    ChainIo io;
    io.in_bf = cur_bf;
    io.out_bf = last ? nullptr : (uint32_t*)p->ws[r & 1];
    io.plane = plane;
    rc = run_axis(p, p->order[r], true, nullptr, nullptr, 0, last ? out : nullptr, nullptr, 0, batch, s, &io);
    if (rc) return rc;
    cur_bf = io.out_bf;
  }
  return FFX_OK;
}

// Run a chain of passes (forward or adjoint) from `in` (read only) into
// `out`; ws[alt_ws] serves as the alternate buffer and ws[1 - alt_ws] as the
// spare copy of the input when an in-place call meets a pass that cannot run
// in place.  The first pass may form 2 * grad * in on load.
int chain_into(ffx_plan_s* p, const int* axes, bool adjoint, const float2* in, const float* grad,
               int grad_shared, int64_t batch, float2* out, int alt_ws, cudaStream_t s) {
  const int d = p->ndim;
  // forward fields take the BF16 chain (its planes live in ws[0] and ws[1])
  // unless the input is ws[1], which its split writes, or the output is the
  // buffer its last pass reads
  if (!adjoint && !grad && axes == p->order && (const void*)in != p->ws[1] && (void*)out != p->ws[(d - 2) & 1] &&
      bf16_chain_ok(p, batch, in, out, nullptr))
    return chain_bf16(p, in, batch, out, nullptr, s);
  float2* outs[3];
  float2* probe[3];
  const bool need_alt = plan_chain(p, axes, d, out, (float2*)(uintptr_t)8, probe);
  float2* alt = nullptr;
  int rc;
  if (need_alt) {
    if ((rc = ensure_ws(p, alt_ws, batch))) return rc;
    alt = (float2*)p->ws[alt_ws];
  }
  plan_chain(p, axes, d, out, alt, outs);
  const float2* cur = in;
  if (in == outs[0] && !inplace_ok(p->axis[axes[0]])) {
    const int spare = 1 - alt_ws;
    if ((rc = ensure_ws(p, spare, batch))) return rc;
    cudaError_t e =
        cudaMemcpyAsync(p->ws[spare], in, (size_t)batch * p->M * sizeof(float2), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "input copy");
    cur = (const float2*)p->ws[spare];
  }
  for (int r = 0; r < d; ++r) {
    rc = run_axis(p, axes[r], adjoint, cur, r == 0 ? grad : nullptr, r == 0 ? grad_shared : 0, outs[r], nullptr,
                  0, batch, s);
    if (rc) return rc;
    cur = outs[r];
  }
  return FFX_OK;
}

// ---------------------------------------------------------------------------
// one-launch forward map of small lattices
// ---------------------------------------------------------------------------

// A plan fuses its forward passes when it has at least two axes, every axis
// takes a dense form with at most 64 points (its shared-memory image exists),
// the device runs cooperative launches, and one block of the fused kernel fits
// on every SM; calls with batches up to p->fused use it.  FFX_UNFUSED keeps
// the per-axis launches.
int call_form(const ffx_plan_s* p, const Axis& ax, int64_t lines) {
  if (ax.form == FFX_FORM_TC) return tc_capable(ax) ? FFX_FORM_TC : FFX_FORM_DENSE;
  if ((p->flags & FFX_FORM_MASK) != FFX_FORM_AUTO) return ax.form;
  if (ax.form == FFX_FORM_PAPER || ax.form == FFX_FORM_FOLD) {
    // An FFT-form axis (small lam) moves to the tensor cores when the call
    // fills at least 64 of their items and the dense map on them costs less:
    // on full calls they reach 8N / 3.5 in the cost model's units (measured
    // 3.4-4.3 for N = 64 ... 1024), where the model's plan-time figure is
    // made for a realization's lines alone.
    if (tc_capable(ax) && dense_tc_tiles(ax.N, lines) >= 64 &&
        8.0 * ax.N / 3.5 < model_cost(ax, ax.form, lines))
      return FFX_FORM_TC;
    return ax.form;
  }
  if (ax.form != FFX_FORM_DENSE || lines < kDenseFewLines) return ax.form;
  int k = FFX_FORM_DENSE;
  if (tc_capable(ax) && (ax.N >= 96 || dense_tc_tiles(ax.N, lines) >= 64)) k = FFX_FORM_TC;
  if (ax.few) {
    double best = model_cost(ax, k, lines);
    for (int c : {FFX_FORM_FOLD, FFX_FORM_PAPER}) {
      const double cc = model_cost(ax, c, lines);
      if (cc < best) {
        best = cc;
        k = c;
      }
    }
  }
  return k;
}

int plan_fusion(ffx_plan_s* p) {
  p->fused = 0;
  if (p->ndim < 2 || (p->flags & (FFX_UNFUSED | FFX_TC_UNSPLIT)) || !p->grid_bar) return FFX_OK;
  int Ns[3];
  for (int k = 0; k < p->ndim; ++k) {
    const Axis& ax = p->axis[p->order[k]];
    if (!(ax.form == FFX_FORM_DENSE || ax.form == FFX_FORM_TC) || !ax.img[0] || ax.N > kDenseInPlaceMaxN)
      return FFX_OK;
    Ns[k] = ax.N;
  }
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, p->device);
  if (!coop) return FFX_OK;
  const size_t smem = fused_smem(Ns, p->ndim);
  cudaError_t e = cudaFuncSetAttribute(fused_func(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_func(), fused_threads(), smem);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return FFX_OK;
  }
  // Batches whose first pass has at most two 32-line tiles per block: beyond
  // that the per-axis kernels (several blocks per SM) keep the ALUs busier.
  const int64_t tiles = (p->M / Ns[0] + 31) / 32;
  p->fused = std::max<int64_t>(1, 2 * (int64_t)p->sms / tiles);
  // nor past the batch whose per-axis passes all move to the tensor cores
  for (int64_t b = 2; b <= p->fused; ++b) {
    bool all_tc = true;
    for (int k = 0; k < p->ndim; ++k)
      all_tc = all_tc && call_form(p, p->axis[p->order[k]], b * (p->M / Ns[k])) == FFX_FORM_TC;
    if (all_tc) {
      p->fused = b - 1;
      break;
    }
  }
  p->fused_grid = p->sms;  // one block per SM (every block is resident: cooperative launch)
  p->fused_smem_bytes = smem;
  // Every axis 64 points with its tensor-core slices, and a form that allows
  // the tensor cores: the fused launch runs the products on them.
  const uint32_t form = p->flags & FFX_FORM_MASK;
  bool tc_ok = (form == FFX_FORM_AUTO || form == FFX_FORM_TC) && p->sms >= 4;
  for (int k = 0; k < p->ndim; ++k) tc_ok = tc_ok && p->axis[k].N == 64 && p->axis[k].ft_ts;
  if (tc_ok) {
    int tc_per_sm = 0;
    if (fused_tc_prepare(&tc_per_sm) == cudaSuccess && tc_per_sm >= 1) {
      p->fused_tc = 1;
      p->fused_tc_grid = (p->sms / 4) * 4;  // row blocks are fixed per block: a multiple of 4
    } else {
      cudaGetLastError();
    }
  }
  return FFX_OK;
}

// The forward map as one launch, passes in the order `axes`: pass k reads
// `in` (k = 0) or the workspace, writes the workspace, and the last pass
// writes out_c, or out_d (a density), or out_col (the density summed along the
// last pass's axis); the last two summed over the batch with FFX_ACCUMULATE.
// The FP32 launch owns whole lines per tile and runs the middle passes in
// place; the tensor-core launch splits a line's rows over four blocks, so its
// passes alternate between two workspaces.
int run_fused(ffx_plan_s* p, const int* axes, const float2* in, float2* out_c, float* out_d, float* out_col,
              int64_t batch, cudaStream_t stream) {
  int rc;
  const bool tc = p->fused_tc && !out_col && ((uintptr_t)in & 15) == 0;
  if ((rc = ensure_ws(p, 0, batch))) return rc;
  if (tc && p->ndim > 2 && (rc = ensure_ws(p, 1, batch))) return rc;
  float2* ws[2] = {(float2*)p->ws[0], tc && p->ndim > 2 ? (float2*)p->ws[1] : (float2*)p->ws[0]};
  FusedArgs a;
  std::memset(&a, 0, sizeof(a));
  a.npass = p->ndim;
  a.M = p->M;
  a.batch = batch;
  a.bar = p->grid_bar;
  a.err = p->dev_err;
  a.spin = p->wait_limit;
  int64_t off = 0;
  for (int k = 0; k < p->ndim; ++k) {
    const int j = axes[k];
    const Axis& ax = p->axis[j];
    const bool last = k == p->ndim - 1;
    FusedPass& P = a.pass[k];
    axis_outer_inner(p, j, &P.outer, &P.inner);
    P.in = k == 0 ? in : ws[(k - 1) & 1];
    P.out_c = last ? out_c : ws[k & 1];
    P.out_d = last ? out_d : nullptr;
    P.out_col = last ? out_col : nullptr;
    P.col_scale = (float)(ax.lam * ax.dx);
    P.acc = (last && (out_d || out_col)) ? p->acc : 0;
    P.ncols = P.acc ? P.outer * P.inner : batch * P.outer * P.inner;
    P.N = ax.N;
    P.img = ax.img[0];
    P.img_off = (int)off;
    off += (int64_t)ax.N * fused_img_stride();
  }
  a.img_floats2 = off;
  const bool traced = p->trace && p->trace_i + 2 <= p->trace_n;
  unsigned rec_flags = cudaEventRecordDefault;
  if (traced) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      rec_flags = cudaEventRecordExternal;
    cudaEventRecordWithFlags((cudaEvent_t)p->trace[p->trace_i], stream, rec_flags);
  }
  cudaError_t e;
  a.local_pass = -1;
  if (tc) {
    for (int k = 0; k < p->ndim; ++k) a.ts[k] = p->axis[axes[k]].ft_ts;
    // A pass may follow the previous one tile by tile when the two passes'
    // line tiles cover the same points: every pass of a 2-D lattice (a tile
    // is two realizations), and two passes of a 3-D lattice that both run
    // along axes 1 and 2 (a tile is two values of axis 0 of one realization).
    // Not into an accumulating pass over several realizations (its tile
    // gathers every realization).
    a.tile_done = p->tile_done;
    for (int k = 1; k < p->ndim; ++k) {
      const bool same = p->ndim == 2 || (axes[k - 1] != 0 && axes[k] != 0);
      const FusedPass& P = a.pass[k];
      const bool gathers = P.acc && batch > 1;
      if (same && !gathers && (P.ncols + 127) / 128 <= kFusedTileFlags) a.local_pass = k;
    }
    e = launch_fused_tc(a, p->fused_tc_grid, stream);
  } else {
    e = launch_fused(a, p->fused_grid, p->fused_smem_bytes, stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "fused launch");
  ++p->launches;
  if (traced) {
    cudaEventRecordWithFlags((cudaEvent_t)p->trace[p->trace_i + 1], stream, rec_flags);
    p->trace_i += 2;
  }
  return FFX_OK;
}

// ---------------------------------------------------------------------------
// per-axis form: cost model, timing, cache
// ---------------------------------------------------------------------------

// Relative cost per point of one axis pass (FP32 flops over the fraction of
// the FP32 peak each form was measured to reach on GB300).
// `lines` = lines of one realization along the axis.  The tensor-core kernel
// tiles lines by 128, so fewer lines leave it latency-bound.  Fewer than
// kDenseFewLines lines (a 1-D field) take the dense form: its few-lines kernel
// spreads the rows of T over N / 8 blocks, while the FFT forms run each line's
// transforms in sequence inside one block.
double model_cost(const Axis& ax, int form, int64_t lines) {
  const double N = ax.N, lg = std::log2(N), lam = ax.lam;
  // the one- and two-term kernel (ffx_conv.cu), measured on full passes at
  // 136-150 (lam = 1) and 180-253 (lam = 2) in these units, near the HBM
  // bound of ~100; the paper form takes it at lam = 1 only, one unit dearer
  // so that ties go to the fold form
  if (form == FFX_FORM_FOLD && conv_supported(ax.N, ax.lam, 0, KIND_FWD_FOLD)) return ax.lam == 1 ? 140 : 230;
  if (form == FFX_FORM_PAPER && conv_supported(ax.N, ax.lam, 0, KIND_FWD_PAPER)) return 141;
  switch (form) {
    case FFX_FORM_PAPER: return lam * (10 * lg + 20) / 0.18;
    case FFX_FORM_FOLD: return (lam * (5 * lg + 14) + 5 * lg) / (N >= 256 ? 0.16 : 0.11);
    // the tensor-core form runs 3x the real flops at ~6x the FP32 rate
    // (measured 1.9-2.3 in these units for N = 64 .. 1024 on full passes);
    // 64-point axes stay dense at plan time and move to the tensor cores per
    // call when the call is large (see call_form)
    case FFX_FORM_TC:
      if (lines < 128) return 1e30;
      return N < 128 ? 8 * N / 0.40 : 8 * N / 2.0;
    default:
      if (lines < kDenseFewLines) return 0;
      return 8 * N / 0.45;
  }
}

std::mutex g_cache_mutex;

std::string cache_key(const char* dev, const Axis& ax, int64_t outer, int64_t inner) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|N=%d|lam=%d|outer=%lld|inner=%lld", dev, ax.N, ax.lam, (long long)outer,
           (long long)inner);
  return buf;
}

// Cache lines (JSON, one object per line):
//   {"key": "...", "form": "dense", "ms": [paper, fold, dense, tc]}
// The last line for a key wins.
int cache_lookup(const std::string& key) {
  const char* path = std::getenv("FFX_TUNE_CACHE");
  if (!path || !*path) return -1;
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  FILE* f = std::fopen(path, "r");
  if (!f) return -1;
  char line[2048];
  int form = -1;
  const std::string want = "\"key\": \"" + key + "\"";
  while (std::fgets(line, sizeof(line), f)) {
    if (!std::strstr(line, want.c_str())) continue;
    if (std::strstr(line, "\"form\": \"paper\"")) form = FFX_FORM_PAPER;
    if (std::strstr(line, "\"form\": \"fold\"")) form = FFX_FORM_FOLD;
    if (std::strstr(line, "\"form\": \"dense\"")) form = FFX_FORM_DENSE;
    if (std::strstr(line, "\"form\": \"tc\"")) form = FFX_FORM_TC;
  }
  std::fclose(f);
  return form;
}

void cache_store(const std::string& key, int form, const double* ms) {
  const char* path = std::getenv("FFX_TUNE_CACHE");
  if (!path || !*path) return;
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  const char* names[] = {"", "paper", "fold", "dense", "tc"};
  std::fprintf(f, "{\"key\": \"%s\", \"form\": \"%s\", \"ms\": [%.6g, %.6g, %.6g, %.6g]}\n", key.c_str(),
               names[form], ms[0], ms[1], ms[2], ms[3]);
  std::fclose(f);
}

// Time the candidate forms of axis j on a batch of one (ws[0] -> ws[1]).
int time_forms(ffx_plan_s* p, int j, cudaStream_t s, double* ms) {
  Axis& ax = p->axis[j];
  const int saved = ax.form;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = FFX_OK;
  for (int f = FFX_FORM_PAPER; f <= FFX_FORM_TC && rc == FFX_OK; ++f) {
    ms[f - 1] = 1e30;
    if (f == FFX_FORM_DENSE && !ax.T) continue;
    if (f == FFX_FORM_TC && !tc_capable(ax)) continue;
    ax.form = f;
    float best = 1e30f;
    for (int rep = 0; rep < 6 && rc == FFX_OK; ++rep) {
      cudaEventRecord(e0, s);
      rc = run_axis(p, j, false, (const float2*)p->ws[0], nullptr, 0, (float2*)p->ws[1], nullptr, 0, 1, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0 && t < best) best = t;  // the first run warms up
    }
    ms[f - 1] = best;
  }
  ax.form = saved;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// Build the dense maps T_j and T_j^H: the fold-form pass applied to the N
// unit vectors (rows of the identity), then transposed / conjugated.
int build_dense(ffx_plan_s* p, int j, float2* T, float2* TH, float2* scratch, cudaStream_t s) {
  Axis& ax = p->axis[j];
  const int N = ax.N;
  float2* I = scratch;
  float2* O = scratch + (size_t)N * N;
  cudaError_t e = launch_identity(I, N, s);
  if (e != cudaSuccess) return cuda_fail(e, "identity");
  PassArgs a;
  std::memset(&a, 0, sizeof(a));
  a.in = I;
  a.out_c = O;
  a.outer = 1;
  a.inner = 1;
  a.M = N;
  a.batch = N;
  a.nlines = N;
  a.lam = ax.lam;
  a.g = ax.g;
  a.Np = ax.Np;
  a.tab.P = ax.P;
  a.tab.K = ax.K;
  a.tab.Kf = ax.Kf;
  a.tab.F = ax.F;
  a.tab.tw = ax.tw;
  a.tab.fold = ax.fold;
  a.qg = choose_qg(ax.foldk, N, ax.lam, ax.grid_fold);
  const int lines = pass_lines_per_tile(ax.foldk, a.qg);
  int64_t grid = (N + lines - 1) / lines;
  if (grid > ax.grid_fold) grid = ax.grid_fold;
  e = ax.foldk.launch(a, (int)grid, s);
  if (e == cudaSuccess) e = launch_dense_build(O, T, TH, N, s);
  if (e != cudaSuccess) return cuda_fail(e, "dense map");
  ax.T = T;
  ax.TH = TH;
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
    case FFX_ETIMEOUT: return "a bounded device wait ran out";
    default: return "unknown error";
  }
}

const char* ffx_last_error(void) { return g_last_error.c_str(); }

int ffx_supported_length(int64_t n) { return supported_length(n) ? 1 : 0; }

int ffx_plan(ffx_plan_t* out, int ndim, const int64_t* dims, const double* spacing, double t,
             const int32_t* magnification, const double* a, const double* abar, uint32_t flags) {
  return ffx_plan_dispersion(out, ndim, dims, spacing, t, magnification, a, abar, nullptr, flags);
}

int ffx_plan_dispersion(ffx_plan_t* out, int ndim, const int64_t* dims, const double* spacing, double t,
                        const int32_t* magnification, const double* a, const double* abar,
                        const double* const* omega, uint32_t flags) {
  g_last_error.clear();
  if (!out) return fail(FFX_EINVAL, "out is NULL");
  *out = nullptr;
  if (ndim < 1 || ndim > 3) return fail(FFX_EINVAL, "ndim must be 1..3, got %d", ndim);
  if (!dims || !spacing || !magnification) return fail(FFX_EINVAL, "dims/spacing/magnification is NULL");
  if (!std::isfinite(t)) return fail(FFX_EINVAL, "t must be finite");
  const uint32_t known =
      FFX_FORM_MASK | FFX_ACCUMULATE | FFX_TUNE | FFX_UNFUSED | FFX_TC_UNSPLIT | FFX_TC_BF16 | FFX_TC_TF32;
  if (flags & ~known) return fail(FFX_EINVAL, "unknown flag bits 0x%x", flags & ~known);
  const uint32_t form = flags & FFX_FORM_MASK;
  if (form > FFX_FORM_TC) return fail(FFX_EINVAL, "unknown form %u", form);
  if ((flags & FFX_TC_UNSPLIT) && form != FFX_FORM_TC)
    return fail(FFX_EINVAL, "FFX_TC_UNSPLIT needs FFX_FORM_TC");
  if ((flags & FFX_TC_BF16) && form != FFX_FORM_TC && form != FFX_FORM_AUTO)
    return fail(FFX_EINVAL, "FFX_TC_BF16 needs FFX_FORM_TC or FFX_FORM_AUTO");
  if ((flags & FFX_TC_TF32) && (flags & FFX_TC_BF16)) return fail(FFX_EINVAL, "FFX_TC_TF32 and FFX_TC_BF16 exclude each other");
  // BF16 operands on the streaming tensor-core passes: asked for, or the
  // automatic form's choice (split BF16 meets the FP32 bar and runs faster
  // than split TF32) unless TF32 or the unsplit variant is asked for
  const bool bf16_ops = (flags & FFX_TC_BF16) ||
                        (form == FFX_FORM_AUTO && !(flags & (FFX_TC_TF32 | FFX_TC_UNSPLIT)));
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
    if (omega && omega[j]) {
      const int64_t lN = (int64_t)magnification[j] * dims[j];
      for (int64_t u = 0; u < lN; ++u)
        if (!std::isfinite(omega[j][u])) return fail(FFX_EINVAL, "omega[%d][%lld] is not finite", j, (long long)u);
    }
    if ((form == FFX_FORM_DENSE || form == FFX_FORM_TC) && dims[j] > kDenseMaxN)
      return fail(FFX_EUNSUPPORTED, "the dense form takes lines up to %d points (axis %d has %lld)",
                  kDenseMaxN, j, (long long)dims[j]);
    M *= dims[j];
  }

  ffx_plan_s* p = new (std::nothrow) ffx_plan_s();
  if (!p) return fail(FFX_ENOMEM, "host allocation failed");
  p->ndim = ndim;
  p->t = t;
  p->flags = flags;
  p->acc = (flags & FFX_ACCUMULATE) ? 1 : 0;
  p->M = M;
  cudaGetDevice(&p->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  p->sms = sms > 0 ? sms : 1;
  for (int j = 0; j < ndim; ++j) p->dims[j] = dims[j];
  // Forward order: longest lines first, so the last pass (which may sum the
  // ensemble and then has only one realization's lines to spread over the
  // GPU) runs on the axis with the most lines.
  for (int j = 0; j < ndim; ++j) p->order[j] = j;
  for (int i = 0; i < ndim; ++i)
    for (int k = i + 1; k < ndim; ++k)
      if (p->dims[p->order[k]] > p->dims[p->order[i]]) std::swap(p->order[i], p->order[k]);

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
  std::vector<int> fold_h;
  for (int j = 0; j < ndim && rc == FFX_OK; ++j) {
    Axis& ax = p->axis[j];
    const int N = (int)dims[j];
    const int lam = magnification[j];
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

    // phase constants in turns (hbar = m = 1): s = (abar - a)/dx, tau = pi t / L^2;
    // another spectrum (Sec. 7) replaces the tau terms by a per-wavevector table
    const double sv = (ax.abar - ax.a) / ax.dx;
    const bool disp = omega && omega[j];
    const double tau = disp ? 0.0 : M_PI * t / (L * L);
    uint64_t* disp_d = nullptr;
    if (disp) {
      std::vector<uint64_t> disp_h((size_t)lam * N);
      for (size_t u = 0; u < disp_h.size(); ++u) disp_h[u] = frac_fx(-t * omega[j][u] / (2.0 * M_PI));
      e = cudaMalloc(&disp_d, disp_h.size() * sizeof(uint64_t));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(disp_d, disp_h.data(), disp_h.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // disp_h goes out of scope
      if (e != cudaSuccess) {
        if (disp_d) cudaFree(disp_d);
        cudaGetLastError();
        rc = fail(FFX_ENOMEM, "dispersion table: %s", cudaGetErrorString(e));
        break;
      }
    }
    e = launch_fill_tables(N, lam, frac_fx(sv / N), frac_fx(tau), frac_fx(2.0 * tau / lam),
                           frac_fx(sv / ((double)lam * N)), frac_fx(tau / ((double)lam * lam)), disp_d, ax.P,
                           ax.K, ax.Kf, ax.F, ax.tw, s);
    if (disp_d) {
      const cudaError_t e2 = cudaStreamSynchronize(s);
      cudaFree(disp_d);
      if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "table fill");
      break;
    }
    // fold table: m0 with (lam/g) m0 = r/g (mod N/g) for g | r, else -1
    const int64_t inv = inv_mod((lam / ax.g) % ax.Np, ax.Np);
    fold_h.assign(N, -1);
    for (int r = 0; r < N; ++r)
      if (r % ax.g == 0) fold_h[r] = (int)(((int64_t)(r / ax.g) * inv) % ax.Np);
    e = cudaMemcpyAsync(ax.fold, fold_h.data(), sizeof(int) * N, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // fold_h is reused
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "fold table upload");
      break;
    }
    if (!find_pass_kernel(N, KIND_FWD_PAPER, &ax.paper) || !find_pass_kernel(N, KIND_FWD_FOLD, &ax.foldk) ||
        !find_pass_kernel(N, KIND_ADJ_FOLD, &ax.adj)) {
      rc = fail(FFX_EUNSUPPORTED, "no kernel for length %d", N);
      break;
    }
    if ((rc = prepare_kernel(ax.paper)) || (rc = prepare_kernel(ax.foldk)) || (rc = prepare_kernel(ax.adj))) break;
    ax.grid_paper = grid_for(ax.paper.func, ax.paper.threads, ax.paper.smem, p->sms);
    ax.grid_fold = grid_for(ax.foldk.func, ax.foldk.threads, ax.foldk.smem, p->sms);
    ax.grid_adj = grid_for(ax.adj.func, ax.adj.threads, ax.adj.smem, p->sms);
    ax.grid_dense = grid_for(dense_kernel_func(), 256, 0, p->sms);
    e = cudaFuncSetAttribute(dense_small_func(N), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dense_small_smem(N));
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "cudaFuncSetAttribute");
      break;
    }
    ax.grid_dense_small = grid_for(dense_small_func(N), 128, dense_small_smem(N), p->sms);
  }
  if (rc == FFX_OK) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "table fill");
  }

  // dense maps where the dense form may be used
  if (rc == FFX_OK) {
    size_t dbytes = 0, scratch = 0;
    for (int j = 0; j < ndim; ++j) {
      const size_t N = (size_t)dims[j];
      if (N <= (size_t)kDenseMaxN && (form == FFX_FORM_AUTO || form == FFX_FORM_DENSE || form == FFX_FORM_TC)) {
        dbytes += 2 * N * N * sizeof(float2);
        if (N <= (size_t)kDenseInPlaceMaxN) dbytes += 2 * dense_small_image_floats2((int)N) * sizeof(float2);
        scratch = std::max(scratch, 2 * N * N * sizeof(float2));
      }
    }
    if (dbytes > 0) {
      void* tmp = nullptr;
      e = cudaMalloc(&p->dense_mem, dbytes);
      if (e == cudaSuccess) e = cudaMalloc(&tmp, scratch);
      if (e != cudaSuccess) {
        cudaGetLastError();
        rc = fail(FFX_ENOMEM, "dense maps: %s", cudaGetErrorString(e));
      } else {
        float2* dcur = (float2*)p->dense_mem;
        for (int j = 0; j < ndim && rc == FFX_OK; ++j) {
          const size_t N = (size_t)dims[j];
          if (N > (size_t)kDenseMaxN) continue;
          rc = build_dense(p, j, dcur, dcur + N * N, (float2*)tmp, s);
          dcur += 2 * N * N;
          if (rc == FFX_OK && N <= (size_t)kDenseInPlaceMaxN) {
            Axis& ax = p->axis[j];
            const size_t isz = dense_small_image_floats2((int)N);
            ax.img[0] = dcur;
            ax.img[1] = dcur + isz;
            dcur += 2 * isz;
            e = launch_dense_small_image(ax.T, ax.img[0], (int)N, s);
            if (e == cudaSuccess) e = launch_dense_small_image(ax.TH, ax.img[1], (int)N, s);
            if (e != cudaSuccess) rc = cuda_fail(e, "dense image");
          }
        }
        if (rc == FFX_OK) {
          e = cudaStreamSynchronize(s);
          if (e != cudaSuccess) rc = cuda_fail(e, "dense map");
        }
      }
      if (tmp) cudaFree(tmp);
    }
  }

  // split tensor-core operands, and the device error counter
  if (rc == FFX_OK) {
    size_t tbytes = kTcHeader;
    for (int j = 0; j < ndim; ++j)
      if (dense_tc_supported(p->axis[j].N) && p->axis[j].T && (form == FFX_FORM_AUTO || form == FFX_FORM_TC)) {
        tbytes += 2 * dense_tc_t_bytes(p->axis[j].N) + (p->axis[j].N == 64 ? fused_tc_slice_bytes() : 0);
        if (bf16_ops && dense_bf16_supported(p->axis[j].N)) tbytes += 2 * dense_bf16_t_bytes(p->axis[j].N);
      }
    e = cudaMalloc(&p->tc_mem, tbytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = fail(FFX_ENOMEM, "tensor-core operands: %s", cudaGetErrorString(e));
    } else {
      p->dev_err = (int*)p->tc_mem;
      p->grid_bar = (unsigned*)((char*)p->tc_mem + 64);
      p->tile_done = (unsigned*)((char*)p->tc_mem + 1024);
      cudaMemsetAsync(p->tc_mem, 0, kTcHeader, s);
      int native = 0;
      if (cudaDeviceGetAttribute(&native, cudaDevAttrHostNativeAtomicSupported, p->device) == cudaSuccess &&
          native && cudaHostAlloc((void**)&p->host_err, sizeof(int), cudaHostAllocMapped) == cudaSuccess) {
        *(volatile int*)p->host_err = 0;
        int* d = nullptr;
        if (cudaHostGetDevicePointer((void**)&d, p->host_err, 0) == cudaSuccess && d) {
          p->dev_err = d;
        } else {
          cudaFreeHost(p->host_err);
          p->host_err = nullptr;
        }
      }
      cudaGetLastError();
      unsigned char* tcur = (unsigned char*)p->tc_mem + kTcHeader;
      for (int j = 0; j < ndim && rc == FFX_OK; ++j) {
        Axis& ax = p->axis[j];
        if (!(dense_tc_supported(ax.N) && ax.T && (form == FFX_FORM_AUTO || form == FFX_FORM_TC))) continue;
        for (int q = 0; q < 2; ++q) {
          ax.tc_t[q] = tcur;
          tcur += dense_tc_t_bytes(ax.N);
        }
        e = launch_tc_build_t(ax.T, ax.tc_t[0], ax.N, s);
        if (e == cudaSuccess) e = launch_tc_build_t(ax.TH, ax.tc_t[1], ax.N, s);
        if (e == cudaSuccess && ax.N == 64) {
          ax.ft_ts = tcur;
          tcur += fused_tc_slice_bytes();
          e = launch_fused_tc_slices(ax.T, ax.ft_ts, s);
        }
        if (e == cudaSuccess && bf16_ops && dense_bf16_supported(ax.N)) {
          for (int q = 0; q < 2; ++q) {
            ax.bf_t[q] = tcur;
            tcur += dense_bf16_t_bytes(ax.N);
          }
          e = launch_bf16_build_t(ax.T, ax.bf_t[0], ax.N, s);
          if (e == cudaSuccess) e = launch_bf16_build_t(ax.TH, ax.bf_t[1], ax.N, s);
          if (e == cudaSuccess) e = dense_bf16_prepare();
        }
        if (e == cudaSuccess)
          e = dense_tc_prepare();
        if (e != cudaSuccess) rc = cuda_fail(e, "tensor-core operands");
      }
      if (rc == FFX_OK) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "tensor-core operands");
      }
    }
  }
  for (int j = 0; j < ndim && rc == FFX_OK; ++j)
    if (form == FFX_FORM_TC && !tc_capable(p->axis[j])) p->axis[j].form = FFX_FORM_DENSE;

  // per-axis form
  if (rc == FFX_OK) {
    char dev[256] = "unknown";
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) snprintf(dev, sizeof(dev), "%s", prop.name);
    bool tuned_any = false;
    for (int j = 0; j < ndim && rc == FFX_OK; ++j) {
      Axis& ax = p->axis[j];
      if (form != FFX_FORM_AUTO) {
        ax.form = (form == FFX_FORM_TC && !tc_capable(ax)) ? FFX_FORM_DENSE : (int)form;
        continue;
      }
      int64_t outer, inner;
      axis_outer_inner(p, j, &outer, &inner);
      const std::string key = cache_key(dev, ax, outer, inner);
      int f = cache_lookup(key);
      if (f == FFX_FORM_DENSE && !ax.T) f = -1;
      if (f == FFX_FORM_TC && !tc_capable(ax)) f = -1;
      if (f < 0 && (flags & FFX_TUNE)) {
        if (!tuned_any) {
          if ((rc = ensure_ws(p, 0, 1)) || (rc = ensure_ws(p, 1, 1))) break;
          e = cudaMemsetAsync(p->ws[0], 0, (size_t)M * sizeof(float2), s);
          if (e != cudaSuccess) {
            rc = cuda_fail(e, "tuning input");
            break;
          }
          tuned_any = true;
        }
        double ms[4];
        if ((rc = time_forms(p, j, s, ms))) break;
        f = FFX_FORM_PAPER;
        for (int c = FFX_FORM_FOLD; c <= FFX_FORM_TC; ++c)
          if (ms[c - 1] < ms[f - 1]) f = c;
        cache_store(key, f, ms);
      }
      if (f < 0) {
        f = FFX_FORM_PAPER;
        for (int c = FFX_FORM_FOLD; c <= FFX_FORM_TC; ++c) {
          if (c == FFX_FORM_DENSE && !ax.T) continue;
          if (c == FFX_FORM_TC && !tc_capable(ax)) continue;
          if (model_cost(ax, c, outer * inner) < model_cost(ax, f, outer * inner)) f = c;
        }
        ax.few = (f == FFX_FORM_DENSE && outer * inner < kDenseFewLines);
      }
      ax.form = f;
    }
    if (rc == FFX_OK && tuned_any) {
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) rc = cuda_fail(e, "tuning");
    }
  }
  if (rc == FFX_OK && ndim >= 2 && dense_bf16_chain_supported()) {
    bool all = true;
    for (int j = 0; j < ndim; ++j) all = all && p->axis[j].bf_t[0] != nullptr;
    if (all) {
      p->chain_bf16 = 1;
      for (int r = 0; r < ndim; ++r) p->order[r] = ndim - 1 - r;
    }
  }
  if (rc == FFX_OK) rc = plan_fusion(p);
  cudaStreamDestroy(s);
  if (rc != FFX_OK) {
    for (int w = 0; w < kWs; ++w)
      if (p->ws[w]) cudaFree(p->ws[w]);
    if (p->dense_mem) cudaFree(p->dense_mem);
    if (p->tc_mem) cudaFree(p->tc_mem);
    if (p->host_err) cudaFreeHost(p->host_err);
    cudaFree(p->tables);
    delete p;
    return rc;
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
  p->dev_err = many_device_errors(mp);
  for (int j = 0; j < 3; ++j) p->axis[j].form = many_form(mp);
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
  for (int k = 0; k < 2; ++k)
    if (p->stage[k]) cudaFree(p->stage[k]);
  if (p->many) {
    many_destroy(p->many);
    delete p;
    return FFX_OK;
  }
  for (int w = 0; w < kWs; ++w)
    if (p->ws[w]) cudaFree(p->ws[w]);
  if (p->dense_mem) cudaFree(p->dense_mem);
  if (p->tc_mem) cudaFree(p->tc_mem);
  if (p->host_err) cudaFreeHost(p->host_err);
  if (p->tables) cudaFree(p->tables);
  delete p;
  return FFX_OK;
}

int ffx_plan_tc_bf16(ffx_plan_t p) {
  if (!p) return -1;
  if (p->many) return many_bf16(p->many) ? 1 : 0;
  for (int j = 0; j < p->ndim; ++j)
    if (p->axis[j].bf_t[0]) return 1;
  return 0;
}

int ffx_plan_set_wait_limit(ffx_plan_t p, int64_t polls) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (polls < 0) return fail(FFX_EINVAL, "polls < 0");
  p->wait_limit = polls == 0 ? kCrossBlockSpin : (long long)polls;
  return FFX_OK;
}

int ffx_plan_form(ffx_plan_t p) {
  if (!p) return -1;
  const int f = p->axis[0].form;
  for (int j = 1; j < p->ndim; ++j)
    if (p->axis[j].form != f) return FFX_FORM_AUTO;
  return f;
}

int ffx_plan_axis_form(ffx_plan_t p, int axis) {
  if (!p || axis < 0 || axis >= p->ndim) return -1;
  return p->axis[axis].form;
}

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

int ffx_plan_device_errors(ffx_plan_t p) {
  if (!p) return -1;
  if (!p->dev_err) return 0;
  if (p->host_err) {
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    return *(volatile int*)p->host_err;
  }
  int h = 0;
  if (cudaMemcpy(&h, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return h;
}

int64_t ffx_workspace_bytes(ffx_plan_t p, int64_t batch) {
  if (!p || batch < 0) return -1;
  int64_t total = 0;
  for (int w = 0; w < kWs; ++w) total += (int64_t)p->ws_bytes[w];
  const int64_t need = batch * p->M * (int64_t)sizeof(float2);
  return total > need ? total : need;
}

int ffx_launches_per_call(ffx_plan_t p, int backward) {
  if (!p) return -1;
  if (p->fused >= 1 && !backward) return 1;
  return backward ? 2 * p->ndim : p->ndim;  // many-plans: one persistent kernel per phase
}

int64_t ffx_plan_fused(ffx_plan_t p) { return p ? p->fused : -1; }

int ffx_plan_bf16_chain(ffx_plan_t p, int64_t batch) {
  if (!p || batch < 1) return -1;
  if (p->many || batch <= p->fused) return 0;
  const void* aligned = (const void*)(uintptr_t)16;
  return bf16_chain_ok(p, batch, aligned, aligned, aligned) ? 1 : 0;
}

int64_t ffx_plan_launch_count(ffx_plan_t p) { return p ? p->launches : -1; }

int ffx_plan_call_form(ffx_plan_t p, int axis, int64_t batch) {
  if (!p || p->many || axis < 0 || axis >= p->ndim || batch < 1) return -1;
  if (batch <= p->fused) return p->fused_tc ? FFX_FORM_TC : FFX_FORM_DENSE;  // the fused launch
  int64_t outer, inner;
  axis_outer_inner(p, axis, &outer, &inner);
  const int64_t lines = (p->acc && axis == p->order[p->ndim - 1] ? 1 : batch) * outer * inner;
  return call_form(p, p->axis[axis], lines);
}

// The forward passes in the order `axes`, the last one writing densities
// (summed over the batch with FFX_ACCUMULATE).  Every pass but the last
// writes a complex field: ws[0], switching to ws[1] and back for passes that
// cannot run in place.
int forward_density(ffx_plan_s* p, const int* axes, const float2* in, int64_t batch, float* out_d,
                    cudaStream_t s) {
  const int d = p->ndim;
  if (axes == p->order && (const void*)in != p->ws[1] && bf16_chain_ok(p, batch, in, nullptr, out_d))
    return chain_bf16(p, in, batch, nullptr, out_d, s);
  const float2* cur = in;
  int rc;
  if (d > 1) {
    if ((rc = ensure_ws(p, 0, batch))) return rc;
    float2* ws0 = (float2*)p->ws[0];
    float2* target = ws0;
    for (int k = 0; k < d - 1; ++k) {
      const int j = axes[k];
      if (k > 0 && !inplace_ok(p->axis[j])) {
        if ((rc = ensure_ws(p, 1, batch))) return rc;
        target = (cur == ws0) ? (float2*)p->ws[1] : ws0;
      }
      rc = run_axis(p, j, false, cur, nullptr, 0, target, nullptr, 0, batch, s);
      if (rc) return rc;
      cur = target;
    }
  }
  return run_axis(p, axes[d - 1], false, cur, nullptr, 0, nullptr, out_d, p->acc, batch, s);
}

int ffx_expand(ffx_plan_t p, const void* psi0, int64_t batch, float* out_density, void* stream) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (int trc = check_timeout(p)) return trc;
  if (batch < 0) return fail(FFX_EINVAL, "batch < 0");
  if (batch == 0) return FFX_OK;
  int rc;
  if ((rc = check_ptr(psi0, "psi0")) || (rc = check_ptr(out_density, "out_density"))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->many) {
    if (batch != 1) return fail(FFX_EINVAL, "a many-instance plan takes batch = 1");
    std::string err;
    rc = many_expand(p->many, psi0, out_density, nullptr, s, &err);
    if (rc) return fail(rc, "%s", err.c_str());
    p->launches += many_kernels(p->many, 0);
    return FFX_OK;
  }
  if (batch <= p->fused) return run_fused(p, p->order, (const float2*)psi0, nullptr, out_density, nullptr, batch, s);
  return forward_density(p, p->order, (const float2*)psi0, batch, out_density, s);
}

int ffx_expand_host(ffx_plan_t p, const void* psi0_host, int64_t batch, float* out_host, void* stream) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (int trc = check_timeout(p)) return trc;
  if (batch < 0) return fail(FFX_EINVAL, "batch < 0");
  if (batch == 0) return FFX_OK;
  if (!psi0_host) return fail(FFX_EINVAL, "psi0_host is NULL");
  if (!out_host) return fail(FFX_EINVAL, "out_host is NULL");
  if (p->many && batch != 1) return fail(FFX_EINVAL, "a many-instance plan takes batch = 1");
  int rc;
  const size_t in_bytes = (size_t)batch * (size_t)p->M * sizeof(float2);
  const size_t out_bytes = (size_t)(p->acc ? 1 : batch) * (size_t)p->M * sizeof(float);
  if ((rc = ensure_stage(p, 0, in_bytes)) || (rc = ensure_stage(p, 1, out_bytes))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(p->stage[0], psi0_host, in_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && p->acc)  // the sum adds to what out_host holds
    e = cudaMemcpyAsync(p->stage[1], out_host, out_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "input copy to the device");
  if ((rc = ffx_expand(p, p->stage[0], batch, (float*)p->stage[1], stream))) return rc;
  e = cudaMemcpyAsync(out_host, p->stage[1], out_bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "density copy to the host");
  return FFX_OK;
}

int ffx_expand_column(ffx_plan_t p, const void* psi0, int64_t batch, int axis, float* out_column, void* stream) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (int trc = check_timeout(p)) return trc;
  if (batch < 0) return fail(FFX_EINVAL, "batch < 0");
  if (p->many) return fail(FFX_EUNSUPPORTED, "ffx_expand_column does not take a many-instance plan");
  if (axis < 0 || axis >= p->ndim) return fail(FFX_EINVAL, "axis %d out of range", axis);
  if (batch == 0) return FFX_OK;
  int rc;
  if ((rc = check_ptr(psi0, "psi0")) || (rc = check_ptr(out_column, "out_column"))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // the integrated axis runs last: its pass sees whole lines along it
  int axes[3], n = 0;
  for (int k = 0; k < p->ndim; ++k)
    if (p->order[k] != axis) axes[n++] = p->order[k];
  axes[n] = axis;
  if (batch <= p->fused) return run_fused(p, axes, (const float2*)psi0, nullptr, nullptr, out_column, batch, s);
  // densities into ws[2], then the sum along the axis
  if ((rc = ensure_ws(p, 2, batch))) return rc;
  float* rho = (float*)p->ws[2];
  if (p->acc) {
    cudaError_t e = cudaMemsetAsync(rho, 0, (size_t)p->M * sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(e, "density scratch");
  }
  if ((rc = forward_density(p, axes, (const float2*)psi0, batch, rho, s))) return rc;
  int64_t outer, inner;
  axis_outer_inner(p, axis, &outer, &inner);
  const Axis& ax = p->axis[axis];
  cudaError_t e = launch_axis_sum(rho, p->acc ? outer : batch * outer, ax.N, inner, (float)(ax.lam * ax.dx), p->acc,
                                  out_column, p->sms, s);
  if (e != cudaSuccess) return cuda_fail(e, "column sum");
  ++p->launches;
  return FFX_OK;
}

// The forward field map of a batch into `out` (may equal `in`): the fused
// launch for small batches, else the pass chain (ws[0], ws[1] as spares).
int field_into(ffx_plan_s* p, const float2* in, int64_t batch, float2* out, cudaStream_t s) {
  if (batch <= p->fused) return run_fused(p, p->order, in, out, nullptr, nullptr, batch, s);
  return chain_into(p, p->order, false, in, nullptr, 0, batch, out, 0, s);
}

int ffx_expand_positive_p(ffx_plan_t p, const void* psi0, const void* psi0_plus, int64_t batch, float* out_density,
                          void* stream) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (int trc = check_timeout(p)) return trc;
  if (batch < 0) return fail(FFX_EINVAL, "batch < 0");
  if (p->many) return fail(FFX_EUNSUPPORTED, "ffx_expand_positive_p does not take a many-instance plan");
  if (batch == 0) return FFX_OK;
  int rc;
  if ((rc = check_ptr(psi0, "psi0")) || (rc = check_ptr(psi0_plus, "psi0_plus")) ||
      (rc = check_ptr(out_density, "out_density")))
    return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = ensure_ws(p, 2, batch)) || (rc = ensure_ws(p, 3, batch))) return rc;
  float2* w1 = (float2*)p->ws[2];
  float2* w2 = (float2*)p->ws[3];
  if ((rc = field_into(p, (const float2*)psi0, batch, w1, s))) return rc;
  cudaError_t e = launch_conj_copy((const float2*)psi0_plus, w2, batch * p->M, p->sms, s);
  if (e != cudaSuccess) return cuda_fail(e, "conjugate copy");
  ++p->launches;
  if ((rc = field_into(p, w2, batch, w2, s))) return rc;
  e = launch_pair_density(w1, w2, p->M, batch, p->acc, out_density, p->sms, s);
  if (e != cudaSuccess) return cuda_fail(e, "pair density");
  ++p->launches;
  return FFX_OK;
}

int ffx_plan_output_axis(ffx_plan_t p, int axis, double* x0, double* step) {
  if (!p || !x0 || !step) return fail(FFX_EINVAL, "plan, x0 or step is NULL");
  if (p->many) return fail(FFX_EUNSUPPORTED, "a many-instance plan has no single output lattice");
  if (axis < 0 || axis >= p->ndim) return fail(FFX_EINVAL, "axis %d out of range", axis);
  *x0 = p->axis[axis].abar;
  *step = p->axis[axis].lam * p->axis[axis].dx;
  return FFX_OK;
}

int ffx_fringe_phase(const float* image, int64_t rows, int64_t ny, int64_t row_stride, int64_t y_stride, double y0,
                     double dy, double D, double t, double* out_phase, void* stream) {
  g_last_error.clear();
  if (rows < 0 || ny < 0) return fail(FFX_EINVAL, "rows or ny < 0");
  if (rows == 0) return FFX_OK;
  if (ny < 3) return fail(FFX_EINVAL, "ny = %lld: a peak needs three points", (long long)ny);
  if (!(t != 0.0) || !(dy > 0.0) || !std::isfinite(D) || !std::isfinite(y0))
    return fail(FFX_EINVAL, "need t != 0, dy > 0, finite D and y0");
  if (!image || ((uintptr_t)image & 3)) return fail(FFX_EINVAL, "image is NULL or not 4-byte aligned");
  int rc;
  if ((rc = check_ptr(out_phase, "out_phase"))) return rc;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = launch_fringe(image, rows, ny, row_stride, y_stride, y0, dy, D, t, out_phase, sms > 0 ? sms : 1,
                                (cudaStream_t)stream);
  return e == cudaSuccess ? FFX_OK : cuda_fail(e, "fringe readout");
}


int ffx_expand_field(ffx_plan_t p, const void* psi0, int64_t batch, void* out_field, void* stream) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (int trc = check_timeout(p)) return trc;
  if (batch < 0) return fail(FFX_EINVAL, "batch < 0");
  if (batch == 0) return FFX_OK;
  int rc;
  if ((rc = check_ptr(psi0, "psi0")) || (rc = check_ptr(out_field, "out_field"))) return rc;
  if (p->many) {
    if (batch != 1) return fail(FFX_EINVAL, "a many-instance plan takes batch = 1");
    std::string err;
    rc = many_expand(p->many, psi0, nullptr, out_field, (cudaStream_t)stream, &err);
    if (rc) return fail(rc, "%s", err.c_str());
    p->launches += many_kernels(p->many, 1);
    return FFX_OK;
  }
  if (batch <= p->fused)
    return run_fused(p, p->order, (const float2*)psi0, (float2*)out_field, nullptr, nullptr, batch,
                     (cudaStream_t)stream);
  return chain_into(p, p->order, false, (const float2*)psi0, nullptr, 0, batch, (float2*)out_field, 0,
                    (cudaStream_t)stream);
}

int ffx_expand_adjoint(ffx_plan_t p, const void* g_in, int64_t batch, void* g_out, void* stream) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (int trc = check_timeout(p)) return trc;
  if (batch < 0) return fail(FFX_EINVAL, "batch < 0");
  if (batch == 0) return FFX_OK;
  int rc;
  if ((rc = check_ptr(g_in, "g_in")) || (rc = check_ptr(g_out, "g_out"))) return rc;
  if (p->many) return fail(FFX_EUNSUPPORTED, "ffx_expand_adjoint does not take a many-instance plan");
  int axes[3];
  for (int r = 0; r < p->ndim; ++r) axes[r] = p->order[p->ndim - 1 - r];
  return chain_into(p, axes, true, (const float2*)g_in, nullptr, 0, batch, (float2*)g_out, 0,
                    (cudaStream_t)stream);
}

int ffx_expand_backward(ffx_plan_t p, const void* psi0, const float* grad_density, int64_t batch,
                        void* grad_psi0, void* stream) {
  if (!p) return fail(FFX_EINVAL, "plan is NULL");
  if (int trc = check_timeout(p)) return trc;
  if (batch < 0) return fail(FFX_EINVAL, "batch < 0");
  if (batch == 0) return FFX_OK;
  int rc;
  if ((rc = check_ptr(psi0, "psi0")) || (rc = check_ptr(grad_density, "grad_density")) ||
      (rc = check_ptr(grad_psi0, "grad_psi0")))
    return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->many) {
    if (batch != 1) return fail(FFX_EINVAL, "a many-instance plan takes batch = 1");
    std::string err;
    rc = many_backward(p->many, psi0, grad_density, grad_psi0, s, &err);
    if (rc) return fail(rc, "%s", err.c_str());
    p->launches += many_kernels(p->many, 2);
    return FFX_OK;
  }
  // T psi0 into ws[0] (ws[1] as the alternate), then T^H (2 grad * .) into
  // grad_psi0 (ws[1] as the alternate)
  if ((rc = ensure_ws(p, 0, batch))) return rc;
  float2* field = (float2*)p->ws[0];
  if ((rc = chain_into(p, p->order, false, (const float2*)psi0, nullptr, 0, batch, field, 1, s))) return rc;
  // the adjoint half as a BF16 chain where the forward map takes one
  if (bf16_chain_ok(p, batch, field, grad_psi0, nullptr) && bf16_adjoint_ok(p))
    return chain_bf16_adjoint(p, field, grad_density, p->acc, batch, (float2*)grad_psi0, s);
  int axes[3];
  for (int r = 0; r < p->ndim; ++r) axes[r] = p->order[p->ndim - 1 - r];
  return chain_into(p, axes, true, field, grad_density, p->acc, batch, (float2*)grad_psi0, 1, s);
}

}  // extern "C"
