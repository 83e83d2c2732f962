// Plans over many instances of uneven lattices (ffx_plan_many).
//
// Realizations of an ensemble are independent (Sec. 1: hundreds or thousands
// of classical-field realizations), but their lattices and magnifications may
// differ.  Pass k of every instance (its k-th axis, longest lines first) forms
// one phase.  A phase is ONE persistent kernel over a work list of (instance,
// tile range) items, taken from a device counter, biggest first; each item
// runs the same line-pass tile code as the uniform kernels, picked by the
// instance's line length.  The phases are separated by kernel boundaries, not
// device-side waits, and the whole sequence (counter resets + phase kernels)
// is one CUDA graph, built once per plan and mode and replayed on the caller's
// stream.  Buffers are packed: instance i occupies points [off_i, off_i + M_i)
// of the input, the workspace and the output.
//
// Dense mode (FFX_FORM_DENSE, or the automatic form when the dense per-axis
// maps cost less than the fold form for every instance axis): the plan builds
// T and T^H of every distinct (N, lam, dx, t, a, abar) once, with the fold
// pass on the unit vectors, and each phase is one persistent kernel over
// (instance, 64 x 32 tiles) items of the dense product.  Those passes are not
// in place for N > 64, so pass k of an instance writes workspace k % 2.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <queue>
#include <tuple>
#include <vector>

#include "../../include/ffx.h"
#include "ffx_dense_tile.cuh"
#include "ffx_internal.h"
#include "ffx_pass.cuh"
#include "ffx_plans.h"
#include "ffx_tc_many.h"

namespace ffx {

// Pointers of one call; pass arguments hold byte offsets into these.
enum ManyBase : int { BASE_NONE = -1, BASE_PSI0 = 0, BASE_WS = 1, BASE_OUTC = 2, BASE_OUTD = 3,
                      BASE_GRAD = 4, BASE_WS2 = 5, NBASE = 6 };
constexpr int KIND_DENSE = 100;  // a dense phase (forward or adjoint: the item's matrix decides)
constexpr int KIND_TC = 101;     // the same on the tensor cores (split TF32)
constexpr int KIND_TC16 = 102;   // the same with split BF16 operands
constexpr int KIND_TC16T = 103;  // the same, every input by TMA tiles (a tile map per pass)
constexpr int KIND_TC16P = 104;  // a BF16 chain pass: planes in, planes (or the output) out, transposed
constexpr int KIND_SPLITG = 105;  // a backward chain's split of 2 grad * field into planes
constexpr int KIND_TC16P1 = 107;  // a BF16 chain's first pass: the caller's FP32 input by TMA tiles, planes out
bool tc_kind(int kind) {
  return kind == KIND_TC || kind == KIND_TC16 || kind == KIND_TC16T || kind == KIND_TC16P || kind == KIND_TC16P1;
}
struct ManyCall {
  const void* base[NBASE];
};

struct ManyItem {
  int arg;         // index into the phase's PassArgs
  int N;           // line length (selects the tile code)
  int in_base, outc_base, outd_base, grad_base;
  long long t0, t1;  // tiles [t0, t1)
};

namespace {

__device__ __forceinline__ const void* rebase(const ManyCall& c, int base, const void* off) {
  return base < 0 ? nullptr : (const void*)((const char*)c.base[base] + (uintptr_t)off);
}

template <int KIND>
__device__ __forceinline__ void run_item(const PassArgs& a, int N, long long t0, long long t1,
                                         unsigned char* smem) {
  switch (N) {
    case 16: pass_tiles<Plan16, KIND, kGroups16>(a, t0, t1, 1, smem); break;
    case 32: pass_tiles<Plan32, KIND, kGroups32>(a, t0, t1, 1, smem); break;
    case 48: pass_tiles<Plan48, KIND, kGroups48>(a, t0, t1, 1, smem); break;
    case 64: pass_tiles<Plan64, KIND, kGroups64>(a, t0, t1, 1, smem); break;
    case 96: pass_tiles<Plan96, KIND, kGroups96>(a, t0, t1, 1, smem); break;
    case 128: pass_tiles<Plan128, KIND, kGroups128>(a, t0, t1, 1, smem); break;
    case 192: pass_tiles<Plan192, KIND, kGroups192>(a, t0, t1, 1, smem); break;
    case 256: pass_tiles<Plan256, KIND, kGroups256>(a, t0, t1, 1, smem); break;
    default: break;  // the host admits only the lengths above
  }
}

constexpr int kManyLengths[] = {16, 32, 48, 64, 96, 128, 192, 256};

constexpr size_t many_smem_bytes() {
  size_t m = 0;
  m = std::max(m, PassSmem<Plan16, kGroups16>::bytes);
  m = std::max(m, PassSmem<Plan32, kGroups32>::bytes);
  m = std::max(m, PassSmem<Plan48, kGroups48>::bytes);
  m = std::max(m, PassSmem<Plan64, kGroups64>::bytes);
  m = std::max(m, PassSmem<Plan96, kGroups96>::bytes);
  m = std::max(m, PassSmem<Plan128, kGroups128>::bytes);
  m = std::max(m, PassSmem<Plan192, kGroups192>::bytes);
  m = std::max(m, PassSmem<Plan256, kGroups256>::bytes);
  return m;
}

// Dense phases: persistent blocks take (instance, tile range) items.
__global__ void __launch_bounds__(256) many_dense_kernel(const DenseArgs* __restrict__ args,
                                                         const ManyItem* __restrict__ items, int n_items,
                                                         int* counter, const ManyCall call) {
  __shared__ DenseTileSmem sm;
  __shared__ int s_item;
  for (;;) {
    __syncthreads();  // everyone has read s_item (and is done with the last tile)
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const ManyItem w = items[it];
    DenseArgs a = args[w.arg];
    a.in = (const float2*)rebase(call, w.in_base, a.in);
    a.out_c = (float2*)rebase(call, w.outc_base, a.out_c);
    a.out_d = (float*)rebase(call, w.outd_base, a.out_d);
    a.grad = (const float*)rebase(call, w.grad_base, a.grad);
    for (long long t = w.t0; t < w.t1; ++t) dense_tile(a, t, sm);
  }
}

template <int KIND>
__global__ void __launch_bounds__(256, 2) many_kernel(const PassArgs* __restrict__ args,
                                                   const ManyItem* __restrict__ items, int n_items,
                                                   int* counter, const ManyCall call) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  for (;;) {
    __syncthreads();  // everyone has read s_item
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const ManyItem w = items[it];
    PassArgs a = args[w.arg];
    a.in = (const float2*)rebase(call, w.in_base, a.in);
    a.out_c = (float2*)rebase(call, w.outc_base, a.out_c);
    a.out_d = (float*)rebase(call, w.outd_base, a.out_d);
    a.grad = (const float*)rebase(call, w.grad_base, a.grad);
    run_item<KIND>(a, w.N, w.t0, w.t1, smem);
  }
}

bool many_length(int64_t N) {
  for (int n : kManyLengths)
    if (n == N) return true;
  return false;
}

uint64_t frac_fx64(double x) {
  double f = x - std::floor(x);
  if (!(f >= 0.0) || f >= 1.0) f = 0.0;
  return (uint64_t)std::ldexp(f, 64);
}

int64_t gcd_64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

int64_t invmod_64(int64_t a, int64_t m) {
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

struct AxisTab {
  int N, lam, g, Np;
  AxisTables tab;
  const float2* T = nullptr;   // dense mode: the per-axis map and its adjoint
  const float2* TH = nullptr;
  const unsigned char* tc[2] = {nullptr, nullptr};  // tensor-core mode: split operand blocks of T, T^H
  const unsigned char* bf[2] = {nullptr, nullptr};  // the same as split BF16 blocks (BF16 phases)
};

struct Instance {
  int ndim;
  int64_t dims[3];
  int64_t M, off;
  int order[3];
  int axis_tab[3];  // index into ManyPlan::tabs
};

struct Phase {
  int kind;
  PassArgs* d_args = nullptr;
  DenseArgs* d_dargs = nullptr;  // dense phases
  ManyItem* d_items = nullptr;
  int n_items = 0;
  TcPassArg* d_targs = nullptr;  // tensor-core phases
  TcItem* d_titems = nullptr;
  long long* d_first = nullptr;   // per block: first item of its run (grid_tc + 1 entries)
  long long n_titems = 0;
  const void* d_xmaps = nullptr;  // BF16 phases: tile maps of inputs in the plan's workspaces
  // a chain's first pass by TMA: per pass argument (instance offset, N, lines)
  // of the tile map made for each call's input
  std::vector<std::array<int64_t, 3>> call_maps;
};

}  // namespace

struct ManyPlan {
  int n = 0;
  int form = FFX_FORM_FOLD;
  int64_t total = 0;
  int max_dim = 0;
  std::vector<Instance> inst;
  std::vector<AxisTab> tabs;
  void* mem = nullptr;      // tables, fold indices, args, items, counters (one allocation)
  float2* ws = nullptr;     // packed workspace (total points)
  float2* ws2 = nullptr;    // dense mode: the second workspace
  bool dense = false;
  bool tc = false;            // dense mode on the tensor cores
  bool bf16 = false;          // tensor-core passes with split BF16 operands where the length allows
  void* dense_mem = nullptr;  // dense mode: T, T^H of every table key
  void* tc_mem = nullptr;     // tensor-core mode: operand blocks of every key
  int* dev_err = nullptr;     // launches that gave up on a bounded wait
  int grid_tc = 0;
  int grid_dense = 0;
  int* counters = nullptr;  // one per phase
  int grid_fwd = 0, grid_adj = 0;
  size_t smem = 0;
  // graphs per mode: 0 density, 1 field, 2 backward
  std::vector<Phase> phases[3];
  cudaGraph_t graph[3] = {nullptr, nullptr, nullptr};
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
  std::vector<cudaGraphNode_t> knodes[3];
  ManyCall last_call[3];
};

namespace {

// Items of one phase: each instance's pass cut into chunks of tiles, sorted
// by estimated cost, biggest first.
void build_items(const ManyPlan& mp, int step_of_instance /* -1: none */, const PassKernelInfo& k,
                 int arg, const Instance& in, int axis_tab, int in_base, int outc_base, int outd_base,
                 int grad_base, std::vector<std::pair<double, ManyItem>>& out) {
  (void)step_of_instance;
  (void)mp;
  const AxisTab& at = mp.tabs[axis_tab];
  const int64_t lines = in.M / at.N;
  const int lpt = k.lines;
  const int64_t ntiles = (lines + lpt - 1) / lpt;
  const int64_t chunk = 4;
  const double per_tile = (double)at.lam * at.N * std::log2((double)at.N + 1.0) * lpt;
  for (int64_t t0 = 0; t0 < ntiles; t0 += chunk) {
    ManyItem w;
    w.arg = arg;
    w.N = at.N;
    w.in_base = in_base;
    w.outc_base = outc_base;
    w.outd_base = outd_base;
    w.grad_base = grad_base;
    w.t0 = t0;
    w.t1 = std::min(ntiles, t0 + chunk);
    out.push_back({per_tile * (double)(w.t1 - w.t0), w});
  }
}

PassArgs pass_args_for(const Instance& in, int axis, const AxisTab& at, size_t in_off, size_t outc_off,
                       size_t outd_off, size_t grad_off, bool use_outc, bool use_outd, bool use_grad) {
  PassArgs a;
  std::memset(&a, 0, sizeof(a));
  int64_t outer = 1, inner = 1;
  for (int i = 0; i < axis; ++i) outer *= in.dims[i];
  for (int i = axis + 1; i < in.ndim; ++i) inner *= in.dims[i];
  a.in = (const float2*)(uintptr_t)in_off;
  a.out_c = use_outc ? (float2*)(uintptr_t)outc_off : nullptr;
  a.out_d = use_outd ? (float*)(uintptr_t)outd_off : nullptr;
  a.grad = use_grad ? (const float*)(uintptr_t)grad_off : nullptr;
  a.outer = outer;
  a.inner = inner;
  a.M = in.M;
  a.batch = 1;
  a.nlines = outer * inner;
  a.acc = 0;
  a.grad_shared = 0;
  a.lam = at.lam;
  a.g = at.g;
  a.Np = at.Np;
  a.qg = 1;
  a.tab = at.tab;
  return a;
}

}  // namespace

namespace {

// T_j and T_j^H of every table key: the fold pass (the uniform line kernel of
// that length) on the N unit vectors, then the transpose / conjugate.
int build_dense_maps(ManyPlan* mp, bool tc, bool bf16, cudaStream_t s, std::string* err) {
  size_t bytes = (size_t)mp->total * sizeof(float2);  // the second workspace
  int nmax = 0;
  for (const AxisTab& at : mp->tabs) {
    bytes += 2 * (size_t)at.N * at.N * sizeof(float2);
    nmax = std::max(nmax, at.N);
  }
  const size_t scratch = 2 * (size_t)nmax * nmax * sizeof(float2);
  cudaError_t e = cudaMalloc(&mp->dense_mem, bytes + scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    mp->dense_mem = nullptr;
    *err = std::string("dense maps: ") + cudaGetErrorString(e);
    return FFX_ENOMEM;
  }
  char* cur = (char*)mp->dense_mem;
  mp->ws2 = (float2*)cur;
  cur += (size_t)mp->total * sizeof(float2);
  float2* I = (float2*)(cur + (bytes - (size_t)mp->total * sizeof(float2)));
  float2* O = I + (size_t)nmax * nmax;
  for (AxisTab& at : mp->tabs) {
    const int N = at.N;
    float2* T = (float2*)cur;
    float2* TH = T + (size_t)N * N;
    cur += 2 * (size_t)N * N * sizeof(float2);
    PassKernelInfo info;
    if (!find_pass_kernel(N, KIND_FWD_FOLD, &info)) {
      *err = "no fold kernel for length " + std::to_string(N);
      return FFX_EUNSUPPORTED;
    }
    e = cudaFuncSetAttribute(info.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)info.smem);
    if (e == cudaSuccess) e = launch_identity(I, N, s);
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in = I;
    a.out_c = O;
    a.outer = 1;
    a.inner = 1;
    a.M = N;
    a.batch = N;
    a.nlines = N;
    a.lam = at.lam;
    a.g = at.g;
    a.Np = at.Np;
    a.qg = 1;
    a.tab = at.tab;
    const int lines = pass_lines_per_tile(info, 1);
    if (e == cudaSuccess) e = info.launch(a, (N + lines - 1) / lines, s);
    if (e == cudaSuccess) e = launch_dense_build(O, T, TH, N, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // I and O are reused by the next key
    if (e != cudaSuccess) {
      cudaGetLastError();
      *err = std::string("dense map: ") + cudaGetErrorString(e);
      return FFX_ECUDA;
    }
    at.T = T;
    at.TH = TH;
  }
  mp->dense = true;
  mp->form = FFX_FORM_DENSE;
  if (!tc) return FFX_OK;
  // tensor-core mode: the split operand blocks of every key's T and T^H (TF32,
  // and BF16 for the lengths the BF16 kernel takes), and the kernels'
  // shared-memory allowance (one block per SM)
  e = many_tc_prepare();
  int per = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, many_tc_func(), many_tc_threads(), many_tc_smem());
  if (e != cudaSuccess || per < 1) {
    cudaGetLastError();
    return FFX_OK;  // the FP32 dense phases
  }
  if (bf16) {
    per = 0;
    e = many_bf16_prepare();
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, many_bf16_func(0), many_bf16_threads(),
                                                        many_bf16_smem());
    for (int m : {1, 2, 4}) {
      if (e != cudaSuccess) break;
      int per_m = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_m, many_bf16_func(m), many_bf16_threads(),
                                                        many_bf16_smem());
      if (per_m < per) per = per_m;
    }
    if (e != cudaSuccess || per < 1) {
      cudaGetLastError();
      bf16 = false;  // split TF32 throughout
    }
  }
  size_t tbytes = 0;
  for (const AxisTab& at : mp->tabs) {
    tbytes += 2 * dense_tc_t_bytes(at.N);
    if (bf16 && many_bf16_supported(at.N)) tbytes += 2 * dense_bf16_t_bytes(at.N);
  }
  e = cudaMalloc(&mp->tc_mem, tbytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    mp->tc_mem = nullptr;
    *err = std::string("tensor-core operands: ") + cudaGetErrorString(e);
    return FFX_ENOMEM;
  }
  unsigned char* tcur = (unsigned char*)mp->tc_mem;
  for (AxisTab& at : mp->tabs) {
    unsigned char* t0 = tcur;
    unsigned char* t1 = tcur + dense_tc_t_bytes(at.N);
    tcur = t1 + dense_tc_t_bytes(at.N);
    e = launch_tc_build_t(at.T, t0, at.N, s);
    if (e == cudaSuccess) e = launch_tc_build_t(at.TH, t1, at.N, s);
    if (e == cudaSuccess && bf16 && many_bf16_supported(at.N)) {
      at.bf[0] = tcur;
      at.bf[1] = tcur + dense_bf16_t_bytes(at.N);
      tcur += 2 * dense_bf16_t_bytes(at.N);
      e = launch_bf16_build_t(at.T, (unsigned char*)at.bf[0], at.N, s);
      if (e == cudaSuccess) e = launch_bf16_build_t(at.TH, (unsigned char*)at.bf[1], at.N, s);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      *err = std::string("tensor-core operands: ") + cudaGetErrorString(e);
      return FFX_ECUDA;
    }
    at.tc[0] = t0;
    at.tc[1] = t1;
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *err = std::string("tensor-core operands: ") + cudaGetErrorString(e);
    return FFX_ECUDA;
  }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  mp->grid_tc = sms;
  mp->tc = true;
  mp->bf16 = bf16;
  mp->form = FFX_FORM_TC;
  return FFX_OK;
}

}  // namespace

int many_create(ManyPlan** out, int n, const ffx_instance_desc* d, uint32_t flags, std::string* err) {
  *out = nullptr;
  if (n < 1 || !d) {
    *err = "n_instances must be >= 1 and descs non-NULL";
    return FFX_EINVAL;
  }
  if (flags & FFX_ACCUMULATE) {
    *err = "FFX_ACCUMULATE is not defined for instances of different lattices";
    return FFX_EINVAL;
  }
  const uint32_t form = flags & FFX_FORM_MASK;
  if (flags & ~(FFX_FORM_MASK | FFX_TC_BF16 | FFX_TC_TF32)) {
    *err = "unknown flag bits (FFX_TUNE, FFX_UNFUSED and FFX_TC_UNSPLIT do not apply to many-instance plans)";
    return FFX_EINVAL;
  }
  if ((flags & FFX_TC_BF16) && (flags & FFX_TC_TF32)) {
    *err = "FFX_TC_BF16 and FFX_TC_TF32 exclude each other";
    return FFX_EINVAL;
  }
  if ((flags & (FFX_TC_BF16 | FFX_TC_TF32)) && form != FFX_FORM_TC && form != FFX_FORM_AUTO) {
    *err = "FFX_TC_BF16 and FFX_TC_TF32 need FFX_FORM_TC or FFX_FORM_AUTO";
    return FFX_EINVAL;
  }
  if (form != FFX_FORM_AUTO && form != FFX_FORM_PAPER && form != FFX_FORM_FOLD && form != FFX_FORM_DENSE &&
      form != FFX_FORM_TC) {
    *err = "unknown form (paper, fold, dense, tc or automatic)";
    return FFX_EINVAL;
  }
  ManyPlan* mp = new ManyPlan();
  mp->n = n;
  mp->form = (form == FFX_FORM_PAPER) ? FFX_FORM_PAPER : FFX_FORM_FOLD;
  // geometry checks and table keys
  typedef std::tuple<int64_t, int, double, double, double, double> Key;  // N, lam, dx, t, a, abar
  std::map<Key, int> keymap;
  std::vector<Key> keys;
  for (int i = 0; i < n; ++i) {
    const ffx_instance_desc& e = d[i];
    Instance in;
    if (e.ndim < 1 || e.ndim > 3) {
      *err = "instance " + std::to_string(i) + ": ndim must be 1..3";
      delete mp;
      return FFX_EINVAL;
    }
    if (!std::isfinite(e.t)) {
      *err = "instance " + std::to_string(i) + ": t must be finite";
      delete mp;
      return FFX_EINVAL;
    }
    in.ndim = e.ndim;
    in.M = 1;
    for (int j = 0; j < e.ndim; ++j) {
      if (e.dims[j] < 1 || !(e.spacing[j] > 0) || !std::isfinite(e.spacing[j]) || e.magnification[j] < 1 ||
          e.magnification[j] > 65536 || (int64_t)e.magnification[j] * e.dims[j] > (int64_t(1) << 24) ||
          (e.has_offsets && (!std::isfinite(e.a[j]) || !std::isfinite(e.abar[j])))) {
        *err = "instance " + std::to_string(i) + ": bad dims, spacing, magnification or offsets";
        delete mp;
        return FFX_EINVAL;
      }
      if (!many_length(e.dims[j])) {
        *err = "instance " + std::to_string(i) + ": line length " + std::to_string(e.dims[j]) +
               " has no batched kernel (16, 32, 48, 64, 96, 128, 192, 256)";
        delete mp;
        return FFX_EUNSUPPORTED;
      }
      in.dims[j] = e.dims[j];
      in.M *= e.dims[j];
      const double L = e.dims[j] * e.spacing[j];
      const double a = e.has_offsets ? e.a[j] : -0.5 * L;
      const double ab = e.has_offsets ? e.abar[j]
                                      : a + (double)(-(((int64_t)(e.magnification[j] - 1) * e.dims[j]) / 2)) *
                                                e.spacing[j];
      Key k(e.dims[j], e.magnification[j], e.spacing[j], e.t, a, ab);
      auto itk = keymap.find(k);
      if (itk == keymap.end()) {
        itk = keymap.emplace(k, (int)keys.size()).first;
        keys.push_back(k);
      }
      in.axis_tab[j] = itk->second;
    }
    in.off = mp->total;
    mp->total += in.M;
    for (int j = 0; j < in.ndim; ++j) in.order[j] = j;
    for (int a = 0; a < in.ndim; ++a)
      for (int b = a + 1; b < in.ndim; ++b)
        if (in.dims[in.order[b]] > in.dims[in.order[a]]) std::swap(in.order[a], in.order[b]);
    mp->max_dim = std::max(mp->max_dim, in.ndim);
    mp->inst.push_back(in);
  }
  // one device allocation: tables | fold | workspace | counters (args/items are added per mode)
  size_t tab_bytes = 0;
  for (const Key& k : keys) {
    const size_t N = (size_t)std::get<0>(k), lam = (size_t)std::get<1>(k);
    tab_bytes += (4 * lam * N + N) * sizeof(float2) + ((N * sizeof(int) + 255) & ~size_t(255));
  }
  const size_t ws_bytes = (size_t)mp->total * sizeof(float2);
  const size_t cnt_bytes = 256;
  cudaError_t e = cudaMalloc(&mp->mem, tab_bytes + ws_bytes + cnt_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *err = std::string("device allocation: ") + cudaGetErrorString(e);
    delete mp;
    return FFX_ENOMEM;
  }
  char* cur = (char*)mp->mem;
  mp->ws = (float2*)cur;
  cur += ws_bytes;
  mp->counters = (int*)cur;
  mp->dev_err = mp->counters + 32;  // the counters' region holds it too (zeroed below)
  cur += cnt_bytes;
  cudaStream_t s;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  std::vector<int> fold_h;
  int rc = FFX_OK;
  e = cudaMemsetAsync(mp->counters, 0, cnt_bytes, s);  // phase counters and the error count
  if (e != cudaSuccess) {
    rc = FFX_ECUDA;
    *err = std::string("counters: ") + cudaGetErrorString(e);
  }
  for (size_t ki = 0; rc == FFX_OK && ki < keys.size(); ++ki) {
    const Key& k = keys[ki];
    AxisTab at;
    at.N = (int)std::get<0>(k);
    at.lam = std::get<1>(k);
    const double dx = std::get<2>(k), t = std::get<3>(k), a = std::get<4>(k), ab = std::get<5>(k);
    at.g = (int)gcd_64(at.lam, at.N);
    at.Np = at.N / at.g;
    const size_t lN = (size_t)at.lam * at.N;
    float2* P = (float2*)cur;
    float2* K = P + lN;
    float2* Kf = K + lN;
    float2* F = Kf + lN;
    float2* tw = F + lN;
    cur += (4 * lN + at.N) * sizeof(float2);
    int* fold = (int*)cur;
    cur += ((size_t)at.N * sizeof(int) + 255) & ~size_t(255);
    const double L = at.N * dx, sv = (ab - a) / dx, tau = M_PI * t / (L * L);
    e = launch_fill_tables(at.N, at.lam, frac_fx64(sv / at.N), frac_fx64(tau), frac_fx64(2.0 * tau / at.lam),
                           frac_fx64(sv / ((double)at.lam * at.N)), frac_fx64(tau / ((double)at.lam * at.lam)),
                           nullptr, P, K, Kf, F, tw, s);
    if (e != cudaSuccess) {
      rc = FFX_ECUDA;
      *err = std::string("table fill: ") + cudaGetErrorString(e);
      break;
    }
    const int64_t inv = invmod_64((at.lam / at.g) % at.Np, at.Np);
    fold_h.assign(at.N, -1);
    for (int r = 0; r < at.N; ++r)
      if (r % at.g == 0) fold_h[r] = (int)(((int64_t)(r / at.g) * inv) % at.Np);
    e = cudaMemcpyAsync(fold, fold_h.data(), sizeof(int) * at.N, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // fold_h is reused
    if (e != cudaSuccess) {
      rc = FFX_ECUDA;
      *err = std::string("fold upload: ") + cudaGetErrorString(e);
      break;
    }
    at.tab.P = P;
    at.tab.K = K;
    at.tab.Kf = Kf;
    at.tab.F = F;
    at.tab.tw = tw;
    at.tab.fold = fold;
    mp->tabs.push_back(at);
  }
  if (rc == FFX_OK) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      rc = FFX_ECUDA;
      *err = std::string("table fill: ") + cudaGetErrorString(e);
    }
  }
  // Dense mode: every key's T and T^H (fold pass on the unit vectors).  The
  // automatic form takes it when the dense map costs less than the fold form
  // on every key (8 N flops per point at ~0.45 of the FP32 peak against
  // lam (5 log2 N + 14) + 5 log2 N at ~0.11).
  // Tensor-core mode (FFX_FORM_TC, or the automatic form once dense): every
  // key's lines a multiple of 16 points from 32 up; otherwise, or if the
  // kernel cannot be resident, the FP32 dense phases.  Its passes take split
  // BF16 operands, but the first adjoint pass of a backward call (with its
  // gradient factors) and the passes of FFX_TC_TF32 plans split TF32.
  if (rc == FFX_OK) {
    bool dense = (form == FFX_FORM_DENSE || form == FFX_FORM_TC);
    if (form == FFX_FORM_AUTO) {
      dense = true;
      for (const AxisTab& at : mp->tabs) {
        const double lg = std::log2((double)at.N);
        if (8.0 * at.N / 0.45 >= (at.lam * (5 * lg + 14) + 5 * lg) / 0.11) dense = false;
      }
    }
    bool tc = (form == FFX_FORM_TC || form == FFX_FORM_AUTO);
    for (const AxisTab& at : mp->tabs) tc = tc && dense_tc_supported(at.N);
    // split BF16 operands on the lengths the BF16 kernel takes, unless split
    // TF32 is asked for
    const bool bf16 = !(flags & FFX_TC_TF32);
    if (dense) rc = build_dense_maps(mp, tc, bf16, s, err);
  }
  cudaStreamDestroy(s);
  if (rc != FFX_OK) {
    if (mp->tc_mem) cudaFree(mp->tc_mem);
    if (mp->dense_mem) cudaFree(mp->dense_mem);
    cudaFree(mp->mem);
    delete mp;
    return rc;
  }
  // persistent grid: resident blocks of the phase kernels
  mp->smem = many_smem_bytes();
  const void* kf = (mp->form == FFX_FORM_PAPER) ? (const void*)many_kernel<KIND_FWD_PAPER>
                                                : (const void*)many_kernel<KIND_FWD_FOLD>;
  const void* ka = (const void*)many_kernel<KIND_ADJ_FOLD>;
  int dev = 0, sms = 1, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mp->smem);
  cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mp->smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kf, 256, mp->smem) != cudaSuccess || per < 1) per = 1;
  mp->grid_fwd = per * sms;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ka, 256, mp->smem) != cudaSuccess || per < 1) per = 1;
  mp->grid_adj = per * sms;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, many_dense_kernel, 256, 0) != cudaSuccess || per < 1)
    per = 1;
  mp->grid_dense = per * sms;
  cudaGetLastError();
  *out = mp;
  return FFX_OK;
}

namespace {

// Dense phases of one mode.  Instance i runs its own chain of steps: forward
// passes k = 0 .. n_i - 1 (phase k), then for the backward adjoint passes
// r = 0 .. n_i - 1 (phase D + r, step n_i + r).  Step s writes workspace s % 2,
// except the final step, which writes the caller's output; step s reads the
// input (s = 0) or the workspace of step s - 1.
int build_dense_phases(ManyPlan* mp, int mode, std::string* err) {
  std::vector<Phase>& phases = mp->phases[mode];
  const int D = mp->max_dim;
  const int nphases = (mode == 2) ? 2 * D : D;
  for (int ph_i = 0; ph_i < nphases; ++ph_i) {
    const bool adj = (mode == 2 && ph_i >= D);
    const int r = adj ? ph_i - D : ph_i;
    Phase ph;
    ph.kind = KIND_DENSE;
    std::vector<DenseArgs> args;
    std::vector<std::pair<double, ManyItem>> items;
    for (const Instance& in : mp->inst) {
      if (r >= in.ndim) continue;
      const int n_i = in.ndim;
      const int k = adj ? n_i - 1 - r : r;  // pass index in the forward order
      const int step = adj ? n_i + r : r;
      const int last_step = (mode == 2) ? 2 * n_i - 1 : n_i - 1;
      const int axis = in.order[k];
      const AxisTab& at = mp->tabs[in.axis_tab[axis]];
      const size_t off_c = (size_t)in.off * sizeof(float2), off_d = (size_t)in.off * sizeof(float);
      auto wsb = [](int st) { return (st % 2 == 0) ? BASE_WS : BASE_WS2; };
      const int in_base = (step == 0) ? BASE_PSI0 : wsb(step - 1);
      int outc_base = BASE_NONE, outd_base = BASE_NONE;
      if (step == last_step) {
        if (mode == 0)
          outd_base = BASE_OUTD;
        else
          outc_base = BASE_OUTC;
      } else {
        outc_base = wsb(step);
      }
      const int grad_base = (adj && r == 0) ? BASE_GRAD : BASE_NONE;
      DenseArgs a;
      std::memset(&a, 0, sizeof(a));
      int64_t outer = 1, inner = 1;
      for (int i = 0; i < axis; ++i) outer *= in.dims[i];
      for (int i = axis + 1; i < in.ndim; ++i) inner *= in.dims[i];
      a.A = adj ? at.TH : at.T;
      a.in = (const float2*)(uintptr_t)off_c;
      a.out_c = outc_base >= 0 ? (float2*)(uintptr_t)off_c : nullptr;
      a.out_d = outd_base >= 0 ? (float*)(uintptr_t)off_d : nullptr;
      a.grad = grad_base >= 0 ? (const float*)(uintptr_t)off_d : nullptr;
      a.outer = outer;
      a.inner = inner;
      a.M = in.M;
      a.batch = 1;
      a.ncols = outer * inner;
      a.N = at.N;
      const int arg = (int)args.size();
      args.push_back(a);
      const int64_t ntiles = dense_tile_count(at.N, a.ncols);
      const int64_t chunk = 4;
      const double per_tile = (double)at.N * DBM * DBN;
      for (int64_t t0 = 0; t0 < ntiles; t0 += chunk) {
        ManyItem w;
        w.arg = arg;
        w.N = at.N;
        w.in_base = in_base;
        w.outc_base = outc_base;
        w.outd_base = outd_base;
        w.grad_base = grad_base;
        w.t0 = t0;
        w.t1 = std::min(ntiles, t0 + chunk);
        items.push_back({per_tile * (double)(w.t1 - w.t0), w});
      }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, ManyItem>& x, const std::pair<double, ManyItem>& y) {
                       return x.first > y.first;
                     });
    std::vector<ManyItem> flat;
    flat.reserve(items.size());
    for (auto& pi : items) flat.push_back(pi.second);
    const size_t bytes = args.size() * sizeof(DenseArgs) + flat.size() * sizeof(ManyItem);
    void* m = nullptr;
    cudaError_t e = cudaMalloc(&m, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *err = std::string("work list: ") + cudaGetErrorString(e);
      return FFX_ENOMEM;
    }
    ph.d_dargs = (DenseArgs*)m;
    ph.d_items = (ManyItem*)((char*)m + args.size() * sizeof(DenseArgs));
    ph.n_items = (int)flat.size();
    e = cudaMemcpy(ph.d_dargs, args.data(), args.size() * sizeof(DenseArgs), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(ph.d_items, flat.data(), flat.size() * sizeof(ManyItem), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(m);
      *err = std::string("work list upload: ") + cudaGetErrorString(e);
      return FFX_ECUDA;
    }
    phases.push_back(ph);
  }
  return FFX_OK;
}

// One tensor-core phase launch over the passes `args` (split TF32 or BF16
// kernel): the row blocks of one (pass, line tile) form a group that one block
// runs back to back, so the second row block reads the lines from L2 right
// after the first.  Groups are dealt to blocks biggest first, each to the least
// loaded block (cost: K chunks x rows), and every block runs its groups in the
// order dealt.
int deal_tc_phase(ManyPlan* mp, int kind, std::vector<TcPassArg> args, std::vector<Phase>& phases,
                  std::string* err, const std::vector<unsigned char>* plane_maps = nullptr) {
  if (args.empty()) return FFX_OK;
  const bool bf = (kind != KIND_TC);
  // BF16 phases: a tile map of every input of contiguous lines in the plan's
  // workspaces (the kernel loads those as TMA tiles; the others, the caller's
  // input and strided lines, by per-thread copies)
  // by TMA when every pass of the launch has one (one input mode per launch)
  std::vector<unsigned char> maps;
  bool all_maps = kind == KIND_TC16;
  const bool premade = kind == KIND_TC16P || kind == KIND_TC16P1;
  if (premade) maps = *plane_maps;  // the chain's pass arguments carry their map indices
  for (TcPassArg& pa : args) {
    if (premade) break;
    pa.xmap = -1;
    if (!all_maps || pa.d.inner != 1 || (pa.in_base != BASE_WS && pa.in_base != BASE_WS2)) {
      all_maps = false;
      continue;
    }
    const float2* ws = pa.in_base == BASE_WS ? mp->ws : mp->ws2;
    const float2* base = (const float2*)((const char*)ws + (uintptr_t)pa.d.in);
    unsigned char m[128];
    if (!many_bf16_line_map(base, (int)pa.d.N, pa.d.ncols, m)) {
      all_maps = false;
      continue;
    }
    pa.xmap = (int)(maps.size() / 128);
    maps.insert(maps.end(), m, m + 128);
  }
  if (premade) {
  } else if (!all_maps) {
    maps.clear();
    for (TcPassArg& pa : args) pa.xmap = -1;
  } else {
    kind = KIND_TC16T;
  }
  const int64_t LN = bf ? many_bf16_lines() : many_tc_lines();
  Phase ph;
  ph.kind = kind;
  std::vector<std::pair<double, int>> groups;  // (cost, pass)
  for (size_t i = 0; i < args.size(); ++i) groups.push_back({(double)args[i].d.N * args[i].d.N, (int)i});
  std::stable_sort(groups.begin(), groups.end(),
                   [](const std::pair<double, int>& x, const std::pair<double, int>& y) { return x.first > y.first; });
  const int nb = mp->grid_tc;
  std::vector<std::vector<TcItem>> per_block(nb);
  // least loaded block first (ties: lower index)
  typedef std::pair<double, int> Load;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int b = 0; b < nb; ++b) heap.push({0.0, b});
  for (const auto& gr : groups) {
    const TcPassArg& pa = args[gr.second];
    const int N = (int)pa.d.N;
    const int64_t ctiles = (pa.d.ncols + LN - 1) / LN;
    const int mts = bf ? many_bf16_row_blocks(N) : many_tc_row_blocks(N);
    const double per_group = (2.0 * N / 32) * (2.0 * N);  // K chunks x real rows, all row blocks
    for (int64_t ct = 0; ct < ctiles; ++ct) {
      Load l = heap.top();
      heap.pop();
      for (int mt = 0; mt < mts; ++mt) {
        TcItem w;
        w.ct = ct;
        w.arg = gr.second;
        w.mt = mt;
        per_block[l.second].push_back(w);
      }
      l.first += per_group;
      heap.push(l);
    }
  }
  std::vector<TcItem> flat;
  std::vector<long long> first(nb + 1, 0);
  for (int b = 0; b < nb; ++b) {
    first[b] = (long long)flat.size();
    flat.insert(flat.end(), per_block[b].begin(), per_block[b].end());
  }
  first[nb] = (long long)flat.size();
  const size_t abytes = (args.size() * sizeof(TcPassArg) + 255) & ~size_t(255);
  const size_t fbytes = ((size_t)(nb + 1) * sizeof(long long) + 255) & ~size_t(255);
  const size_t ibytes = (flat.size() * sizeof(TcItem) + 255) & ~size_t(255);
  const size_t bytes = abytes + fbytes + ibytes + maps.size();
  void* m = nullptr;
  cudaError_t e = cudaMalloc(&m, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *err = std::string("work list: ") + cudaGetErrorString(e);
    return FFX_ENOMEM;
  }
  ph.d_targs = (TcPassArg*)m;
  ph.d_first = (long long*)((char*)m + abytes);
  ph.d_titems = (TcItem*)((char*)m + abytes + fbytes);
  ph.n_titems = (long long)flat.size();
  ph.d_xmaps = maps.empty() ? nullptr : (const void*)((char*)m + abytes + fbytes + ibytes);
  e = cudaMemcpy(ph.d_targs, args.data(), args.size() * sizeof(TcPassArg), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(ph.d_first, first.data(), first.size() * sizeof(long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ph.d_titems, flat.data(), flat.size() * sizeof(TcItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !maps.empty())
    e = cudaMemcpy((void*)ph.d_xmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(m);
    *err = std::string("work list upload: ") + cudaGetErrorString(e);
    return FFX_ECUDA;
  }
  phases.push_back(ph);
  return FFX_OK;
}

// Tensor-core phases of one mode: the same chains of steps as the dense
// phases, cut into items of 128 lines x 128 real rows.  Each step is one
// launch of the BF16 kernel over the passes it takes (BF16 plans, no gradient
// factors) and one launch of the split-TF32 kernel over the others, where a
// step has both kinds.
int build_tc_phases(ManyPlan* mp, int mode, std::string* err) {
  std::vector<Phase>& phases = mp->phases[mode];
  const int D = mp->max_dim;
  const int nphases = (mode == 2) ? 2 * D : D;
  for (int ph_i = 0; ph_i < nphases; ++ph_i) {
    const bool adj = (mode == 2 && ph_i >= D);
    const int r = adj ? ph_i - D : ph_i;
    std::vector<TcPassArg> args_tf, args_bf;
    for (const Instance& in : mp->inst) {
      if (r >= in.ndim) continue;
      const int n_i = in.ndim;
      const int k = adj ? n_i - 1 - r : r;
      const int step = adj ? n_i + r : r;
      const int last_step = (mode == 2) ? 2 * n_i - 1 : n_i - 1;
      const int axis = in.order[k];
      const AxisTab& at = mp->tabs[in.axis_tab[axis]];
      const size_t off_c = (size_t)in.off * sizeof(float2), off_d = (size_t)in.off * sizeof(float);
      auto wsb = [](int st) { return (st % 2 == 0) ? BASE_WS : BASE_WS2; };
      TcPassArg pa;
      std::memset(&pa, 0, sizeof(pa));
      pa.in_base = (step == 0) ? BASE_PSI0 : wsb(step - 1);
      pa.outc_base = BASE_NONE;
      pa.outd_base = BASE_NONE;
      if (step == last_step) {
        if (mode == 0)
          pa.outd_base = BASE_OUTD;
        else
          pa.outc_base = BASE_OUTC;
      } else {
        pa.outc_base = wsb(step);
      }
      pa.grad_base = (adj && r == 0) ? BASE_GRAD : BASE_NONE;
      int64_t outer = 1, inner = 1;
      for (int i = 0; i < axis; ++i) outer *= in.dims[i];
      for (int i = axis + 1; i < in.ndim; ++i) inner *= in.dims[i];
      DenseArgs& a = pa.d;
      a.in = (const float2*)(uintptr_t)off_c;
      a.out_c = pa.outc_base >= 0 ? (float2*)(uintptr_t)off_c : nullptr;
      a.out_d = pa.outd_base >= 0 ? (float*)(uintptr_t)off_d : nullptr;
      a.grad = pa.grad_base >= 0 ? (const float*)(uintptr_t)off_d : nullptr;
      a.outer = outer;
      a.inner = inner;
      a.M = in.M;
      a.batch = 1;
      a.ncols = outer * inner;
      a.N = at.N;
      const bool bf = at.bf[adj ? 1 : 0] != nullptr && pa.grad_base < 0;
      pa.tblk = bf ? at.bf[adj ? 1 : 0] : at.tc[adj ? 1 : 0];
      (bf ? args_bf : args_tf).push_back(pa);
    }
    int rc = deal_tc_phase(mp, KIND_TC16, args_bf, phases, err);
    if (rc == FFX_OK) rc = deal_tc_phase(mp, KIND_TC, args_tf, phases, err);
    if (rc) return rc;
  }
  return FFX_OK;
}

// The passes of one chain phase: every instance's pass r (of its n_i) along
// axis n_i - 1 - r, with T (adjoint: T^H) on planes of contiguous lines, or
// for the first forward pass the caller's FP32 input (tile maps made per
// input buffer); the output transposed -- point n of line c at c + n R, R the
// pass's lines -- as the next planes (the workspaces in turn: in_base WS2 for
// even r, WS for odd r, out the other) or, after the pass along axis 0, in
// the lattice's own order to out_last (BASE_OUTD densities, else a field).
int chain_phase(ManyPlan* mp, int r, bool adjoint, int out_last, std::vector<Phase>& phases, std::string* err) {
  std::vector<TcPassArg> args;
  std::vector<unsigned char> maps;
  std::vector<std::array<int64_t, 3>> call_maps;
  const bool fp32_in = (r == 0 && !adjoint);
  const int in_base = fp32_in ? BASE_PSI0 : (r % 2 == 0) ? BASE_WS2 : BASE_WS;
  const int ws_out = (r % 2 == 0) ? BASE_WS : BASE_WS2;
  const uint32_t* in_planes = (const uint32_t*)(in_base == BASE_WS2 ? mp->ws2 : mp->ws);
  for (const Instance& in : mp->inst) {
    if (r >= in.ndim) continue;
    const int axis = in.ndim - 1 - r;
    const AxisTab& at = mp->tabs[in.axis_tab[axis]];
    const int64_t R = in.M / at.N;
    TcPassArg pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.in_base = in_base;
    pa.outc_base = BASE_NONE;
    pa.outd_base = BASE_NONE;
    pa.grad_base = BASE_NONE;
    DenseArgs& a = pa.d;
    a.in = (const float2*)(uintptr_t)((size_t)in.off * (fp32_in ? sizeof(float2) : sizeof(uint32_t)));
    if (r == in.ndim - 1) {
      if (out_last == BASE_OUTD) {
        pa.outd_base = BASE_OUTD;
        a.out_d = (float*)(uintptr_t)((size_t)in.off * sizeof(float));
      } else {
        pa.outc_base = out_last;
        a.out_c = (float2*)(uintptr_t)((size_t)in.off * sizeof(float2));
      }
    } else {
      pa.outc_base = ws_out;
      pa.out_planes = 1;
      a.out_bf = (uint32_t*)(uintptr_t)((size_t)in.off * sizeof(uint32_t));
    }
    a.bf_plane = mp->total;
    a.outer = R;
    a.inner = 1;
    a.M = in.M;
    a.batch = 1;
    a.ncols = R;
    a.N = at.N;
    pa.tblk = at.bf[adjoint ? 1 : 0];
    unsigned char m[128];
    std::memset(m, 0, sizeof(m));  // the first pass's maps are made for each call's input
    if (!pa.tblk || (!fp32_in && !many_bf16_plane_map(in_planes + in.off, at.N, R, mp->total, m)))
      return FFX_EUNSUPPORTED;
    pa.xmap = (int)(maps.size() / 128);
    maps.insert(maps.end(), m, m + 128);
    if (fp32_in) call_maps.push_back({in.off, (int64_t)at.N, R});
    args.push_back(pa);
  }
  const int kind = fp32_in ? KIND_TC16P1 : KIND_TC16P;
  int rc = deal_tc_phase(mp, kind, args, phases, err, &maps);
  if (rc == FFX_OK && fp32_in) phases.back().call_maps = call_maps;
  return rc;
}

// BF16 chain phases, as the uniform plans' BF16 chains.  Forward modes (0:
// density, 1: field): the chain phases r = 0 .. D - 1 into the caller's
// output.  Backward (2): the forward chain writes each field to the caller's
// gradient buffer, a split phase forms 2 grad * field as BF16 planes (the
// second workspace) for every point, and the adjoint chain (T^H along the
// last axis first; the axes' factors commute) writes the gradient over the
// fields.  Returns FFX_EUNSUPPORTED (nothing built) where a plane map cannot
// be made.
int build_chain_phases(ManyPlan* mp, int mode, std::string* err) {
  std::vector<Phase> phases;
  const int D = mp->max_dim;
  int rc = FFX_OK;
  const int out_fwd = mode == 0 ? BASE_OUTD : BASE_OUTC;
  for (int r = 0; rc == FFX_OK && r < D; ++r) rc = chain_phase(mp, r, false, out_fwd, phases, err);
  if (rc == FFX_OK && mode == 2) {
    Phase split;
    split.kind = KIND_SPLITG;
    phases.push_back(split);
    for (int r = 0; rc == FFX_OK && r < D; ++r) rc = chain_phase(mp, r, true, BASE_OUTC, phases, err);
  }
  if (rc) {
    for (Phase& ph : phases) cudaFree(ph.d_targs);
    return rc;
  }
  mp->phases[mode] = phases;
  return FFX_OK;
}

// Phases of one mode.  mode 0: density, 1: field, 2: backward.
int build_phases(ManyPlan* mp, int mode, std::string* err) {
  if (mp->tc && mp->bf16 && build_chain_phases(mp, mode, err) == FFX_OK) return FFX_OK;
  if (mp->tc) return build_tc_phases(mp, mode, err);
  if (mp->dense) return build_dense_phases(mp, mode, err);
  std::vector<Phase>& phases = mp->phases[mode];
  const int D = mp->max_dim;
  const int fwd_kind = (mp->form == FFX_FORM_PAPER) ? KIND_FWD_PAPER : KIND_FWD_FOLD;
  const int nsteps = (mode == 2) ? 2 * D : D;
  for (int step = 0; step < nsteps; ++step) {
    const bool adj = (mode == 2 && step >= D);
    const int r = adj ? step - D : step;  // forward step r, or adjoint step r
    Phase ph;
    ph.kind = adj ? KIND_ADJ_FOLD : fwd_kind;
    std::vector<PassArgs> args;
    std::vector<std::pair<double, ManyItem>> items;
    for (const Instance& in : mp->inst) {
      if (r >= in.ndim) continue;
      const int k = adj ? in.ndim - 1 - r : r;  // pass index in the instance's forward order
      const int axis = in.order[k];
      const AxisTab& at = mp->tabs[in.axis_tab[axis]];
      const size_t off_c = (size_t)in.off * sizeof(float2), off_d = (size_t)in.off * sizeof(float);
      int in_base, outc_base = BASE_NONE, outd_base = BASE_NONE, grad_base = BASE_NONE;
      if (!adj) {
        const bool last = (k == in.ndim - 1);
        if (mode == 1) {
          in_base = (k == 0) ? BASE_PSI0 : BASE_OUTC;
          outc_base = BASE_OUTC;
        } else {
          in_base = (k == 0) ? BASE_PSI0 : BASE_WS;
          if (last && mode == 0)
            outd_base = BASE_OUTD;
          else
            outc_base = BASE_WS;
        }
      } else {
        const bool first = (r == 0);
        in_base = first ? BASE_WS : BASE_OUTC;  // the gradient buffer is passed as out_field
        outc_base = BASE_OUTC;
        if (first) grad_base = BASE_GRAD;
      }
      PassArgs a = pass_args_for(in, axis, at, off_c, off_c, off_d, off_d, outc_base >= 0, outd_base >= 0,
                                 grad_base >= 0);
      const int arg = (int)args.size();
      args.push_back(a);
      PassKernelInfo info;
      find_pass_kernel(at.N, ph.kind, &info);
      build_items(*mp, -1, info, arg, in, in.axis_tab[axis], in_base, outc_base, outd_base, grad_base, items);
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, ManyItem>& x, const std::pair<double, ManyItem>& y) {
                       return x.first > y.first;
                     });
    std::vector<ManyItem> flat;
    flat.reserve(items.size());
    for (auto& pi : items) flat.push_back(pi.second);
    const size_t bytes = args.size() * sizeof(PassArgs) + flat.size() * sizeof(ManyItem);
    void* m = nullptr;
    cudaError_t e = cudaMalloc(&m, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *err = std::string("work list: ") + cudaGetErrorString(e);
      return FFX_ENOMEM;
    }
    ph.d_args = (PassArgs*)m;
    ph.d_items = (ManyItem*)((char*)m + args.size() * sizeof(PassArgs));
    ph.n_items = (int)flat.size();
    e = cudaMemcpy(ph.d_args, args.data(), args.size() * sizeof(PassArgs), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(ph.d_items, flat.data(), flat.size() * sizeof(ManyItem), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(m);
      *err = std::string("work list upload: ") + cudaGetErrorString(e);
      return FFX_ECUDA;
    }
    phases.push_back(ph);
  }
  return FFX_OK;
}

const void* phase_func(int kind) {
  switch (kind) {
    case KIND_TC: return many_tc_func();
    case KIND_TC16: return many_bf16_func(0);
    case KIND_TC16T: return many_bf16_func(1);
    case KIND_TC16P: return many_bf16_func(2);
    case KIND_TC16P1: return many_bf16_func(4);
    case KIND_FWD_PAPER: return (const void*)many_kernel<KIND_FWD_PAPER>;
    case KIND_FWD_FOLD: return (const void*)many_kernel<KIND_FWD_FOLD>;
    case KIND_DENSE: return (const void*)many_dense_kernel;
    default: return (const void*)many_kernel<KIND_ADJ_FOLD>;
  }
}

// The tensor-core kernel's parameters for a phase and a call's buffers.
static_assert(NBASE <= kTcBases, "call bases");
TcParams tc_params(const ManyPlan* mp, const Phase& ph, const ManyCall& call) {
  TcParams tp;
  std::memset(&tp, 0, sizeof(tp));
  tp.args = ph.d_targs;
  tp.items = ph.d_titems;
  tp.block_first = ph.d_first;
  tp.n_items = ph.n_titems;
  tp.err = mp->dev_err;
  tp.xmaps = ph.d_xmaps;
  for (int b = 0; b < NBASE; ++b) tp.call.base[b] = call.base[b];
  return tp;
}

// Kernel-node parameters of a phase (params: the kernel's argument pointers).
void phase_node_params(const ManyPlan* mp, const Phase& ph, void** params, cudaKernelNodeParams* kp) {
  std::memset(kp, 0, sizeof(*kp));
  kp->func = (void*)phase_func(ph.kind);
  if (tc_kind(ph.kind)) {
    const bool bf = ph.kind != KIND_TC;
    kp->gridDim = dim3(mp->grid_tc);
    kp->blockDim = dim3(bf ? many_bf16_threads() : many_tc_threads());
    kp->sharedMemBytes = (unsigned)(bf ? many_bf16_smem() : many_tc_smem());
    kp->kernelParams = params;
    return;
  }
  if (ph.kind == KIND_DENSE) {
    kp->gridDim = dim3(mp->grid_dense);
    kp->sharedMemBytes = 0;  // static
  } else {
    kp->gridDim = dim3(ph.kind == KIND_ADJ_FOLD ? mp->grid_adj : mp->grid_fwd);
    kp->sharedMemBytes = (unsigned)mp->smem;
  }
  kp->blockDim = dim3(256);
  kp->kernelParams = params;
}

// A phase kernel node's argument values and their pointers, alive while the
// node is added or updated.
struct NodeArgs {
  int* counter;
  TcParams tp;
  const void* s_field;
  const void* s_grad;
  void* s_hi;
  void* s_lo;
  long long s_n2, s_m2;
  int s_shared, s_unsplit;
  void* params[8];
};

// Node parameters of phase k for a call's buffers.
void node_args(const ManyPlan* mp, Phase& ph, size_t k, const ManyCall& call, NodeArgs& na,
               cudaKernelNodeParams* kp) {
  na.counter = mp->counters + k;
  if (ph.kind == KIND_SPLITG) {
    // a backward chain's split: 2 grad * field, the fields in the caller's
    // gradient buffer, into BF16 planes in the second workspace (head plane,
    // then the tail plane `total` pairs on)
    na.s_field = call.base[BASE_OUTC];
    na.s_grad = call.base[BASE_GRAD];
    na.s_hi = mp->ws2;
    na.s_lo = (uint32_t*)mp->ws2 + mp->total;
    na.s_n2 = mp->total / 2;
    na.s_m2 = mp->total / 2;
    na.s_shared = 0;
    na.s_unsplit = 0;
    void* const args[8] = {(void*)&na.s_field, (void*)&na.s_grad, (void*)&na.s_hi, (void*)&na.s_lo,
                           (void*)&na.s_n2,    (void*)&na.s_m2,   (void*)&na.s_shared, (void*)&na.s_unsplit};
    for (int i = 0; i < 8; ++i) na.params[i] = args[i];
    std::memset(kp, 0, sizeof(*kp));
    kp->func = (void*)bf16_split_grad_func();
    kp->gridDim = dim3(bf16_split_grid(mp->total, mp->grid_tc));
    kp->blockDim = dim3(256);
    kp->sharedMemBytes = 0;
    kp->kernelParams = na.params;
    return;
  }
  if (tc_kind(ph.kind)) {
    na.tp = tc_params(mp, ph, call);
    na.params[0] = (void*)&na.tp;
  } else {
    na.params[0] = ph.kind == KIND_DENSE ? (void*)&ph.d_dargs : (void*)&ph.d_args;
    na.params[1] = (void*)&ph.d_items;
    na.params[2] = (void*)&ph.n_items;
    na.params[3] = (void*)&na.counter;
    na.params[4] = (void*)&call;
  }
  phase_node_params(mp, ph, na.params, kp);
}

// The graph of one mode: memset(counter_k) -> phase kernel k -> memset(counter_k+1) -> ...
int build_graph(ManyPlan* mp, int mode, const ManyCall& call, std::string* err) {
  if (mp->phases[mode].empty()) {
    int rc = build_phases(mp, mode, err);
    if (rc) return rc;
  }
  cudaGraph_t g;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) {
    *err = std::string("cudaGraphCreate: ") + cudaGetErrorString(e);
    return FFX_ECUDA;
  }
  cudaGraphNode_t prev = nullptr;
  std::vector<cudaGraphNode_t>& kn = mp->knodes[mode];
  kn.clear();
  std::vector<Phase>& phases = mp->phases[mode];
  for (size_t k = 0; k < phases.size(); ++k) {
    Phase& ph = phases[k];
    cudaMemsetParams ms;
    std::memset(&ms, 0, sizeof(ms));
    ms.dst = mp->counters + k;
    ms.value = 0;
    ms.elementSize = sizeof(int);
    ms.width = 1;
    ms.height = 1;
    cudaGraphNode_t mnode, knode;
    e = cudaGraphAddMemsetNode(&mnode, g, prev ? &prev : nullptr, prev ? 1 : 0, &ms);
    if (e != cudaSuccess) break;
    NodeArgs na;
    cudaKernelNodeParams kp;
    node_args(mp, ph, k, call, na, &kp);
    e = cudaGraphAddKernelNode(&knode, g, &mnode, 1, &kp);
    if (e != cudaSuccess) break;
    kn.push_back(knode);
    prev = knode;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&mp->exec[mode], g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    *err = std::string("graph build: ") + cudaGetErrorString(e);
    return FFX_ECUDA;
  }
  mp->graph[mode] = g;
  mp->last_call[mode] = call;
  return FFX_OK;
}

// The tile maps of a chain's first pass over the call's input, uploaded on the
// call's stream (ordered after the launches that used the previous ones).
int refresh_call_maps(ManyPlan* mp, int mode, const ManyCall& call, cudaStream_t s, std::string* err) {
  for (Phase& ph : mp->phases[mode]) {
    if (ph.call_maps.empty()) continue;
    std::vector<unsigned char> maps(ph.call_maps.size() * 128);
    for (size_t i = 0; i < ph.call_maps.size(); ++i) {
      const std::array<int64_t, 3>& g = ph.call_maps[i];
      const float2* base = (const float2*)call.base[BASE_PSI0] + g[0];
      if (!many_bf16_line_map(base, (int)g[1], g[2], maps.data() + 128 * i)) {
        *err = "tile map of the input";
        return FFX_ECUDA;
      }
    }
    cudaError_t e = cudaMemcpyAsync((void*)ph.d_xmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      *err = std::string("tile map upload: ") + cudaGetErrorString(e);
      return FFX_ECUDA;
    }
  }
  return FFX_OK;
}

int launch_mode(ManyPlan* mp, int mode, const ManyCall& call, cudaStream_t s, std::string* err) {
  int rc;
  if (!mp->exec[mode]) {
    if ((rc = build_graph(mp, mode, call, err))) return rc;
    if ((rc = refresh_call_maps(mp, mode, call, s, err))) return rc;
  } else if (std::memcmp(&call, &mp->last_call[mode], sizeof(call)) != 0) {
    if (call.base[BASE_PSI0] != mp->last_call[mode].base[BASE_PSI0] &&
        (rc = refresh_call_maps(mp, mode, call, s, err)))
      return rc;
    // new buffers: rewrite the phase kernels' call pointers in the executable graph
    std::vector<Phase>& phases = mp->phases[mode];
    for (size_t k = 0; k < phases.size(); ++k) {
      Phase& ph = phases[k];
      NodeArgs na;
      cudaKernelNodeParams kp;
      node_args(mp, ph, k, call, na, &kp);
      cudaError_t e = cudaGraphExecKernelNodeSetParams(mp->exec[mode], mp->knodes[mode][k], &kp);
      if (e != cudaSuccess) {
        *err = std::string("graph update: ") + cudaGetErrorString(e);
        return FFX_ECUDA;
      }
    }
    mp->last_call[mode] = call;
  }
  cudaError_t e = cudaGraphLaunch(mp->exec[mode], s);
  if (e != cudaSuccess) {
    *err = std::string("cudaGraphLaunch: ") + cudaGetErrorString(e);
    return FFX_ECUDA;
  }
  return FFX_OK;
}

}  // namespace

void many_destroy(ManyPlan* mp) {
  if (!mp) return;
  for (int m = 0; m < 3; ++m) {
    if (mp->exec[m]) cudaGraphExecDestroy(mp->exec[m]);
    if (mp->graph[m]) cudaGraphDestroy(mp->graph[m]);
    for (Phase& ph : mp->phases[m])
      cudaFree(tc_kind(ph.kind) ? (void*)ph.d_targs
               : ph.kind == KIND_DENSE                      ? (void*)ph.d_dargs
                                                            : (void*)ph.d_args);
  }
  if (mp->tc_mem) cudaFree(mp->tc_mem);
  if (mp->dense_mem) cudaFree(mp->dense_mem);
  cudaFree(mp->mem);
  delete mp;
}

int64_t many_total(const ManyPlan* mp) { return mp->total; }
int64_t many_kernels(const ManyPlan* mp, int mode) { return (int64_t)mp->phases[mode].size(); }
int64_t many_offset(const ManyPlan* mp, int i) { return (i < 0 || i >= mp->n) ? -1 : mp->inst[i].off; }
int many_form(const ManyPlan* mp) { return mp->form; }
bool many_bf16(const ManyPlan* mp) {
  if (!mp->tc || !mp->bf16) return false;
  for (const AxisTab& at : mp->tabs)
    if (at.bf[0]) return true;
  return false;
}
int many_max_dim(const ManyPlan* mp) { return mp->max_dim; }
int* many_device_errors(const ManyPlan* mp) { return mp->dev_err; }

// Tensor-core phases copy and store 16 bytes at a time: 16-byte aligned buffers.
bool tc_buffers_ok(const ManyPlan* mp, const void* a, const void* b, const void* c, std::string* err) {
  if (!mp->tc || ((((uintptr_t)a) | ((uintptr_t)b) | ((uintptr_t)c)) & 15) == 0) return true;
  *err = "the tensor-core phases of a many-instance plan take 16-byte aligned buffers";
  return false;
}

int many_expand(ManyPlan* mp, const void* psi0, float* out_d, void* out_c, cudaStream_t s, std::string* err) {
  if (!tc_buffers_ok(mp, psi0, out_d, out_c, err)) return FFX_EINVAL;
  if (mp->dense && out_c && out_c == psi0) {
    // a one-pass instance reads and writes the caller's buffer in the same
    // (not in-place) dense pass
    for (const Instance& in : mp->inst)
      if (in.ndim == 1 && in.dims[0] > DBM) {
        *err = "in-place field of a dense many-instance plan with a 1-D instance longer than 64 points";
        return FFX_EUNSUPPORTED;
      }
  }
  ManyCall c;
  std::memset(&c, 0, sizeof(c));
  c.base[BASE_PSI0] = psi0;
  c.base[BASE_WS] = mp->ws;
  c.base[BASE_WS2] = mp->ws2;
  c.base[BASE_OUTC] = out_c;
  c.base[BASE_OUTD] = out_d;
  return launch_mode(mp, out_d ? 0 : 1, c, s, err);
}

int many_backward(ManyPlan* mp, const void* psi0, const float* grad, void* grad_psi0, cudaStream_t s,
                  std::string* err) {
  if (!tc_buffers_ok(mp, psi0, grad, grad_psi0, err)) return FFX_EINVAL;
  if (mp->dense && grad_psi0 == psi0) {
    // a one-pass instance's first pass reads the caller's input and writes the
    // gradient buffer (its field) in the same (not in-place) dense pass
    for (const Instance& in : mp->inst)
      if (in.ndim == 1 && in.dims[0] > DBM) {
        *err = "in-place gradient of a dense many-instance plan with a 1-D instance longer than 64 points";
        return FFX_EUNSUPPORTED;
      }
  }
  ManyCall c;
  std::memset(&c, 0, sizeof(c));
  c.base[BASE_PSI0] = psi0;
  c.base[BASE_WS] = mp->ws;
  c.base[BASE_WS2] = mp->ws2;
  c.base[BASE_OUTC] = grad_psi0;
  c.base[BASE_GRAD] = grad;
  return launch_mode(mp, 2, c, s, err);
}

}  // namespace ffx
