// Internal types shared by the plan code and the line-pass kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ffx.h"

namespace ffx {

// Per-axis phase tables (device memory, filled once per plan).
//   P [q][n]  = exp(-2 pi i q n / (lam N))                       (eq. presA pre-chirp)
//   K [q][m]  = exp(2 pi i [l s/N - tau l^2 - (2 tau/lam) l q])  (eq. presB k-space phase)
//   Kf[q][m]  = K[q][m] * exp(2 pi i [q s/(lam N) - tau q^2/lam^2]) / (lam N)
//               (the q-only part of eq. presf, and the final scale, moved
//                before the fold of the fine spectrum)
//   F [q][nb] = exp(2 pi i [q s/(lam N) + q nb/N - tau q^2/lam^2]) / (lam N)
//               (eq. presf with the 1/N of the inverse FFT)
//   tw[k]     = exp(-2 pi i k / N)                               (FFT twiddles)
//   fold[r]   = m0 with lam*m0 = r (mod N) when gcd(lam,N) | r, else -1
// with s = (abar - a)/dx, tau = pi t / L^2, l the symmetric index of eq. kj
// (odd-N umklapp of Sec. 5.2 applied for q >= lam/2).
struct AxisTables {
  const float2* P;
  const float2* K;
  const float2* Kf;
  const float2* F;
  const float2* tw;
  const int* fold;
};

enum PassKind : int { KIND_FWD_PAPER = 0, KIND_FWD_FOLD = 1, KIND_ADJ_FOLD = 2 };

// One pass of the 1-D map (or its adjoint) along one lattice axis, over every
// line of a [B][outer][N][inner] complex64 array.
struct PassArgs {
  const float2* in;      // input lines (complex64)
  const float* grad;     // non-null: input element is 2 * grad * in (adjoint's first pass)
  float2* out_c;         // complex output (may equal in), or null
  float* out_d;          // density output, or null
  int64_t outer;         // product of the axes before this one (per realization)
  int64_t inner;         // product of the axes after this one (the axis stride)
  int64_t M;             // points per realization
  int64_t batch;         // realizations
  int64_t nlines;        // lines covered by the tile grid
  int acc;               // 1: out_d[M] += sum over the batch (tiles loop over b)
  int grad_shared;       // 1: grad is [M], shared by every realization
  int lam;               // magnification lam
  int g;                 // gcd(lam, N)
  int Np;                // N / g
  int qg;                // thread groups sharing one line's q-sum (0 or 1: none)
  AxisTables tab;
};

// Launch one pass.  Returns a cudaError_t.
typedef cudaError_t (*PassLauncher)(const PassArgs& a, int grid, cudaStream_t stream);

// A block holds `groups` line-groups of T threads (threads = groups * T).  With
// qg groups per line, a tile is groups / qg lines.
struct PassKernelInfo {
  PassLauncher launch;
  const void* func;   // kernel symbol (for occupancy queries)
  int threads;        // threads per block at most (groups * T)
  int lines;          // lines per tile with qg = 1 (= groups)
  int T;              // threads per line-group
  int max_qg;         // largest qg the kernel accepts (1 when lines need named barriers)
  size_t smem;        // dynamic shared memory bytes
};

inline int pass_lines_per_tile(const PassKernelInfo& k, int qg) { return k.lines / (qg > 1 ? qg : 1); }

// Kernel registry: returns false if no kernel exists for (N, kind).
bool find_pass_kernel(int N, int kind, PassKernelInfo* out);
bool supported_length(int64_t N);

// FFT-form passes with one or two terms (ffx_conv.cu), on lines of 16, 64,
// 256 or 1024 points without the ensemble sum: lam = 1 (kind KIND_FWD_PAPER,
// KIND_FWD_FOLD or KIND_ADJ_FOLD), lam = 2 (KIND_FWD_FOLD)
bool conv_supported(int N, int lam, int acc, int kind);
cudaError_t launch_conv(const PassArgs& a, int kind, int N, int sms, cudaStream_t s);

// Set the calling thread's message for ffx_last_error().
void set_last_error_message(const char* msg);

// Dense form of one axis pass (ffx_dense.cu): OUT = A * IN along the axis,
// A = T (forward) or T^H (adjoint), row-major [N][N] complex64.  Not safe in
// place when N > 64 (row blocks of one column run in different blocks).
struct DenseArgs {
  const float2* A;
  const float2* Aimg;  // lines <= 64: A's shared-memory image (see ffx_dense.cu)
  int* err;            // device error counter (bounded waits)
  const float2* in;
  const float* grad;   // non-null: input element is 2 * grad * in
  float2* out_c;
  float* out_d;
  int64_t outer, inner, M, batch;
  int64_t ncols;       // columns (lines) covered by the tile grid
  int N;
  int acc, grad_shared;
  int unsplit;  // tensor-core kernels: one TF32 product (operands rounded, no tails)
  // BF16 pass chains (ffx_tc16.cu): the input (in_bf) and/or the output
  // (out_bf) as BF16 head and tail planes of (re, im) pairs, bf_plane pairs
  // apart (the tail plane is absent from unsplit chains); the output's own
  // line decomposition (oouter, oinner; 0 = the input's)
  const uint32_t* in_bf;
  uint32_t* out_bf;
  int64_t bf_plane;
  int64_t oouter, oinner;
};
const void* dense_kernel_func();
cudaError_t launch_dense(const DenseArgs& a, int grid, cudaStream_t stream);
int64_t dense_tiles(int N, int64_t ncols);
constexpr int kDenseInPlaceMaxN = 64;
// lines of at most 64 points: a kernel with T resident in shared memory
const void* dense_small_func(int N);
size_t dense_small_smem(int N);
cudaError_t launch_dense_small(const DenseArgs& a, int grid, cudaStream_t stream);
int64_t dense_small_tiles(int N, int64_t ncols);
size_t dense_small_image_floats2(int N);
cudaError_t launch_dense_small_image(const float2* T, float2* img, int N, cudaStream_t s);
constexpr int kDenseMaxN = 1024;
// dense form on the tensor cores (ffx_tc.cu), split TF32, for lines of N
// points with N a multiple of 16 from 32 up to kDenseMaxN; in place only for
// N <= 64
bool dense_tc_supported(int N);
cudaError_t dense_tc_prepare();  // shared-memory attributes of the kernel's variants
size_t dense_tc_t_bytes(int N);
cudaError_t launch_dense_tc(const DenseArgs& a, const unsigned char* Tblk, int* err, int grid,
                            cudaStream_t stream);
int64_t dense_tc_tiles(int N, int64_t ncols);
cudaError_t launch_tc_build_t(const float2* T, unsigned char* Tblk, int N, cudaStream_t s);
// the same passes with BF16 operands (ffx_tc16.cu, kind::f16): split into
// heads and tails (three products), or unsplit with DenseArgs::unsplit; lines
// of N points with N a multiple of 32 from 64 up to kDenseMaxN; same items
// (dense_tc_tiles) and in-place rule as the split-TF32 kernel
bool dense_bf16_supported(int N);
size_t dense_bf16_t_bytes(int N);
cudaError_t dense_bf16_prepare();
cudaError_t launch_bf16_build_t(const float2* T, unsigned char* Tblk, int N, cudaStream_t s);
cudaError_t launch_dense_bf16(const DenseArgs& a, const unsigned char* Tblk, int* err, int grid, cudaStream_t s);
// whether BF16 planes can be read as TMA tiles here (the driver offers
// cuTensorMapEncodeTiled): the condition of the BF16 pass chain
bool dense_bf16_chain_supported();
// n complex values (n even, `in` 16-byte aligned) into BF16 head and tail
// planes (the tail `plane` pairs after the head; head only when unsplit)
cudaError_t launch_bf16_split(const float2* in, uint32_t* planes, int64_t n, int64_t plane, int unsplit, int sms,
                              cudaStream_t s);
// The same for a backward call's adjoint chain: planes of 2 g psi, g per point
// of each realization or (grad_shared) one [M] array for the batch.
cudaError_t launch_bf16_split_grad(const float2* field, const float* grad, int grad_shared, int64_t M,
                                   uint32_t* planes, int64_t n, int64_t plane, int unsplit, int sms, cudaStream_t s);
cudaError_t launch_identity(float2* I, int N, cudaStream_t s);

// The d passes of a small lattice (every axis <= 64 points, dense form) in one
// cooperative launch with grid-wide barriers between the passes (ffx_fused.cu).
struct FusedPass {
  const float2* in;   // the pass's input lines
  float2* out_c;      // complex output (the workspace, or the caller's field)
  float* out_d;       // density output of the last pass, or null
  float* out_col;     // detector image of the last pass (sum over its axis), or null
  float col_scale;    // lam_j dx_j: the magnified spacing along that axis
  const float2* img;  // T_j's shared-memory image in global memory ([N][65])
  int64_t outer, inner, ncols;
  int N, acc, img_off;  // img_off: position of the image in shared memory (float2 units)
};
struct FusedArgs {
  FusedPass pass[3];
  int npass;
  int64_t M, batch;
  int64_t img_floats2;  // sum of the images (Bs follows them in shared memory)
  unsigned* bar;        // [2]: grid-barrier arrivals, blocks done (the last block resets both)
  int* err;
  const unsigned char* ts[3];  // tensor-core variant: per pass, T_j's split 32-row slices
  // tensor-core variant: pass local_pass (> 0) starts each line tile once the
  // previous pass's four row blocks of the same tile are written (tile_done
  // counters, kFusedTileFlags of them, reset by the last block) instead of
  // after a grid barrier; -1: grid barriers only
  unsigned* tile_done;
  int local_pass;
  // polls before a wait on other blocks (grid barrier, tile counters) gives
  // up; waits on a block's own copies and tensor-core work keep kSpinLimit
  long long spin;
};
constexpr int kFusedTileFlags = 256;
constexpr long long kCrossBlockSpin = 1ll << 22;  // default of FusedArgs::spin
size_t fused_smem(const int* N, int npass);
// Tensor-core variant for lattices whose axes all have 64 points: 4 row
// blocks of 32 real rows; each block's T slice is head and tail of 32 rows x
// 128 K in core-matrix order (fused_tc_slice_bytes per axis, all 4 blocks).
size_t fused_tc_slice_bytes();
cudaError_t launch_fused_tc_slices(const float2* T, unsigned char* out, cudaStream_t s);
cudaError_t fused_tc_prepare(int* per_sm);
cudaError_t launch_fused_tc(const FusedArgs& a, int grid, cudaStream_t stream);
int fused_img_stride();
const void* fused_func();
int fused_threads();
cudaError_t launch_fused(const FusedArgs& a, int grid, size_t smem, cudaStream_t stream);

// Detector readout (ffx_column.cu): sums of a density [outer][N][inner] along
// N, and the fringe phase of eq. dphase2 per image row.
cudaError_t launch_axis_sum(const float* rho, int64_t outer, int N, int64_t inner, float scale, int acc, float* out,
                            int sms, cudaStream_t s);
cudaError_t launch_fringe(const float* img, int64_t rows, int64_t ny, int64_t rs, int64_t ys, double y0, double dy,
                          double D, double t, double* out, int sms, cudaStream_t s);

// Positive-P pairs (ffx_pairs.cu).
cudaError_t launch_conj_copy(const float2* in, float2* out, int64_t n, int sms, cudaStream_t s);
cudaError_t launch_pair_density(const float2* w1, const float2* w2, int64_t M, int64_t batch, int acc, float* out,
                                int sms, cudaStream_t s);
cudaError_t launch_dense_build(const float2* O, float2* T, float2* TH, int N, cudaStream_t s);

// Plans over many instances (ffx_many.cu).
struct ManyPlan;
int many_create(ManyPlan** out, int n, const ffx_instance_desc* d, uint32_t flags, std::string* err);
void many_destroy(ManyPlan* mp);
int64_t many_total(const ManyPlan* mp);
// kernels one call launches (its graph's phase nodes); mode 0 densities,
// 1 fields, 2 backward
int64_t many_kernels(const ManyPlan* mp, int mode);
int64_t many_offset(const ManyPlan* mp, int i);
int many_form(const ManyPlan* mp);
bool many_bf16(const ManyPlan* mp);  // some tensor-core passes take split BF16 operands
int many_max_dim(const ManyPlan* mp);
int* many_device_errors(const ManyPlan* mp);  // device count of launches that gave up on a wait
int many_expand(ManyPlan* mp, const void* psi0, float* out_d, void* out_c, cudaStream_t s, std::string* err);
int many_backward(ManyPlan* mp, const void* psi0, const float* grad, void* grad_psi0, cudaStream_t s,
                  std::string* err);

// Plan-time table fill (one launch per axis).
cudaError_t launch_fill_tables(int N, int lam, uint64_t c_sN, uint64_t c_tau, uint64_t c_2tl,
                               uint64_t c_slN, uint64_t c_tl2, const uint64_t* disp, float2* P, float2* K,
                               float2* Kf, float2* F, float2* tw, cudaStream_t stream);

}  // namespace ffx
