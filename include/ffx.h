/*
 * ffx -- free-flight expansion of a compact wavefunction onto a magnified
 * lattice, on one NVIDIA GB300 (sm_103a).
 *
 * The operation (Deuar, arXiv:1602.03395, Sec. 5.2, eq. FF with eqs. FFpsi,
 * presf, presB, presA, FFaux):  an initial field psi_n on the lattice
 * x_n = a + n dx (eq. xj), n = 0..M-1 per axis, surrounded by vacuum
 * (eq. vacuum), flies freely for a time t.  The result is produced on the
 * magnified lattice xbar_nbar = abar + nbar * lam * dx (eq. wbx) with the same
 * number of points, lam a positive integer per axis (Sec. 5.1).  The map is the
 * exact free flight of the vacuum-padded field on the periodic lattice of
 * lam*M points per axis, sampled every lam points (Sec. 5.1 derivation).
 * Units: hbar = m = 1; a physical hbar*t/m is passed as t.
 *
 * The library evaluates eq. FF axis by axis (every phase in it is a product
 * over axes, so the d-dimensional map is the tensor product of 1-D maps) with
 * CUDA kernels.  It then forms the density |Psibar|^2 (Sec. 2) and, on
 * request, sums it over an ensemble of realizations (Sec. 1).
 *
 * Conventions shared by every entry point
 *  - Arrays are row-major (C order); the last axis is contiguous.  A batch of
 *    B realizations is laid out [B][M_0]...[M_{d-1}].
 *  - Complex data is interleaved complex64 (float re, float im), 8-byte
 *    aligned.  Densities are float32.
 *  - Every data pointer is a DEVICE pointer owned by the caller; the library
 *    neither frees nor retains it.  The plan owns its phase tables and its
 *    workspace (device memory).
 *  - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *    void*; NULL means the legacy default stream).  No entry point except
 *    ffx_plan / ffx_plan_destroy synchronizes with the host, but where noted
 *    (a first call that allocates or uploads).
 *  - A plan's calls share its workspace: calls on one plan that overlap on the
 *    GPU race.  Issue them on one stream (or order them), one plan per
 *    concurrent stream.
 *  - Errors are returned as codes, never as exceptions.  ffx_last_error()
 *    gives a message for the most recent failure in the calling thread.
 *  - A plan may be used from one host thread at a time.
 */
#ifndef FFX_H
#define FFX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define FFX_OK           0
#define FFX_EINVAL       1  /* bad argument: dims, lam, spacing, pointer, size */
#define FFX_ENOMEM       2  /* device allocation failed */
#define FFX_ECUDA        3  /* a CUDA call failed; see ffx_last_error() */
#define FFX_EUNSUPPORTED 4  /* valid request this build has no kernel for */
#define FFX_ETIMEOUT     5  /* a kernel of the plan gave up on a bounded wait */

/* ---- plan flags -------------------------------------------------------- */
/* Form of the per-axis sum over the fine momentum index q (eq. FFpsi).
 * FFX_FORM_PAPER: every term runs presA (pre-chirp + FFT), presB (k-space
 *   phase + inverse FFT), then presf with the n'' gather of eq. FFaux, and
 *   the terms are summed (Sec. 5.2 as printed; 2*lam line FFTs per axis).
 * FFX_FORM_FOLD: the same sum re-associated: f^(q) times the inverse-FFT
 *   kernel at n'' equals a plain inverse-DFT kernel at the fine index
 *   (lam*m + q) mod M, so every term's k-space line is folded into one
 *   spectrum and a single inverse FFT follows (lam + 1 line FFTs per axis).
 *   Same map, same rounding class.
 * FFX_FORM_DENSE: the same per-axis map as an N x N complex matrix T_j,
 *   built at plan time by running the fold form on the N unit vectors, then
 *   applied as a batched complex matrix product (8*M_j flops per point instead
 *   of lam_j*(5 log2 M_j + 14)); lines up to 1024 points.
 * 0 (FFX_FORM_AUTO) chooses per axis among these four: a tuned choice from
 *   the cache named by the environment variable FFX_TUNE_CACHE if it holds
 *   one for this device and geometry, else measured at plan time with
 *   FFX_TUNE, else a fixed cost model (dense or tensor-core when 8 M_j is well
 *   below the FFT form's work). */
#define FFX_FORM_AUTO   0x0u
#define FFX_FORM_PAPER  0x1u
#define FFX_FORM_FOLD   0x2u
#define FFX_FORM_DENSE  0x3u
/* FFX_FORM_TC: the dense form on the tensor cores (tcgen05, TF32 operands
 *   split into head and tail, three products accumulated in FP32) for axes of
 *   N points with N a multiple of 16 from 32 up to 1024; other lengths, and
 *   buffers not aligned to 16 bytes, use FFX_FORM_DENSE. */
#define FFX_FORM_TC     0x4u
#define FFX_FORM_MASK   0xFu
/* With FFX_FORM_AUTO: time every form of every axis at plan time (a few ms,
 * on a batch of one, in temporary workspace), use the fastest, and append the
 * result to the FFX_TUNE_CACHE file when that variable is set. */
#define FFX_TUNE        0x20u
/* ffx_expand writes the SUM over the batch of |Psibar|^2, added to what
 * out_density holds ([M_0..M_{d-1}], out += sum_b rho_b), instead of one
 * density per realization.  The sum runs over b in order (deterministic). */
#define FFX_ACCUMULATE  0x10u
/* Keep one launch per axis pass.  Without it, a plan with two or three axes
 * that all take a dense form with at most 64 points runs ffx_expand and
 * ffx_expand_field on small batches (ffx_plan_fused) as ONE cooperative
 * launch (one block per SM, the d passes separated by grid-wide barriers,
 * every T_j resident in shared memory); same arithmetic, same results. */
#define FFX_UNFUSED     0x40u
/* With FFX_FORM_TC only: one tensor-core product per K-step, with the input
 * and T_j rounded to TF32 (round to nearest; to BF16 with FFX_TC_BF16) and no
 * tails.  A faster and less
 * accurate variant, reported beside the split one: its density error is of
 * order 1e-3 against the 2e-5 of the split products.  Such plans never fuse
 * their passes into one launch, and axes the tensor cores do not take keep
 * the FP32 dense form.  Any other form with this flag: FFX_EINVAL. */
#define FFX_TC_UNSPLIT  0x80u
/* With FFX_FORM_TC or FFX_FORM_AUTO (where it is the default, see
 * FFX_TC_TF32): the tensor-core passes of the streaming
 * kernel (lines of N points, N a multiple of 32 from 64 to 1024; the 64-point
 * plain passes with at most four items per block, the 32-point passes and the
 * fused launch keep split TF32) take BF16 operands on kind::f16 products:
 * every FP32 value v is split into hi = bf16(v) and lo = bf16(v - hi), and
 * X_hi T_hi, X_hi T_lo and X_lo T_hi are accumulated in FP32 (density error
 * of order 1e-6, within the 2e-5 of the FP32 path).  With FFX_TC_UNSPLIT
 * (FFX_FORM_TC only): one product on operands rounded to BF16, the reported
 * BF16 variant (density error of order 1e-3). */
#define FFX_TC_BF16     0x100u
/* Under FFX_FORM_AUTO the streaming tensor-core passes take split BF16
 * operands (as FFX_TC_BF16) unless this flag asks for split TF32 operands
 * throughout, or FFX_TC_UNSPLIT is given.  FFX_TC_TF32 with FFX_TC_BF16:
 * FFX_EINVAL. */
#define FFX_TC_TF32     0x200u

typedef struct ffx_plan_s* ffx_plan_t;

/*
 * ffx_plan -- build a plan for one lattice geometry and flight time.
 *
 *  out           receives the plan handle (set to NULL on failure).
 *  ndim          number of lattice axes, 1..3.
 *  dims[ndim]    M_j >= 1, points per axis (row-major order).  Each M_j must
 *                be a line length this build has a kernel for (see
 *                ffx_supported_length); others return FFX_EUNSUPPORTED.
 *  spacing[ndim] dx_j > 0 (Sec. 2.1: dx_j = L_j / M_j).
 *  t             flight time t_flight (eq. free0), any finite real.
 *  magnification[ndim]  lam_j >= 1, integers (Sec. 5.1 requires integer
 *                lam_j); values above 65536 return FFX_EINVAL.
 *  a[ndim]       input lattice offsets a_j (eq. xj), or NULL for -L_j/2.
 *  abar[ndim]    output lattice offsets abar_j (eq. wbx), or NULL for
 *                a_j + s_j dx_j with s_j = -floor((lam_j - 1) M_j / 2), which
 *                centres the magnified box on the input box.  Any real
 *                offset is accepted.
 *  flags         FFX_FORM_* | FFX_ACCUMULATE.
 *
 * Runs on the current CUDA device, allocates the plan's phase tables there
 * and fills them (exact integer / 64-bit fixed-point phase reduction, then
 * double-precision sincospi), and synchronizes before returning.
 */
int ffx_plan(ffx_plan_t* out, int ndim, const int64_t* dims, const double* spacing,
             double t, const int32_t* magnification, const double* a,
             const double* abar, uint32_t flags);

/* Release the plan's device memory.  NULL is accepted.  Synchronizes the
 * device first, so work still queued on the plan finishes. */
int ffx_plan_destroy(ffx_plan_t plan);

/*
 * ffx_plan_dispersion -- as ffx_plan, for a spectrum other than the free
 * particle's (Sec. 7, Generalizations): the momentum-space evolution
 * exp(-i t omega(k)) replaces exp(-i t k^2 / 2) of eq. free0.  The dispersion
 * is separable, omega(k) = sum_j omega_j(k_j), so the map keeps its per-axis
 * form.
 *
 *  omega       NULL (every axis free), or ndim host pointers: NULL for a free
 *              axis, else lam_j * dims[j] finite doubles, omega_j sampled at
 *              the huge-lattice wavevectors k_u = 2 pi u~ / (lam_j L_j),
 *              u = 0 .. lam_j dims[j] - 1, u~ the symmetric index of u on
 *              lam_j dims[j] points (u~ = u below half, u - lam_j dims[j] from
 *              half on).  Read once at plan creation.
 *  The phases t omega are reduced to turns in FP64 on the host; free axes
 *  keep the exact fixed-point reduction.  Every form and call of the plan
 *  applies the generalized map.
 */
int ffx_plan_dispersion(ffx_plan_t* out, int ndim, const int64_t* dims, const double* spacing, double t,
                        const int32_t* magnification, const double* a, const double* abar,
                        const double* const* omega, uint32_t flags);

/*
 * ffx_plan_many -- one plan over many instances of possibly different
 * lattices, magnifications and flight times (an ensemble of realizations,
 * Sec. 1), run as one persistent kernel per axis pass over a work list of all
 * instances' tiles, the passes captured in one CUDA graph that is replayed on
 * every call.
 *
 *  descs[n_instances]  one geometry per instance (ndim 1..3, dims, spacing,
 *                      t, magnification; offsets a/abar if has_offsets, else
 *                      the defaults of ffx_plan).  Line lengths must be one of
 *                      16, 32, 48, 64, 96, 128, 192, 256 (FFX_EUNSUPPORTED
 *                      otherwise).
 *  flags               FFX_FORM_PAPER, FFX_FORM_FOLD, FFX_FORM_DENSE,
 *                      FFX_FORM_TC or FFX_FORM_AUTO (the dense maps when they
 *                      cost less than the fold form on every instance axis,
 *                      else fold; dense maps on the tensor cores when every
 *                      line length is a multiple of 16 from 32); with
 *                      FFX_FORM_TC or FFX_FORM_AUTO, FFX_TC_TF32 (split TF32
 *                      operands throughout) or FFX_TC_BF16 (the default, see
 *                      below); FFX_ACCUMULATE, FFX_TUNE, FFX_UNFUSED and
 *                      FFX_TC_UNSPLIT are rejected (FFX_EINVAL; instances on
 *                      different lattices have no common density grid).
 *
 * The dense form builds T_j and T_j^H of every distinct axis geometry at plan
 * creation (the fold pass on the unit vectors) and runs each phase as one
 * persistent kernel over 64 x 32 tiles of all instances (FP32); it adds a
 * second packed workspace.  FFX_FORM_TC (and the automatic form, see above)
 * also builds their tensor-core operand blocks and runs each phase as
 * persistent launches over items of 128 lines x 128 real rows, one block per
 * SM: on split BF16 operands (kind::f16 products, density error of order
 * 1e-6), or with FFX_TC_TF32 on split TF32 operands.  Calls on BF16 operands
 * run as chains: each instance's passes from its last axis to its first, the
 * intermediate results kept as BF16 head and tail planes in the workspaces;
 * a backward call runs the forward chain into its gradient buffer, one launch
 * that splits 2 grad * field into planes, and the adjoint chain.
 * Every call of a plan on the tensor cores takes 16-byte aligned buffers
 * (FFX_EINVAL otherwise); the first forward call with a new input buffer
 * uploads the chain's tile maps of it from host memory on the call's stream
 * (a copy that waits for the stream's earlier work), so such a call cannot
 * be captured into a CUDA graph.  A plan
 * with a 16-point axis keeps the FP32 phases (ffx_plan_form reports which).
 * Dense passes are not in place for
 * lines over 64 points, so an in-place ffx_expand_field with a 1-D instance
 * longer than 64 points returns FFX_EUNSUPPORTED.  ffx_plan_device_errors
 * counts tensor-core phases that gave up on a bounded wait.
 *
 * Data are packed: instance i occupies points [off_i, off_i + M_i) of the
 * input, of the density or field output, and of the gradient buffers, with
 * off_i from ffx_plan_many_offset (instances in order, no padding).  Calls
 * take batch = 1 (the whole set).  ffx_expand, ffx_expand_field and
 * ffx_expand_backward accept such a plan; ffx_expand_adjoint does not
 * (FFX_EUNSUPPORTED).  The plan allocates its tables and a packed workspace
 * at creation; the first call of each kind builds its graph (host work and a
 * small device allocation for the work list).
 */
typedef struct ffx_instance_desc {
  int32_t ndim;
  int64_t dims[3];
  double spacing[3];
  double t;
  int32_t magnification[3];
  int32_t has_offsets;
  double a[3];
  double abar[3];
} ffx_instance_desc;

int ffx_plan_many(ffx_plan_t* out, int n_instances, const ffx_instance_desc* descs, uint32_t flags);

/* Packed offset (in points) of instance i, or -1 (not a many-plan, bad i). */
int64_t ffx_plan_many_offset(ffx_plan_t plan, int i);

/* Points per call: M for a single-lattice plan, sum of M_i for a many-plan. */
int64_t ffx_plan_points(ffx_plan_t plan);

/*
 * ffx_expand -- densities after free flight (eq. FF, then |Psibar|^2).
 *
 *  psi0         device complex64 [batch][M...], read only.
 *  batch        number of realizations B >= 0.  B = 0 does nothing.
 *  out_density  device float32: [batch][M...] (one density per realization),
 *               or [M...] with FFX_ACCUMULATE (out += sum_b |Psibar_b|^2).
 *               Must not overlap psi0.
 *  stream       cudaStream_t or NULL.
 *
 * Uses the plan's workspace (batch * M complex64 for d >= 2), grown on demand:
 * the first call with a larger batch allocates (cudaMalloc, host-synchronous).
 */
int ffx_expand(ffx_plan_t plan, const void* psi0, int64_t batch, float* out_density,
               void* stream);

/*
 * ffx_expand_host -- ffx_expand on host buffers, one call per step: copies
 * psi0_host ([batch][M] complex64 in host memory) into a device staging
 * buffer of the plan, runs ffx_expand on it, and copies the densities back to
 * out_host ([batch][M] float32, or [M] with FFX_ACCUMULATE: then out_host's
 * values are copied in first and the batch sum is added to them).  A
 * many-instance plan takes batch = 1 and its packed layout.
 *
 * Asynchronous on `stream` like ffx_expand: the host buffers must stay valid,
 * and out_host unread, until the stream reaches the copies
 * (cudaStreamSynchronize); page-locked (pinned) host memory lets the copies
 * overlap other work.  The staging buffers are allocated on first use and
 * grown with larger batches (cudaMalloc, which synchronizes the device), and
 * are shared by calls on the same plan: calls on different streams need
 * different plans.  Returns FFX_EINVAL (NULL pointers, batch < 0, a
 * many-instance batch other than 1), FFX_ENOMEM, FFX_ECUDA, or ffx_expand's
 * codes.
 */
int ffx_expand_host(ffx_plan_t plan, const void* psi0_host, int64_t batch, float* out_host, void* stream);

/*
 * ffx_expand_field -- the complex field Psibar itself, [batch][M...] complex64.
 * out_field may equal psi0 (in place); otherwise the two must not overlap.
 * Needs no workspace.  The phase of Psibar is that of the magnified lattice,
 * which Sec. 5.4 warns is not fit for further evolution; its density is exact.
 */
int ffx_expand_field(ffx_plan_t plan, const void* psi0, int64_t batch, void* out_field,
                     void* stream);

/*
 * ffx_expand_backward -- gradient of a real loss L(rho) with respect to psi0.
 *
 *  grad_density  device float32 dL/drho: [batch][M...], or [M...] with
 *                FFX_ACCUMULATE (the same gradient reaches every realization).
 *  grad_psi0     device complex64 [batch][M...], overwritten with
 *                T^H (2 * grad_density * T psi0), i.e. dL/dRe(psi0) +
 *                i dL/dIm(psi0) (PyTorch's convention for complex inputs).
 *                T^H is the adjoint of the per-axis maps, applied in reverse
 *                axis order; T psi0 is recomputed, not stored.
 *  Uses the plan's workspace (batch * M complex64).
 */
int ffx_expand_backward(ffx_plan_t plan, const void* psi0, const float* grad_density,
                        int64_t batch, void* grad_psi0, void* stream);

/* Apply only the adjoint map: grad_psi0 = T^H g for a complex64 field g
 * ([batch][M...]).  g_in and g_out may be equal (in place). */
int ffx_expand_adjoint(ffx_plan_t plan, const void* g_in, int64_t batch, void* g_out,
                       void* stream);

/* ---- expansion without device allocation --------------------------------- */
/* Sizes of the library's static device scratch (every GPU that loads the
 * library holds them until the process exits: 8 MiB + 2 MiB + 32 KiB). */
#define FFX_NOALLOC_MAX_FIELD (1 << 20) /* complex64 elements: batch * M, ndim >= 2 */
#define FFX_NOALLOC_MAX_TABLE (1 << 18) /* complex64: sum over axes of 4*lam_j*M_j + M_j */
#define FFX_NOALLOC_MAX_FOLD  8192      /* ints: sum over axes of M_j */

/*
 * ffx_expand_noalloc -- the map of ffx_plan + ffx_expand, always with the fold
 * form (FFX_FORM_FOLD) and one density per realization, in one call that
 * allocates no memory.  The paper
 * has no counterpart; this exists for callers that cannot call cudaMalloc
 * while they run: a host framework that has reserved nearly all device memory
 * for its own pool (a raw cudaMalloc would fail or fragment it), or a
 * real-time loop that forbids allocation, and the device-wide synchronisation
 * of cudaMalloc/cudaFree, after start-up.
 *
 * Arguments are those of ffx_plan (dims, spacing, t, magnification, a, abar;
 * a/abar nullable) and ffx_expand (psi0 [batch][M...] complex64 and
 * out_density [batch][M...] float32, caller-owned device memory; stream).
 * Instead of a plan's tables and workspace it uses the static device arrays
 * sized above: the phase tables are rebuilt there on every call (small
 * kernels on `stream`), and for ndim >= 2 the field between axis passes is
 * kept there.  Sizes beyond FFX_NOALLOC_MAX_* return FFX_EINVAL with the
 * limit named in ffx_last_error(); unsupported lengths FFX_EUNSUPPORTED.
 *
 * The first call on a device looks up the device addresses of the static
 * arrays (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture.  Every call, on every stream, shares the
 * same arrays, and they keep the last call's contents (each call rewrites all
 * it reads, so nothing has to start at zero): calls that overlap on the GPU
 * race.  Serialise them, e.g. by issuing them all on one stream.
 */
int ffx_expand_noalloc(int ndim, const int64_t* dims, const double* spacing, double t,
                       const int32_t* magnification, const double* a, const double* abar,
                       const void* psi0, int64_t batch, float* out_density, void* stream);

/* ---- introspection ------------------------------------------------------ */

/* 1 if this build has a line kernel for length n, else 0. */
int ffx_supported_length(int64_t n);

/*
 * ffx_expand_column -- the detector image (Sec. 6): the density integrated
 * along one lattice axis, as the paper's detector integrates over the imaging
 * direction (rho(x, y) = integral dz |Psi|^2, Fig. 4).
 *
 *  axis          the lattice axis integrated over (0 .. ndim-1).
 *  out_column    device float32, the lattice without that axis:
 *                [batch][dims without axis], or [dims without axis] added to
 *                (+=) with FFX_ACCUMULATE (summed over the batch).  Entry =
 *                lam_axis * spacing_axis * sum over the axis of |Psibar|^2
 *                (the magnified lattice's spacing along the axis, eq. wbx).
 *  The map runs with the integrated axis as the last pass.  Small lattices
 *  that fuse (ffx_plan_fused) sum inside the fused launch; otherwise the
 *  densities go to plan workspace and one more launch sums them.  Sums run in
 *  a fixed order (deterministic).  Not for many-instance plans
 *  (FFX_EUNSUPPORTED).
 */
int ffx_expand_column(ffx_plan_t plan, const void* psi0, int64_t batch, int axis, float* out_column,
                      void* stream);

/*
 * ffx_expand_positive_p -- the density of positive-P pairs after free flight
 * (Sec. 7, Generalizations).  The field psi0 (for the annihilation operator)
 * evolves by the map T, the independent field psi0_plus (for the creation
 * operator) by its complex conjugate conj(T); the normally ordered density is
 *   out_density = Re(Psibar+ * Psibar),  Psibar = T psi0, Psibar+ = conj(T) psi0_plus,
 * per realization [batch][M...], or with FFX_ACCUMULATE summed over the batch
 * (in order) and added to out_density [M...].  With psi0_plus = conj(psi0) it
 * is |Psibar|^2.  conj(T) psi0_plus is computed as conj(T conj(psi0_plus)):
 * both fields run through the same passes.  Uses plan workspace (two
 * batch * M complex64 fields besides the passes' own).  Not for
 * many-instance plans (FFX_EUNSUPPORTED).
 */
int ffx_expand_positive_p(ffx_plan_t plan, const void* psi0, const void* psi0_plus, int64_t batch,
                          float* out_density, void* stream);

/* Positions of the magnified output lattice along `axis` (eq. wbx):
 * xbar_n = *x0 + n * *step, with *x0 = abar_axis, *step = lam_axis * spacing_axis. */
int ffx_plan_output_axis(ffx_plan_t plan, int axis, double* x0, double* step);

/*
 * ffx_fringe_phase -- the relative phase of two clouds split by D along y,
 * read from their interference fringes (eq. dphase2, hbar = m = 1):
 * Delta theta_0 = y_peak * D / t, y_peak the density peak nearest y = 0.
 *
 *  image       device float32 density or detector image; element (r, j) at
 *              image[r * row_stride + j * y_stride], r < rows, j < ny (ny >= 3),
 *              sampled at y_j = y0 + j * dy (dy > 0).
 *  out_phase   device float64 [rows]: per row, the interior local maximum
 *              (v[j] > v[j-1] and v[j] >= v[j+1]) with the smallest |y_j| (the
 *              lower j on a tie), refined to the vertex of the parabola through
 *              log v at j-1, j, j+1 (FP64; no refinement if a value is not
 *              positive), times D / t.  NaN for a row with no interior maximum.
 *              Phases are not wrapped.
 *  Works on any image; the paper has no counterpart for the GPU kernel, it
 *  states the estimate.  FFX_EINVAL for bad sizes, t = 0, dy <= 0, a NULL or
 *  misaligned pointer.
 */
int ffx_fringe_phase(const float* image, int64_t rows, int64_t ny, int64_t row_stride, int64_t y_stride,
                     double y0, double dy, double D, double t, double* out_phase, void* stream);

/* Bytes of plan-owned workspace a call with this batch uses. */
int64_t ffx_workspace_bytes(ffx_plan_t plan, int64_t batch);

/* 1 if the plan's streaming tensor-core passes take BF16 operands
 * (FFX_TC_BF16, or the automatic form's default), 0 if not, -1 for a NULL
 * plan; many-instance plans: 1 if some of their tensor-core phases do. */
int ffx_plan_tc_bf16(ffx_plan_t plan);

/* The form every axis runs (FFX_FORM_PAPER, _FOLD, _DENSE or _TC), or
 * FFX_FORM_AUTO if the axes differ. */
int ffx_plan_form(ffx_plan_t plan);

/* The form lattice axis `axis` runs, or -1. */
int ffx_plan_axis_form(ffx_plan_t plan, int axis);

/* Number of kernel launches one ffx_expand / ffx_expand_backward call makes
 * with a batch of one.  A call that runs as a BF16 chain
 * (ffx_plan_bf16_chain) makes one more: the split of its input into BF16
 * planes (in ffx_expand_backward: the forward half of a 3-D plan). */
int ffx_launches_per_call(ffx_plan_t plan, int backward);

/* The largest batch for which ffx_expand and ffx_expand_field run as one
 * fused launch (see FFX_UNFUSED): a batch whose first pass has at most two
 * 32-line tiles per SM, and, under FFX_FORM_AUTO, below the batch whose
 * per-axis passes would all run on the tensor cores (see
 * ffx_plan_call_form).  0 if the plan never fuses, -1 for a NULL plan.
 * When every axis has 64 points and the plan's form is FFX_FORM_AUTO or
 * FFX_FORM_TC, the fused launch forms its products on the tensor cores
 * (split TF32, as FFX_FORM_TC) for a 16-byte-aligned psi0; otherwise with the
 * FP32 dense arithmetic, bitwise equal to the per-axis FFX_FORM_DENSE passes. */
int64_t ffx_plan_fused(ffx_plan_t plan);

/* The form whose kernel a forward call with this batch runs on lattice axis
 * `axis`: for a fused call the fused launch's arithmetic (FFX_FORM_TC or
 * FFX_FORM_DENSE, see ffx_plan_fused); else the axis's form, except that
 * under FFX_FORM_AUTO a dense axis whose pass covers at least 32 lines (in
 * all, batch x lines) and either has lines of at least 96 points or at least
 * 64 tensor-core items (128 lines x 128 real rows) runs on the tensor cores
 * (FFX_FORM_TC; a 16-byte-misaligned buffer still takes the FP32 kernel).
 * Dense passes over fewer than 32 lines run the FP32 few-lines kernel.
 * Results of the two kernels agree to rounding (within the FP32 tolerance),
 * not bit for bit; explicit forms never switch.  -1 on a bad argument or a
 * many-instance plan. */
int ffx_plan_call_form(ffx_plan_t plan, int axis, int64_t batch);

/* Kernels the plan's calls have launched so far, counted as each call
 * enqueues them (a call captured into a CUDA graph counts once, at capture;
 * replays of the graph do not count); -1 for a NULL plan.  The difference
 * across one call is that call's number of kernel launches. */
int64_t ffx_plan_launch_count(ffx_plan_t plan);

/* 1 if ffx_expand over `batch` realizations (16-byte aligned buffers) runs
 * as a BF16 chain, else 0; -1 on a bad argument (ffx_expand_field and the
 * forward half of ffx_expand_backward take the same chains).  A
 * BF16 chain runs when every axis's pass of the call would take the
 * streaming BF16 tensor-core kernel (FFX_TC_BF16, or the automatic form's
 * default, and ffx_plan_call_form's choice FFX_FORM_TC): the passes run from
 * the last axis to the first (ffx_plan_pass_order), each writing its output
 * transposed -- point n' of a line goes n' (M / N_j) places after the line's
 * first -- so that the next pass's lines are contiguous, and the fields
 * between passes are kept as BF16 head and tail planes (bf16(v),
 * bf16(v - bf16(v)) of each FP32 value v: the operands the next pass would
 * split it into, so the results are those of the per-axis passes in the same
 * order).  The planes use the plan's two field workspaces. */
int ffx_plan_bf16_chain(ffx_plan_t plan, int64_t batch);

/* Forward pass order: writes the lattice axis of pass k to order[k],
 * k = 0..ndim-1.  The adjoint runs the same axes in reverse. */
int ffx_plan_pass_order(ffx_plan_t plan, int32_t* order);

/* Profiling hook.  events: n_events cudaEvent_t handles (created by the
 * caller with timing enabled, passed as void*).  Every later kernel launch of
 * the plan records events[2i] just before and events[2i+1] just after itself
 * on the call's stream, i counting launches, until the array is full.
 * NULL (or n_events = 0) switches tracing off.  The library keeps the
 * pointer, not a copy: the array must outlive the traced calls.  Calls made
 * while the stream is being captured into a CUDA graph record the events as
 * event-record nodes of the graph (cudaEventRecordExternal), so they time the
 * launches when the graph runs.  Every entry point except ffx_plan,
 * ffx_plan_many and ffx_plan_destroy is stream-ordered and can be captured once
 * the plan's workspace has grown to the batch used (a first, uncaptured call
 * grows it). */
int ffx_plan_trace(ffx_plan_t plan, void* const* events, int64_t n_events);

/* Number of events recorded since the last ffx_plan_trace call. */
int64_t ffx_plan_trace_count(ffx_plan_t plan);

/* Waits that ran out inside the plan's kernels so far (tensor-core passes
 * bound every wait on the tensor cores and count a timeout here instead of
 * hanging); 0 when all is well.  Synchronizes with the device.
 *
 * Where the device has native atomics to host memory (cudaDevAttr-
 * HostNativeAtomicSupported, e.g. a GB300 next to its Grace CPU), the count
 * lives in mapped page-locked host memory, and every stream-ordered entry
 * point of a single-lattice plan (ffx_expand, _host, _field, _column,
 * _positive_p, _backward, _adjoint) first checks it without synchronizing:
 * if it grew since the last such report, the call launches nothing and returns
 * FFX_ETIMEOUT (once per new timeout), since the earlier call's output is not
 * valid.  A timeout is seen once its launch has finished, e.g. after a stream
 * synchronization.  Many-instance plans report through this function only. */
int ffx_plan_device_errors(ffx_plan_t plan);

/* Poll budget of the waits in which a block of the plan's fused launch
 * (ffx_plan_fused) waits for OTHER blocks: its grid-wide barriers and the
 * per-tile counters between passes.  polls >= 1 sets it; 0 restores the
 * default (2^22 polls, far beyond a healthy wait).  A wait that runs out sets
 * the block's abort flag: the block stops its passes, waits (with the normal
 * bound) for its own bulk copies and tensor-core work, frees its tensor
 * memory, counts the timeout (ffx_plan_device_errors) and exits; the next call
 * returns FFX_ETIMEOUT.  Waits on a block's own copies and products keep their
 * fixed bound.  The paper has no counterpart: this exercises the failure
 * path of the bounded waits.  FFX_EINVAL for polls < 0. */
int ffx_plan_set_wait_limit(ffx_plan_t plan, int64_t polls);

/* Static strings for return codes; never NULL. */
const char* ffx_error_string(int code);

/* Message for the most recent failure in the calling thread ("" if none). */
const char* ffx_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FFX_H */
