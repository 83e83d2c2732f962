// Many-instance phases on the tensor cores: the work list of one phase for
// the split-TF32 dense kernel of ffx_tc.cu (the pass of every instance's k-th
// axis, cut into items of 128 lines x 128 real output rows).
#pragma once

#include "ffx_internal.h"

namespace ffx {

// One instance pass: the dense pass arguments with byte offsets in place of
// pointers (rebased per call on the bases below; -1 = unused) and the pass's
// split operand blocks (launch_tc_build_t layout).
struct TcPassArg {
  DenseArgs d;
  const unsigned char* tblk;
  int in_base, outc_base, outd_base, grad_base;
  int xmap;  // BF16 phases: index of the input's tile map in TcParams::xmaps, or -1
  // BF16 chains: the output is BF16 head and tail planes (d.out_bf, an offset
  // on outc_base's buffer; d.bf_plane pairs apart), transposed
  int out_planes;
};

// One work item: line tile ct (128 lines) and row block mt of pass `arg`.
struct TcItem {
  long long ct;
  int arg, mt;
};

constexpr int kTcBases = 8;
struct TcBases {
  const void* base[kTcBases];
};

// Kernel parameters.  Uniform launches: the pass `a` with operand blocks
// `tblk`, items (line tile, row block) numbered row block fastest, block b
// taking items b, b + gridDim.x, ...  Many-instance launches: `items` over the
// passes `args`, block b taking items [block_first[b], block_first[b + 1]).
// `err` counts launches that gave up on a bounded wait.
struct TcParams {
  DenseArgs a;
  const unsigned char* tblk;
  const TcPassArg* args;
  const TcItem* items;
  const long long* block_first;  // gridDim.x + 1 entries
  long long n_items;
  TcBases call;
  int* err;
  // BF16 phases: tile maps (128-byte CUtensorMap objects) of contiguous lines
  // in the plan's own workspaces, indexed by TcPassArg::xmap
  const void* xmaps;
};

const void* many_tc_func();   // kernel(const TcParams), many-instance variant
int many_tc_threads();
size_t many_tc_smem();        // dynamic shared memory (with the gradient ring)
cudaError_t many_tc_prepare();
int many_tc_lines();          // lines per item
int many_tc_row_blocks(int N);

// The BF16 variant (ffx_tc16.cu) for lines of 32 to 256 points, a multiple
// of 16: the same work lists and parameters, with split BF16 operand blocks
// of T (launch_bf16_build_t layout) in TcPassArg::tblk.  No gradient passes.
// mode 0: FP32 input by per-thread copies; 1: FP32 contiguous lines by TMA
// tiles (every pass a tile map); 2: BF16 planes by TMA tiles (chains); 4: as
// 1 with a chain pass's transposed output (a chain's first pass)
const void* many_bf16_func(int mode);
int many_bf16_threads();
size_t many_bf16_smem();
cudaError_t many_bf16_prepare();
int many_bf16_lines();
int many_bf16_row_blocks(int N);
bool many_bf16_supported(int N);
// Encode the tile map of `lines` contiguous lines of N complex points at
// `base` (16-byte aligned) into map[128] (64-byte aligned); false if the
// driver cannot.
bool many_bf16_line_map(const float2* base, int N, int64_t lines, void* map);
// The same for BF16 head and tail planes of `lines` contiguous lines of N
// points: the head plane at `head` (16-byte aligned), the tail plane `plane`
// pairs after it (4 * plane a multiple of 16).
bool many_bf16_plane_map(const uint32_t* head, int N, int64_t lines, int64_t plane, void* map);
// The grid of launch_bf16_split for n points.
int bf16_split_grid(int64_t n, int sms);
// A backward chain's split (launch_bf16_split_grad's kernel) as a graph node:
// kernel(field float4*, grad float2*, hi uint2*, lo uint2*, n2, m2, shared, unsplit).
const void* bf16_split_grad_func();

}  // namespace ffx
