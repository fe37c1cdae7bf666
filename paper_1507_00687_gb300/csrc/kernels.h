// Kernel launchers (host side).  Internal to the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "plan.h"

namespace fmm {

constexpr int kRowOStep = 0;
constexpr int kRowIStep = 1;

cudaError_t launch_row_exp(const void* X, int dt, int64_t R, int64_t C, int64_t ld, const int* ce, int cs,
                           int* out, int mode, int* status, cudaStream_t st);
cudaError_t launch_col_exp(const void* X, int dt, int64_t R, int64_t C, int64_t ld, const int* re, int rs,
                           int* out, int* status, cudaStream_t st);
cudaError_t launch_zero_sentinel(int* p, int64_t n, cudaStream_t st);
cudaError_t launch_fill(int* p, int64_t n, int v, cudaStream_t st);
// Y = 2^(rs re_i + cs ce_k) X (exact), Y in fp32 (bf16 when X is bf16).
cudaError_t launch_apply_exp(const void* X, int dt, int64_t R, int64_t C, int64_t ld, const int* re, int rs,
                             const int* ce, int cs, void* Y, int64_t ldy, cudaStream_t st);

// One operand of the fused multiply as the kernel sees it: a tile has
// "t" rows (the M side for A, the N side for B) and "k" columns.  Element
// (t, k) of the logical operand is at ptr[t*ld + k] when kcontig, else at
// ptr[k*ld + t].
struct TileOperand {
  const void* ptr;
  int64_t ld;
  int dtype;     // kF32 / kBF16 / kF16
  int kcontig;   // 1: k is the contiguous index
  int vec_ok;    // 16-byte vector loads allowed along the contiguous index
  int64_t T, K;  // logical extents
  int64_t bt, bk;  // leaf block extents along t and k
  int blk_t_shift;  // term block packing: t block = (blk >> blk_t_shift) & 0xFFFF
  int blk_k_shift;  //                      k block = (blk >> blk_k_shift) & 0xFFFF
};

struct EpilogueArgs {
  float* C;
  int64_t ldc;
  int64_t M, N;
  int64_t bm, bn;  // leaf block extents
  const int* eA;   // C scale 2^(eA_i + eB_j), nullable
  const int* eB;
  int vec_ok;
};

struct GemmArgs {
  TileOperand a, b;
  EpilogueArgs c;
  const LeafDesc* leaves;
  int64_t num_leaves;
  int64_t kl;          // leaf K extent
  int64_t pm, pk, pn;  // leaf block grid (products of m0, k0, n0)
  int* status;
  uint64_t timeout_ns;
};

// Launch the fused recursive-fast-multiply kernel for a flattened plan.
cudaError_t launch_fused_gemm(const GemmArgs& args, int leaf_format, cudaStream_t st);

// Number of SMs of the current device (cached).
int device_sm_count();

}  // namespace fmm
