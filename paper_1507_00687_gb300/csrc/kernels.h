// Kernel launchers (host side).  Internal to the library.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "plan.h"

namespace fmm {

constexpr int kRowOStep = 0;
constexpr int kRowIStep = 1;

// skip (may be NULL): a device flag; when it is set at launch time the
// reduction does nothing (an adaptive iteration that has stopped).
cudaError_t launch_row_exp(const void* X, int dt, int64_t R, int64_t C, int64_t ld, const int* ce, int cs,
                           int* out, int mode, int* status, cudaStream_t st, const int* skip = nullptr);
cudaError_t launch_col_exp(const void* X, int dt, int64_t R, int64_t C, int64_t ld, const int* re, int rs,
                           int* out, int* status, cudaStream_t st, const int* skip = nullptr);
// Adaptive Alg. 3: test one step's factors 2^(next - cur) against [lo, hi]
// and adopt next; then record the step and stop when it was tested and
// passed (ctl: stopped, failed, steps applied).
cudaError_t launch_scale_accept(const int* next, int* cur, int64_t n, int lo, int hi, int* ctl, cudaStream_t st);
cudaError_t launch_scale_stop(int* ctl, int tested, int t, int* steps_out, cudaStream_t st);
cudaError_t launch_zero_sentinel(int* p, int64_t n, cudaStream_t st);
// The step pair O, I of Alg. 3 from no scaling (M, K, N > 0) in two
// launches: eA, eB (O step) then d (I step); no initialisation needed.
cudaError_t launch_oi_from_zero(const void* A, const void* B, int dt, int64_t M, int64_t K, int64_t N, int64_t lda,
                                int64_t ldb, int* eA, int* d, int* eB, int* status, cudaStream_t st);

// One problem of a batched reduction (rows: R x C, ld; shift: column
// exponents for row reductions, row exponents for column reductions, sign
// `sign`, nullable; out: per-row or per-column result).  gx, rows_per_cta:
// the column-reduction CTA grid of this problem.
struct ReduceArgs {
  const void* X;
  int64_t R, C, ld;
  const int* shift;
  int sign;
  int* out;
  int vec;
  int rows_per_cta;
  int64_t gx;
};
constexpr int kBatchColRows = 256;  // rows per CTA of a batched column reduction (one atomic per column each)
constexpr int kBatchColSpan = 2048;  // columns per CTA of a column reduction

// Batched reductions over `count` problems of one element type.  args and
// start live in device memory: start[p] = first warp (row reductions: one
// row per warp) or first CTA (column reductions: args[p].gx spans x
// ceil(R / rows_per_cta) chunks) of problem p, start[count] the total.
cudaError_t launch_row_exp_batched(const ReduceArgs* args, const int64_t* start, int count, int64_t total, int dt,
                                   bool shift, int mode, int* status, cudaStream_t st);
cudaError_t launch_col_exp_batched(const ReduceArgs* args, const int64_t* start, int count, int64_t total, int dt,
                                   bool shift, int* status, cudaStream_t st);
cudaError_t launch_fill(int* p, int64_t n, int v, cudaStream_t st);
// out[p * ncb + q] = max |X| over block (p, q) of the nrb x ncb grid of
// ceil(R / nrb) x ceil(C / ncb) blocks (ncb <= 64); Inf/NaN skipped and
// flagged in *status.
cudaError_t launch_block_max(const void* X, int dt, int64_t R, int64_t C, int64_t ld, int nrb, int ncb, float* out,
                             int* status, cudaStream_t st);


// One operand of the fused multiply as the kernel sees it: a tile has
// "t" rows (the M side for A, the N side for B) and "k" columns.  The
// operand is "prepared": every leaf block (bt x bk, tile multiples) starts at
// element (tb*bt, kb*bk) of the tensor map's (t, k) grid, and everything
// outside the logical matrix inside a block is zero.  kcontig: k is the
// contiguous index of the tensor (TMA x = k, y = t); else t is (x = t, y = k).
struct TileOperand {
  const void* ptr;
  int64_t ld;
  int dtype;       // kF32 / kBF16
  int kcontig;
  int64_t bt, bk;  // prepared block extents (multiples of 128 and 64)
  int blk_t_shift; // term block packing: t block = (blk >> blk_t_shift) & 0xFFFF
  int blk_k_shift; //                      k block = (blk >> blk_k_shift) & 0xFFFF
};

struct EpilogueArgs {
  float* C;
  int64_t ldc;
  int64_t M, N;
  int64_t bm, bn;  // logical leaf block extents
  const int* eA;   // C scale 2^(eA_i + eB_j), nullable
  const int* eB;
  int vec_ok;
};

struct GemmArgs {
  alignas(64) CUtensorMap map_a;
  alignas(64) CUtensorMap map_b;
  TileOperand a, b;
  EpilogueArgs c;
  const LeafDesc* leaves;
  int64_t num_leaves;
  int* status;
  uint64_t timeout_ns;
};

// Prepare one operand: Y (R' x C', leading dimension ldy) = the blocked,
// zero-padded, power-of-two-scaled copy of X (R x C, ld): output row r'
// = rb * row_pad + r takes source row rb * row_blk + r when r < row_blk,
// columns likewise; entries outside the source are 0; each value is
// multiplied by 2^(rs re[row] + cs ce[col]) (exact).  Y is fp32, or bf16
// when X is bf16.
cudaError_t launch_prepare(const void* X, int dt, int64_t R, int64_t C, int64_t ld, int64_t row_blk,
                           int64_t row_pad, int64_t col_blk, int64_t col_pad, const int* re, int rs, const int* ce,
                           int cs, void* Y, int64_t Rp, int64_t Cp, int64_t ldy, cudaStream_t st);

// One side of the operand combination pass: for every leaf r of a plan,
// S_r = sum over the leaf's terms of coef * X(block), in FP32 in term
// order, each element of X scaled by 2^(rs re[row] + cs ce[col]) of its
// memory row / column, rounded to the leaf format.  X is a row-major memory
// matrix (rows x cols, ld) cut into blocks of b_rows x b_cols; each combined
// block keeps that orientation and is padded to p_rows x p_cols: plane p
// (0 = the rounded value, 1 = the bf16 remainder of the hi+lo split), leaf
// r, row i, column j at out[((p R + r) p_rows + i) p_cols + j].
struct CombineArgs {
  const void* src;
  int64_t ld;
  int dtype;            // kF32 / kBF16 / kF16
  int64_t rows, cols;   // memory extents of X
  int64_t b_rows, b_cols;
  int64_t n_rb, n_cb;   // number of row / column blocks
  int64_t p_rows, p_cols;  // multiples of 32 and 64
  int t_rows;           // memory rows follow the operand's t index (else its k index)
  const int* re;        // memory-row exponents (nullable), sign rs
  int rs;
  const int* ce;        // memory-column exponents (nullable), sign cs
  int cs;
  const LeafDesc* leaves;
  int64_t num_leaves;
  int side;             // 0: the leaves' A terms, 1: their B terms
  const int32_t* t_start;  // the side's compact term list (Plan::lists)
  const int32_t* t_blk;
  const float* t_coef;
  int64_t t_nnz;
  int blk_t_shift, blk_k_shift;
  void* out;            // 16-bit elements
  int fmt;              // FMM_LEAF_BF16 / FMM_LEAF_F16 / FMM_LEAF_BF16X3
  // Scaling between recursive steps (null: off): every element of a term of
  // leaf r is multiplied by 2^(between_sign d[r / leaves_per_node][k1]), k1
  // its k index inside its level-1 block: (kb mod kb_inner) * bk + k.
  const int* between_d;
  int between_sign;
  int64_t between_k1;       // k extent of a level-1 block (row length of d)
  int64_t leaves_per_node;  // leaves below one level-1 product
  int64_t kb_inner;         // leaf k blocks per level-1 k block
  int64_t bk;               // leaf block k extent
  // E4M3 leaves (fmt FMM_LEAF_E4M3B128): out holds bytes, K-major for both
  // sides ([leaf][t][k], p_rows = padded t, p_cols = padded k, multiples of
  // 128), and scale_out[(leaf * p_cols / 128 + kb) * p_rows + t] = 2^s of
  // each row's 128-block; with sf_atoms, scale_out holds the same blocks'
  // scales as UE8M0 bytes (s + 127) in the tensor core's block-scale
  // layout instead: per (leaf, kb, 128-row group g) a 512-byte atom whose
  // byte (t mod 32) * 16 + ((t mod 128) / 32) * 4 + j is row t's scale for
  // the 32-wide K sub-block j (the four equal here).
  float* scale_out;
  int sf_atoms;
};

// E4M3 combination pass (see CombineArgs::scale_out); a.p_rows / p_cols are
// the padded t / k extents whatever the source's layout.  Input tiles are
// staged in shared memory when they fit, else read per term (any number of
// input blocks).
cudaError_t launch_combine_e4m3(const CombineArgs& a, cudaStream_t st);

// Multiply kernel for E4M3 leaves: stored products only, both operands
// K-major bytes ([leaf][t][k], tensor maps with 128 x 128 byte boxes), one
// 128-wide K block per pipeline stage accumulated into a TMEM block
// accumulator and folded into FP32 running sums with 2^(sa + sb).
struct Fp8Args {
  alignas(64) CUtensorMap map_a;
  alignas(64) CUtensorMap map_b;
  const float* fa;  // [leaf][kb][tp_a] factors 2^sa (block_scaled: UE8M0 atoms, CombineArgs::sf_atoms)
  const float* fb;  // [leaf][kb][tp_b] factors 2^sb (likewise)
  float* mbuf;      // [leaf][tp_a][tp_b] fp32
  int64_t tp_a, tp_b, kp, num_leaves;
  int* status;
  uint64_t timeout_ns;
  int block_scaled;  // kind::mxf8f6f4.block_scale (scales applied by the tensor core), else the per-block fold
};
cudaError_t launch_fp8_gemm(const Fp8Args& a, cudaStream_t st);

// Node-exponent pass of the scaling between recursive steps: for each
// level-1 product r (the terms of `a` are the level-1 plan's), the FP32
// sequential sum S_r over the level-1 blocks (b_rows x b_cols, n_rb x n_cb
// of them), and out[r * k1 + k] = max over t of the frexp exponent of
// S_r[t, k] (atomicMax; out pre-filled with kZeroExp).  k runs along the
// memory columns when a.t_rows, else along the memory rows.
cudaError_t launch_node_exp(const CombineArgs& a, int* out, int64_t k1, cudaStream_t st);
// d[i] = floor((rexp[i] - cexp[i]) / 2), 0 where either has no nonzero entry.
cudaError_t launch_between_finalize(const int* cexp, const int* rexp, int* d, int64_t n, cudaStream_t st);

cudaError_t launch_combine(const CombineArgs& a, cudaStream_t st);
// Both operands' combination passes, in one launch when both take the
// unrolled small-block form, else as two launches (a0 first).
cudaError_t launch_combine_pair(const CombineArgs& a0, const CombineArgs& a1, cudaStream_t st);
// The same pair of passes streamed through bulk tensor copies (FP32 sources
// of at most 2 x 2 blocks; m0, m1: tensor maps over the sources' memory,
// 256 x 8 float boxes, no swizzle, zero fill); cudaErrorNotSupported when
// the operands do not qualify (nothing launched).
cudaError_t launch_combine_pair_stream(const CombineArgs& a0, const CUtensorMap& m0, const CombineArgs& a1,
                                       const CUtensorMap& m1, uint64_t timeout_ns, int* status, cudaStream_t st);

// Multiply kernel over combined operands (the pass schedule): each operand
// is the 16-bit output of the combination pass, K-major ([plane][R][tp][kp],
// k contiguous) or MN-major ([plane][R][kp][tp], t contiguous), read whole
// tiles at a time through the tensor maps (box 64 k x 128 / BN t for
// K-major, 64 t x 64 k for MN-major).
struct DirectArgs {
  alignas(64) CUtensorMap map_a;
  alignas(64) CUtensorMap map_b;
  // CTA-pair kernel, stored products: M_r as a 2-D fp32 tensor (R * tp_a
  // rows of tp_b), boxes of 32 x 32 with the 128-byte swizzle, for bulk
  // tensor stores of the epilogue's chunks (tma_store set)
  alignas(64) CUtensorMap map_m;
  int tma_store;
  EpilogueArgs c;
  const LeafDesc* leaves;
  int64_t num_leaves;
  int64_t tp_a, tp_b;  // padded t extent per leaf block (multiples of the tile)
  int64_t kp;          // padded k extent (multiple of 64)
  int a_mn, b_mn;      // operand layouts
  float* mbuf;         // null: fused epilogue into C; else store M_r, [leaf][tp_a][tp_b] fp32
  int accumulate;      // mbuf null: (leaf, tile) units add into C (zeroed) by atomic FP32 additions
  int* status;
  uint64_t timeout_ns;
  // Test of the timeout path (FMM_TEST_STALL set in the environment): the
  // epilogue first waits, bounded, on a barrier that nothing arrives at.
  int stall_test;
  // CTA-pair kernel: only the tile rows tm_begin .. tm_begin + tm_count - 1
  // (tm_count 0: all), so that a product can run as two launches
  int64_t tm_begin, tm_count;
};

// Output combination pass (third line of Eq. 4.4) over stored leaf products:
// for every C block k and element, C = sum over the leaves r in leaf order of
// w_kr 2^(eA_i + eB_j) M_r (the first term stored, the rest added), exactly
// as the fused epilogue would.  mbuf as DirectArgs::mbuf.
struct OutArgs {
  const float* mbuf;
  int64_t tp_a, tp_b;
  EpilogueArgs c;
  const LeafDesc* leaves;
  int64_t num_leaves;
  int64_t c_blocks;  // pm x pn C blocks (at most kMaxOutBlocks)
  int64_t pn;        // C blocks per block row
  const int32_t* c_start;  // the C-side compact term list (Plan::lists)
  const int32_t* c_blk;
  const float* c_coef;
  int64_t c_nnz;
  const int32_t* g_start;  // the C terms grouped by C block (Plan::gather_off), or NULL
  const int32_t* g_leaf;
  const float* g_coef;
  // register-accumulator pass: only leaf-block rows [r_begin, r_end) (r_end
  // 0: up to c.bm)
  int64_t r_begin, r_end;
};
constexpr int kMaxOutBlocks = 96;
cudaError_t launch_out_combine(const OutArgs& a, cudaStream_t st);
// The register-accumulator output pass (at most 16 C blocks) in CTAs of 256
// threads and at most 85 registers each, so that one fits on an SM beside
// a CTA of the CTA-pair multiply kernel and the two run together;
// cudaErrorNotSupported when the plan does not qualify.
cudaError_t launch_out_dense_slim(const OutArgs& a, cudaStream_t st);
// The output pass for plans with more than kMaxOutBlocks C blocks: each CTA
// forms one position tile of one C block from that block's term list.
cudaError_t launch_out_gather(const OutArgs& a, cudaStream_t st);

// Batched combination / output passes over `count` entries whose arguments
// live in device memory; start[p] is the first CTA of entry p (combination:
// (p_rows / tr) x (p_cols / 64) CTAs; output: ceil(bm / tr) x ceil(bn / 64)),
// start[count] = total.  One element type and leaf format per launch; tr
// (rows per CTA) from combine_batched_rows / out_batched_rows for the largest
// block count of the batch; smem the largest entry's shared memory.
int combine_batched_rows(int64_t max_blocks);
// Batched entries whose combination is one term of one block with one leaf
// (the classical product): a plain scaled conversion with wide tiles;
// start[p] is the first CTA of entry p (convert_batched_ctas CTAs each).
int64_t convert_batched_ctas(const CombineArgs& a);
cudaError_t launch_convert_batched(const CombineArgs* args, const int64_t* start, int count, int64_t total, int dt,
                                   int fmt, cudaStream_t st);
int out_batched_rows(int64_t max_c_blocks);
size_t combine_staged_smem(int64_t nb, int tr, int64_t nnz, int64_t leaves);
cudaError_t launch_combine_batched(const CombineArgs* args, const int64_t* start, int count, int64_t total, int dt,
                                   int fmt, int tr, size_t smem, cudaStream_t st);
cudaError_t launch_out_combine_batched(const OutArgs* args, const int64_t* start, int count, int64_t total, int tr,
                                       size_t smem, cudaStream_t st);

// bn: tile width along N (128 or 256).
cudaError_t launch_direct_gemm(const DirectArgs& args, int leaf_format, int bn, cudaStream_t st);
// The same work on CTA pairs (cluster of two, tcgen05 cta_group::2):
// 256 x 256 tiles, tp_a and tp_b multiples of 256; a K-major B operand's
// tensor map has 128-row boxes (each CTA loads half of B's tile).
cudaError_t launch_pair_gemm(const DirectArgs& args, int leaf_format, cudaStream_t st);
// The same over a batch: tab (device memory) holds `count` problems (tp_a,
// tp_b multiples of 256), unit_start their consecutive unit numbering;
// `layout` gives the status word, the wait limit and the operand layouts.
cudaError_t launch_pair_gemm_batched(const DirectArgs& layout, const DirectArgs* tab, const int64_t* unit_start,
                                     int count, int64_t total_units, int leaf_format, cudaStream_t st);

// The same kernel over a batch: tab (device memory) holds `count` problems,
// each with its tensor maps, leaves and stored-product buffer (mbuf set);
// unit_start (device) numbers their (leaf, tile) units consecutively.
// `layout` gives the status word, the wait limit and the operand layouts
// (a_mn, b_mn), which all problems share, as they share leaf format and bn.
cudaError_t launch_direct_gemm_batched(const DirectArgs& layout, const DirectArgs* tab, const int64_t* unit_start,
                                       int count, int64_t total_units, int leaf_format, int bn, cudaStream_t st);

// K extent of one pipeline stage of that kernel (the k extent of its
// operand boxes): 32 for the hi+lo split, else 64.
int direct_gemm_bk(int leaf_format);

// Launch the fused recursive-fast-multiply kernel for a flattened plan.
cudaError_t launch_fused_gemm(const GemmArgs& args, int leaf_format, cudaStream_t st);

// While kernel timing is enabled (fmm_kernel_timing), an object of this
// type brackets one kernel launch with CUDA events on its stream; kinds:
// "scale", "prepare", "combine", "multiply".
class KernelTimer {
 public:
  KernelTimer(const char* kind, cudaStream_t st);
  ~KernelTimer();
  KernelTimer(const KernelTimer&) = delete;
  KernelTimer& operator=(const KernelTimer&) = delete;

 private:
  const char* kind_;
  cudaStream_t st_;
  void* start_ = nullptr;
  void* stop_ = nullptr;
};

// Number of SMs of the current device (cached).
int device_sm_count();

}  // namespace fmm
