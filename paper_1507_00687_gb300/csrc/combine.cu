// Operand combination pass (the first two lines of Eq. 4.4, with the
// operand scaling of Algs. 1-3 applied on the way in):
//   S_r = sum_t u_t A'(blk_t),   A' = 2^(-eA) A 2^(d)    (and T_r from B')
// for every leaf r of a flattened plan, written once into the workspace in
// the leaf format so that the multiply kernel streams the tensor-core
// operands with bulk tensor copies and no further arithmetic.
//
// Arithmetic per element (the same as the load-stage producers of the fused
// kernel): acc = 0; acc = fma(coef_t, x_t, acc) over the terms in index
// order in FP32, x_t the exactly scaled input; then hi = rn(acc) in the
// leaf format and, for the hi+lo split, lo = rn_bf16(acc - hi).
//
// The pass works in the source's memory coordinates: the source is a
// row-major matrix whose rows are cut into blocks of b_rows and columns into
// blocks of b_cols, and each combined leaf block keeps that orientation, so
// both the reads and the writes run along the contiguous index.  One CTA
// covers a 32 x 64 position tile of every leaf block and walks all leaves,
// so the input block tiles it reads stay in L1 while the leaves re-read
// them; every output element (padding included) is written.  HBM-bound:
// each input element is read once from DRAM, each output element written
// once.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "../../include/fmm.h"
#include "device.cuh"
#include "gemm_common.cuh"
#include "kernels.h"

namespace fmm {
namespace {

constexpr int kTR = 32;   // rows per CTA tile
constexpr int kTC = 64;   // columns per CTA tile
constexpr int kThreads = 256;
constexpr int kRowsPerThread = kTR * kTC / (kThreads * 4);  // 2

template <int DT>
__device__ __forceinline__ float load_elem(const void* p, int64_t i) {
  if constexpr (DT == kF32) {
    return __ldg(reinterpret_cast<const float*>(p) + i);
  } else if constexpr (DT == kBF16) {
    return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p) + i) << 16);
  } else {
    return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p) + i)));
  }
}

// Four consecutive elements from a 16-byte (fp32) or 8-byte (16-bit)
// aligned address.
template <int DT>
__device__ __forceinline__ void load4(const void* p, int64_t i, float (&v)[4]) {
  if constexpr (DT == kF32) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(p) + i));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    const uint2 x = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const unsigned short*>(p) + i));
    if constexpr (DT == kBF16) {
      v[0] = __uint_as_float(x.x << 16); v[1] = __uint_as_float(x.x & 0xFFFF0000u);
      v[2] = __uint_as_float(x.y << 16); v[3] = __uint_as_float(x.y & 0xFFFF0000u);
    } else {
      v[0] = __half2float(__ushort_as_half((unsigned short)(x.x & 0xFFFFu)));
      v[1] = __half2float(__ushort_as_half((unsigned short)(x.x >> 16)));
      v[2] = __half2float(__ushort_as_half((unsigned short)(x.y & 0xFFFFu)));
      v[3] = __half2float(__ushort_as_half((unsigned short)(x.y >> 16)));
    }
  }
}

// Round 4 sums and store them (and the bf16 remainders for the split) as
// 8 bytes per plane.
template <int FMT>
__device__ __forceinline__ void store4(unsigned short* hi, unsigned short* lo, const float (&v)[4]) {
  uint32_t h[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if constexpr (FMT == FMM_LEAF_F16) {
      __half2 x = __floats2half2_rn(v[2 * j], v[2 * j + 1]);
      h[j] = *reinterpret_cast<uint32_t*>(&x);
    } else {
      __nv_bfloat162 x = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      h[j] = *reinterpret_cast<uint32_t*>(&x);
    }
  }
  *reinterpret_cast<uint2*>(hi) = make_uint2(h[0], h[1]);
  if constexpr (FMT == FMM_LEAF_BF16X3) {
    uint32_t l[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float r0 = v[2 * j] - __uint_as_float(h[j] << 16);
      const float r1 = v[2 * j + 1] - __uint_as_float(h[j] & 0xFFFF0000u);
      __nv_bfloat162 x = __floats2bfloat162_rn(r0, r1);
      l[j] = *reinterpret_cast<uint32_t*>(&x);
    }
    *reinterpret_cast<uint2*>(lo) = make_uint2(l[0], l[1]);
  }
}

// The scaled elements (lr, lc .. lc + 3) of one term's block tile (zero
// outside the source).
template <int DT>
__device__ __forceinline__ void load_term4(const CombineArgs& a, int32_t blk, int64_t lr, int64_t lc, bool vec_ok,
                                           float (&x)[4]) {
  const int64_t bt = (blk >> a.blk_t_shift) & 0xFFFF, bk = (blk >> a.blk_k_shift) & 0xFFFF;
  const int64_t rb = a.t_rows ? bt : bk, cb = a.t_rows ? bk : bt;
  // rows / columns of this block that exist in the source
  const int64_t nr = min(a.b_rows, a.rows - rb * a.b_rows), nc = min(a.b_cols, a.cols - cb * a.b_cols);
  const int64_t gr = rb * a.b_rows + lr, gc = cb * a.b_cols + lc;
  if (vec_ok && lr < nr && lc + 4 <= nc) {
    load4<DT>(a.src, gr * a.ld + gc, x);
    if (a.re || a.ce) {
      const int er = a.re ? a.rs * __ldg(a.re + gr) : 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = scale_pow2(x[j], er + (a.ce ? a.cs * __ldg(a.ce + gc + j) : 0));
    }
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x[j] = 0.f;
      if (lr < nr && lc + j < nc) {
        const float v = load_elem<DT>(a.src, gr * a.ld + gc + j);
        const int e = (a.re ? a.rs * __ldg(a.re + gr) : 0) + (a.ce ? a.cs * __ldg(a.ce + gc + j) : 0);
        x[j] = scale_pow2(v, e);
      }
    }
  }
}

// Unstaged form (plans with more input blocks than kMaxStaged): a CTA
// covers one kTR x 64 position tile for a contiguous range of leaves
// (blockIdx.z) and sums each leaf's terms from the source in term order,
// issuing the loads of kTermBatch terms together.
constexpr int kTermBatch = 4;

template <int DT, int FMT>
__global__ void __launch_bounds__(kThreads) combine_kernel(const CombineArgs a) {
  pdl_wait();
  pdl_trigger();
  const int64_t r0 = (int64_t)blockIdx.y * kTR, c0 = (int64_t)blockIdx.x * kTC;
  const int tid = threadIdx.x;
  const int tr = tid >> 4, tc = (tid & 15) * 4;  // rows tr, tr + 16; columns tc .. tc + 3
  const int64_t R = a.num_leaves;
  const int es = DT == kF32 ? 4 : 2;
  const bool vec_ok = ((uintptr_t)a.src % (4 * es) == 0) && (a.ld % 4 == 0) && (a.b_cols % 4 == 0);
  unsigned short* out = static_cast<unsigned short*>(a.out);
  const int64_t plane = R * a.p_rows * a.p_cols;
  const int64_t per = (R + gridDim.z - 1) / gridDim.z;
  const int64_t r_end = min(R, (int64_t)(blockIdx.z + 1) * per);
  // a tile wholly in the padding of every block only writes zeros
  const bool pad = r0 >= a.b_rows || c0 >= a.b_cols;
  for (int64_t r = (int64_t)blockIdx.z * per; r < r_end; ++r) {
    const int t1 = pad ? 0 : __ldg(a.t_start + r + 1);
    float acc[kRowsPerThread][4];
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int t = pad ? 0 : __ldg(a.t_start + r); t < t1; t += kTermBatch) {
      float x[kTermBatch][kRowsPerThread][4];
      float coef[kTermBatch];
#pragma unroll
      for (int u = 0; u < kTermBatch; ++u) {
        const bool live = t + u < t1;
        const int32_t blk = live ? __ldg(a.t_blk + t + u) : 0;
        coef[u] = live ? __ldg(a.t_coef + t + u) : 0.f;
#pragma unroll
        for (int i = 0; i < kRowsPerThread; ++i) {
          if (live) {
            load_term4<DT>(a, blk, r0 + tr + 16 * i, c0 + tc, vec_ok, x[u][i]);
          } else {
            x[u][i][0] = x[u][i][1] = x[u][i][2] = x[u][i][3] = 0.f;
          }
        }
      }
      // in term order
#pragma unroll
      for (int u = 0; u < kTermBatch; ++u)
        if (t + u < t1)
#pragma unroll
          for (int i = 0; i < kRowsPerThread; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(coef[u], x[u][i][j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i) {
      const int64_t off = (r * a.p_rows + r0 + tr + 16 * i) * a.p_cols + c0 + tc;
      store4<FMT>(out + off, out + off + plane, acc[i]);
    }
  }
}

// Staged form for plans with at most kMaxStaged input blocks: every input
// block's TR x 64 tile is loaded and scaled once into shared memory (in
// block order), the side's compact term list is copied there too, and each
// leaf's terms are summed from shared memory in term order -- the same
// arithmetic as above with each element scaled once instead of once per
// use.  TR * 16 threads, one row of 4 columns each.
constexpr int kMaxStaged = 64;

template <int DT, int FMT, int TR, int RPT, bool BETWEEN = false, int LS = 1>
__device__ __forceinline__ void combine_staged_body(const CombineArgs& a, int64_t bx, int64_t by, float4* tile4,
                                                    int r_begin, int r_end) {
  // RPT rows per thread: rows tr + (TR / RPT) q, q < RPT; 4 columns each.
  // LS groups of threads share the staged tiles: group ls stages blocks
  // ls, ls + LS, ... and forms leaves r_begin + ls, + LS, ... (LS > 1 gives
  // the small CTAs of plans with many blocks enough warps).
  constexpr int kP = TR * 16 / RPT;  // threads per group (one per position)
  constexpr int kT = kP * LS;
  const int64_t r0 = by * TR, c0 = bx * kTC;
  const int ls = (int)threadIdx.x / kP, pt = (int)threadIdx.x % kP;
  const int tr = pt >> 4, tq = pt & 15, tc = tq * 4;
  const int es = DT == kF32 ? 4 : 2;
  const bool vec_ok = ((uintptr_t)a.src % (4 * es) == 0) && (a.ld % 4 == 0) && (a.b_cols % 4 == 0) &&
                      (!a.ce || (uintptr_t)a.ce % 16 == 0);
  const int n_rb = (int)a.n_rb, n_cb = (int)a.n_cb;
  const int nb = n_rb * n_cb;
  const int R = (int)a.num_leaves;
  const int nnz = (int)a.t_nnz;
  // term list in shared memory: float4 offset of the term's block tile, coef
  int* toff = reinterpret_cast<int*>(tile4 + nb * TR * 16);
  float* tcoef = reinterpret_cast<float*>(toff + nnz);
  int* tstart = reinterpret_cast<int*>(tcoef + nnz);
  int* tkb = tstart + R + 1;  // k block of each term (between-steps scaling only)
  for (int i = threadIdx.x; i < nnz; i += kT) {
    const int32_t blk = __ldg(a.t_blk + i);
    const int bt = (blk >> a.blk_t_shift) & 0xFFFF, bk = (blk >> a.blk_k_shift) & 0xFFFF;
    toff[i] = (a.t_rows ? bt * n_cb + bk : bk * n_cb + bt) * TR * 16;
    tcoef[i] = __ldg(a.t_coef + i);
    if (BETWEEN) tkb[i] = bk;
  }
  for (int i = threadIdx.x; i <= R; i += kT) tstart[i] = __ldg(a.t_start + i);
  const int64_t lc = c0 + tc;
  // Blocks are staged kStageGroup at a time: the group's element and
  // exponent loads are all issued before any of them is scaled and stored.
  // Only the small CTAs of plans with more than 16 blocks (a few warps per
  // SM) need that many loads in flight per thread; for the rest the extra
  // registers cost more occupancy than they gain (measured: Strassen with
  // classical <1,2,1>, 8 blocks, 873 -> 813 TFLOP/s at 8192^3 with groups of
  // four; three levels, 32 blocks, 516 -> 538 with groups of eight).
  constexpr int kStageGroup = TR >= 8 ? 1 : 8;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int trq = tr + (TR / RPT) * q;
    const int64_t lr = r0 + trq;
    for (int b0 = ls; b0 < nb; b0 += kStageGroup * LS) {
      float x[kStageGroup][4];
      int ex[kStageGroup][4];
#pragma unroll
      for (int u = 0; u < kStageGroup; ++u) {
        const int b = b0 + u * LS;
        if (b >= nb) break;
        const int rb = b / n_cb, cb = b - (b / n_cb) * n_cb;
        const int64_t nr = min(a.b_rows, a.rows - rb * a.b_rows);
        const int64_t gr = rb * a.b_rows + lr;
        const bool row_in = lr < nr;
        const int er = (a.re && row_in) ? a.rs * __ldg(a.re + gr) : 0;
        const char* src_row = static_cast<const char*>(a.src) + gr * a.ld * es;
        const int64_t nc = min(a.b_cols, a.cols - cb * a.b_cols);
        const int64_t gc = cb * a.b_cols + lc;
        if (vec_ok && row_in && lc + 4 <= nc) {
          load4<DT>(src_row, gc, x[u]);
          int4 ec = make_int4(0, 0, 0, 0);
          if (a.ce) ec = __ldg(reinterpret_cast<const int4*>(a.ce + gc));
          ex[u][0] = er + a.cs * ec.x;
          ex[u][1] = er + a.cs * ec.y;
          ex[u][2] = er + a.cs * ec.z;
          ex[u][3] = er + a.cs * ec.w;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            x[u][j] = 0.f;
            ex[u][j] = 0;
            if (lr < nr && lc + j < nc) {
              x[u][j] = load_elem<DT>(src_row, gc + j);
              ex[u][j] = er + (a.ce ? a.cs * __ldg(a.ce + gc + j) : 0);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kStageGroup; ++u) {
        const int b = b0 + u * LS;
        if (b >= nb) break;
        float y[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] = (a.re || a.ce) ? scale_pow2(x[u][j], ex[u][j]) : x[u][j];
        tile4[(b * TR + trq) * 16 + tq] = make_float4(y[0], y[1], y[2], y[3]);
      }
    }
  }
  __syncthreads();
  unsigned short* out = static_cast<unsigned short*>(a.out);
  const int64_t plane = (int64_t)R * a.p_rows * a.p_cols;
  const int me = tr * 16 + tq;
  constexpr int kRowStep = (TR / RPT) * 16;  // float4 distance between a thread's rows
  const int64_t leaf_stride = a.p_rows * a.p_cols;
  unsigned short* orow = out + (r0 + tr) * a.p_cols + lc + (int64_t)(r_begin + ls) * leaf_stride;
  const int64_t qstride = (int64_t)(TR / RPT) * a.p_cols;
  for (int r = r_begin + ls; r < r_end; r += LS, orow += LS * leaf_stride) {
    int t = tstart[r];
    const int t1 = tstart[r + 1];
    float acc[RPT][4];
#pragma unroll
    for (int q = 0; q < RPT; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    const int* dnode = BETWEEN ? a.between_d + (r / a.leaves_per_node) * a.between_k1 : nullptr;
    for (; t < t1; ++t) {
      const float coef = tcoef[t];
      const int off = toff[t] + me;
      // between-steps scale of this term's elements (exact powers of two)
      float f[RPT][4];
      if constexpr (BETWEEN) {
        const int64_t kbase = (tkb[t] % a.kb_inner) * a.bk;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          if (a.t_rows) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int64_t k = kbase + lc + j;
              f[q][j] = k < a.between_k1 ? exp2i(a.between_sign * __ldg(dnode + k)) : 1.f;
            }
          } else {
            const int64_t k = kbase + r0 + tr + (TR / RPT) * q;
            const float g = k < a.between_k1 ? exp2i(a.between_sign * __ldg(dnode + k)) : 1.f;
            f[q][0] = f[q][1] = f[q][2] = f[q][3] = g;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        float4 v = tile4[off + q * kRowStep];
        if constexpr (BETWEEN) {
          v.x *= f[q][0]; v.y *= f[q][1]; v.z *= f[q][2]; v.w *= f[q][3];
        }
        acc[q][0] = fmaf(coef, v.x, acc[q][0]);
        acc[q][1] = fmaf(coef, v.y, acc[q][1]);
        acc[q][2] = fmaf(coef, v.z, acc[q][2]);
        acc[q][3] = fmaf(coef, v.w, acc[q][3]);
      }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) store4<FMT>(orow + q * qstride, orow + q * qstride + plane, acc[q]);
  }
}

// Groups of threads sharing a CTA's staged tiles (see combine_staged_body):
// more for the small tiles of plans with many blocks.
// For 9 to 16 blocks (8 rows per CTA) the groups raise the warps per SM
// that the shared-memory tiles allow; measured with one, two and four
// groups: Winograd two levels at n = 4096 266 / 293 / 298 TFLOP/s, the
// linear layer X[8192,4096] W[4096,4096] forward 524 / 579 / 594.  With 16
// rows per CTA (5 to 8 blocks) four groups made Strassen with classical
// <1,2,1> at 8192^3 slower (852 -> 727), so those CTAs keep one.
#ifndef FMM_STAGED_MID_GROUPS
#define FMM_STAGED_MID_GROUPS 4
#endif
template <int TR>
constexpr int staged_groups() { return TR <= 2 ? 8 : (TR <= 4 ? 4 : (TR <= 8 ? FMM_STAGED_MID_GROUPS : 1)); }

template <int DT, int FMT, int TR, int RPT, bool BETWEEN>
__global__ void __launch_bounds__(TR * 16 / RPT * staged_groups<TR>()) combine_staged_kernel(const CombineArgs a) {
  extern __shared__ float4 tile4[];  // [block][TR][16], then the term list
  pdl_wait();
  pdl_trigger();
  // blockIdx.z takes a contiguous range of the leaves (the input tiles are
  // staged once per range)
  const int R = (int)a.num_leaves;
  const int per = (R + (int)gridDim.z - 1) / (int)gridDim.z;
  const int r_begin = min(R, (int)blockIdx.z * per), r_end = min(R, r_begin + per);
  combine_staged_body<DT, FMT, TR, RPT, BETWEEN, staged_groups<TR>()>(a, blockIdx.x, blockIdx.y, tile4, r_begin,
                                                                      r_end);
}

// Batched form: tile b belongs to entry p with start[p] <= b < start[p + 1]
// and covers (local mod gx, local / gx), gx = p_cols / 64.  CTAs loop over
// tiles b = blockIdx.x, + gridDim.x, ... (the launch gives one per tile).
template <int DT, int FMT, int TR, int RPT>
__global__ void __launch_bounds__(TR * 16 / RPT) combine_staged_batched_kernel(const CombineArgs* args,
                                                                              const int64_t* start, int count,
                                                                              int64_t total) {
  extern __shared__ float4 tile4[];
  for (int64_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int p = warp_find_problem(start, count, b);
    const CombineArgs& a = args[p];
    const int64_t local = b - __ldg(start + p), gx = a.p_cols / kTC;
    combine_staged_body<DT, FMT, TR, RPT>(a, local % gx, local / gx, tile4, 0, (int)a.num_leaves);
    __syncthreads();  // the next tile reuses the shared memory
  }
}

// Batched conversion for entries whose combination is a single term of a
// single block with one leaf (the classical product): out = round(c x')
// with x' the scaled source element, zero in the padding -- the staged
// pass's arithmetic without its staging.  A CTA covers kConvRows rows x 512
// columns of one entry: each thread takes 8 consecutive columns of
// kConvRows / 4 rows, issuing all of its loads before any store, so that
// small entries still keep many bytes in flight.
constexpr int kConvRows = 16, kConvCols = 512, kConvIt = kConvRows / 4;

template <int DT, int FMT>
__global__ void __launch_bounds__(256) convert_batched_kernel(const CombineArgs* args, const int64_t* start, int count) {
  const int p = warp_find_problem(start, count, blockIdx.x);
  const CombineArgs& a = args[p];
  const int64_t local = blockIdx.x - __ldg(start + p);
  const int64_t gx = (a.p_cols + kConvCols - 1) / kConvCols;
  const int64_t r0 = (local / gx) * kConvRows + (threadIdx.x >> 6);
  const int64_t lc = (local % gx) * kConvCols + (threadIdx.x & 63) * 8;
  if (lc >= a.p_cols) return;
  const int es = DT == kF32 ? 4 : 2;
  const bool vec_ok = ((uintptr_t)a.src % (4 * es) == 0) && (a.ld % 4 == 0);
  const float coef = __ldg(a.t_coef);
  const int64_t nr = min(a.b_rows, a.rows), nc = min(a.b_cols, a.cols);
  const bool vec_cols = vec_ok && lc + 8 <= nc;
  float x[kConvIt][8];
#pragma unroll
  for (int it = 0; it < kConvIt; ++it) {
    const int64_t lr = r0 + 4 * it;
    const char* src_row = static_cast<const char*>(a.src) + lr * a.ld * es;
    if (lr < nr && vec_cols) {
      float v0[4], v1[4];
      load4<DT>(src_row, lc, v0);
      load4<DT>(src_row, lc + 4, v1);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[it][j] = v0[j];
        x[it][4 + j] = v1[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[it][j] = (lr < nr && lc + j < nc) ? load_elem<DT>(src_row, lc + j) : 0.f;
    }
  }
  int ec[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) ec[j] = (a.ce && lc + j < nc) ? a.cs * __ldg(a.ce + lc + j) : 0;
  const int64_t plane = a.p_rows * a.p_cols;
#pragma unroll
  for (int it = 0; it < kConvIt; ++it) {
    const int64_t lr = r0 + 4 * it;
    if (lr >= a.p_rows) break;
    const int er = (a.re && lr < nr) ? a.rs * __ldg(a.re + lr) : 0;
    unsigned short* out = static_cast<unsigned short*>(a.out) + lr * a.p_cols + lc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float acc[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fmaf(coef, scale_pow2(x[it][4 * h + j], er + ec[4 * h + j]), 0.f);
      store4<FMT>(out + 4 * h, out + 4 * h + plane, acc);
    }
  }
}

static int device_sms() {
  static int n[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (n[dev] == 0) {
    cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev);
    if (n[dev] <= 0) n[dev] = 132;
  }
  return n[dev];
}

// Leaf ranges per position tile so that the tiles holding data (not only
// padding) still give about `waves` CTAs per SM when they are few (deep
// plans have small leaf blocks and many leaves); at most one range per leaf.
static unsigned leaf_splits(const CombineArgs& a, int tile_rows, int64_t leaves, int waves) {
  const int64_t tiles = ((std::min(a.b_rows, a.p_rows) + tile_rows - 1) / tile_rows) *
                        ((std::min(a.b_cols, a.p_cols) + kTC - 1) / kTC);
  const int64_t want = ((int64_t)device_sms() * waves + tiles - 1) / tiles;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>({want, leaves, 65535}));
}

// Shared memory of the staged form: block tiles plus the term list (and
// the terms' k blocks, for the between-steps scaling).
inline size_t staged_smem(int nb, int tr, int64_t nnz, int64_t leaves) {
  return (size_t)nb * tr * 256 + (size_t)nnz * 12 + (size_t)(leaves + 1) * 4;
}
constexpr size_t kStagedSmemMax = 200 * 1024;

template <int DT, int FMT, int TR, int RPT, bool BETWEEN>
void launch_staged_tr_b(const CombineArgs& a, int nb, cudaStream_t st) {
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr_done[dev]) {
    cudaFuncSetAttribute(combine_staged_kernel<DT, FMT, TR, RPT, BETWEEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kStagedSmemMax);
    attr_done[dev] = true;
  }
  const dim3 grid((unsigned)(a.p_cols / kTC), (unsigned)(a.p_rows / TR));
  launch_pdl(combine_staged_kernel<DT, FMT, TR, RPT, BETWEEN>, dim3(grid.x, grid.y, leaf_splits(a, TR, a.num_leaves, 4)),
             dim3(TR * 16 / RPT * staged_groups<TR>()), staged_smem(nb, TR, a.t_nnz, a.num_leaves), st, a);
}

template <int DT, int FMT, int TR, int RPT = 1>
void launch_staged_tr(const CombineArgs& a, int nb, cudaStream_t st) {
  if (a.between_d) launch_staged_tr_b<DT, FMT, TR, RPT, true>(a, nb, st);
  else launch_staged_tr_b<DT, FMT, TR, RPT, false>(a, nb, st);
}

template <int DT, int FMT>
void launch_staged(const CombineArgs& a, int nb, cudaStream_t st) {
  // TR rows per CTA so that the staged tiles take at most 32 KB
  if (nb <= 4) launch_staged_tr<DT, FMT, 32, 2>(a, nb, st);
  else if (nb <= 8) launch_staged_tr<DT, FMT, 16>(a, nb, st);
  else if (nb <= 16) launch_staged_tr<DT, FMT, 8>(a, nb, st);
  else if (nb <= 32) launch_staged_tr<DT, FMT, 4>(a, nb, st);
  else launch_staged_tr<DT, FMT, 2>(a, nb, st);
}

// x 2^e with the exponent built directly when 2^e is a normal number.
__device__ __forceinline__ float scale_fast(float x, int e) {
  return ((unsigned)(e + 126) <= 253u) ? x * __int_as_float((e + 127) << 23) : scale_pow2(x, e);
}

// The staged combination for operands of at most 2 x 2 blocks (one level of
// a <2,2,2> rule, or the classical product), with the block loops unrolled
// and each column's scale exponents loaded once per thread: the same
// arithmetic as combine_staged_body (each element scaled once, each leaf's
// terms summed from shared memory in term order, then rounded and split).
// CTA: 32 rows x 64 columns of every block, 256 threads, rows tr and
// tr + 16 of 4 columns each.  The term list sits in shared memory as
// (float4 offset of the term's tile, coefficient) pairs.
template <int DT, int FMT, int NRB, int NCB>
__device__ __forceinline__ void combine_small_body(const CombineArgs& a, int64_t bx, int64_t by, float4* tile4,
                                                   int2* terms) {
  constexpr int TR = 32;
  const int64_t r0 = by * TR, c0 = bx * kTC;
  const int tr = threadIdx.x >> 4, tq = threadIdx.x & 15, tc = tq * 4;
  const int es = DT == kF32 ? 4 : 2;
  const bool vec_ok = ((uintptr_t)a.src % (4 * es) == 0) && (a.ld % 4 == 0) && (a.b_cols % 4 == 0) &&
                      (!a.ce || (uintptr_t)a.ce % 16 == 0);
  const int R = (int)a.num_leaves, nnz = (int)a.t_nnz;
  int* tstart = reinterpret_cast<int*>(terms + nnz);
  for (int i = threadIdx.x; i < nnz; i += 256) {
    const int32_t blk = __ldg(a.t_blk + i);
    const int bt = (blk >> a.blk_t_shift) & 0xFFFF, bk = (blk >> a.blk_k_shift) & 0xFFFF;
    terms[i] = make_int2((a.t_rows ? bt * NCB + bk : bk * NCB + bt) * TR * 16, __float_as_int(__ldg(a.t_coef + i)));
  }
  for (int i = threadIdx.x; i <= R; i += 256) tstart[i] = __ldg(a.t_start + i);
  const int64_t lc = c0 + tc;
  // column exponents of this thread's 4 columns in each block column
  int ec[NCB][4];
  int64_t ncols[NCB];
#pragma unroll
  for (int cb = 0; cb < NCB; ++cb) {
    ncols[cb] = min(a.b_cols, a.cols - cb * a.b_cols);
    const int64_t gc = cb * a.b_cols + lc;
#pragma unroll
    for (int j = 0; j < 4; ++j) ec[cb][j] = (a.ce && lc + j < ncols[cb]) ? a.cs * __ldg(a.ce + gc + j) : 0;
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int trq = tr + 16 * q;
    const int64_t lr = r0 + trq;
#pragma unroll
    for (int rb = 0; rb < NRB; ++rb) {
      const int64_t nr = min(a.b_rows, a.rows - rb * a.b_rows);
      const bool row_in = lr < nr;
      const int64_t gr = rb * a.b_rows + lr;
      const int er = (a.re && row_in) ? a.rs * __ldg(a.re + gr) : 0;
      const char* src_row = static_cast<const char*>(a.src) + gr * a.ld * es;
#pragma unroll
      for (int cb = 0; cb < NCB; ++cb) {
        const int64_t gc = cb * a.b_cols + lc;
        float x[4];
        if (vec_ok && row_in && lc + 4 <= ncols[cb]) {
          load4<DT>(src_row, gc, x);
#pragma unroll
          for (int j = 0; j < 4; ++j) x[j] = scale_fast(x[j], er + ec[cb][j]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            x[j] = (row_in && lc + j < ncols[cb]) ? scale_pow2(load_elem<DT>(src_row, gc + j), er + ec[cb][j]) : 0.f;
        }
        tile4[((rb * NCB + cb) * TR + trq) * 16 + tq] = make_float4(x[0], x[1], x[2], x[3]);
      }
    }
  }
  __syncthreads();
  unsigned short* out = static_cast<unsigned short*>(a.out);
  const int64_t leaf_stride = a.p_rows * a.p_cols;
  const int64_t plane = (int64_t)R * leaf_stride;
  const int me = tr * 16 + tq;
  unsigned short* orow = out + (r0 + tr) * a.p_cols + lc;
  const int64_t qstride = (int64_t)16 * a.p_cols;
  int t = 0;
  for (int r = 0; r < R; ++r, orow += leaf_stride) {
    const int t1 = tstart[r + 1];
    float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
    for (; t < t1; ++t) {
      const int2 term = terms[t];
      const float coef = __int_as_float(term.y);
      const float4 v0 = tile4[term.x + me];
      const float4 v1 = tile4[term.x + me + 256];
      acc0[0] = fmaf(coef, v0.x, acc0[0]);
      acc0[1] = fmaf(coef, v0.y, acc0[1]);
      acc0[2] = fmaf(coef, v0.z, acc0[2]);
      acc0[3] = fmaf(coef, v0.w, acc0[3]);
      acc1[0] = fmaf(coef, v1.x, acc1[0]);
      acc1[1] = fmaf(coef, v1.y, acc1[1]);
      acc1[2] = fmaf(coef, v1.z, acc1[2]);
      acc1[3] = fmaf(coef, v1.w, acc1[3]);
    }
    store4<FMT>(orow, orow + plane, acc0);
    store4<FMT>(orow + qstride, orow + qstride + plane, acc1);
  }
}

template <int DT, int FMT, int NRB, int NCB>
__global__ void __launch_bounds__(256) combine_small_kernel(const CombineArgs a) {
  __shared__ float4 tile4[NRB * NCB * 32 * 16];
  extern __shared__ int2 terms[];  // [nnz] (offset, coef bits), then tstart[R + 1]
  pdl_wait();
  pdl_trigger();
  combine_small_body<DT, FMT, NRB, NCB>(a, blockIdx.x, blockIdx.y, tile4, terms);
}

// Both operands' combination in one launch (the two passes are independent):
// CTAs [0, split) take a0's tiles, the rest a1's (linear tile indices, gx0 /
// gx1 tiles per tile row).
template <int DT, int FMT, int NRB, int NCB>
__global__ void __launch_bounds__(256) combine_small_pair_kernel(const CombineArgs a0, const CombineArgs a1,
                                                                 unsigned split) {
  __shared__ float4 tile4[NRB * NCB * 32 * 16];
  extern __shared__ int2 terms[];
  pdl_wait();
  pdl_trigger();
  if (blockIdx.x < split) {
    const int64_t gx = a0.p_cols / kTC;
    combine_small_body<DT, FMT, NRB, NCB>(a0, blockIdx.x % gx, blockIdx.x / gx, tile4, terms);
  } else {
    const int64_t gx = a1.p_cols / kTC, b = blockIdx.x - split;
    combine_small_body<DT, FMT, NRB, NCB>(a1, b % gx, b / gx, tile4, terms);
  }
}

template <int DT, int FMT>
void launch_small(const CombineArgs& a, cudaStream_t st) {
  const dim3 grid((unsigned)(a.p_cols / kTC), (unsigned)(a.p_rows / 32));
  const size_t smem = (size_t)a.t_nnz * 8 + (size_t)(a.num_leaves + 1) * 4;
  if (a.n_rb == 2 && a.n_cb == 2) launch_pdl(combine_small_kernel<DT, FMT, 2, 2>, grid, dim3(256), smem, st, a);
  else if (a.n_rb == 2) launch_pdl(combine_small_kernel<DT, FMT, 2, 1>, grid, dim3(256), smem, st, a);
  else if (a.n_cb == 2) launch_pdl(combine_small_kernel<DT, FMT, 1, 2>, grid, dim3(256), smem, st, a);
  else launch_pdl(combine_small_kernel<DT, FMT, 1, 1>, grid, dim3(256), smem, st, a);
}

// The operand combination for which the unrolled form applies (see
// launch_fmt): at most 2 x 2 blocks, no between-steps scale, a grid that
// fills the GPU, a small term list.
bool small_ok(const CombineArgs& a, int sms) {
  return a.n_rb <= 2 && a.n_cb <= 2 && !a.between_d && a.p_rows % 32 == 0 && a.p_cols % kTC == 0 &&
         (a.p_cols / kTC) * (a.p_rows / 32) >= 2 * (int64_t)sms && a.t_nnz * 8 + (a.num_leaves + 1) * 4 <= 16384;
}

template <int DT, int FMT>
void launch_small_pair(const CombineArgs& a0, const CombineArgs& a1, cudaStream_t st) {
  const int64_t t0 = (a0.p_cols / kTC) * (a0.p_rows / 32), t1 = (a1.p_cols / kTC) * (a1.p_rows / 32);
  const size_t smem = std::max((size_t)a0.t_nnz * 8 + (size_t)(a0.num_leaves + 1) * 4,
                               (size_t)a1.t_nnz * 8 + (size_t)(a1.num_leaves + 1) * 4);
  const dim3 grid((unsigned)(t0 + t1));
  if (a0.n_rb == 2 && a0.n_cb == 2)
    launch_pdl(combine_small_pair_kernel<DT, FMT, 2, 2>, grid, dim3(256), smem, st, a0, a1, (unsigned)t0);
  else if (a0.n_rb == 2)
    launch_pdl(combine_small_pair_kernel<DT, FMT, 2, 1>, grid, dim3(256), smem, st, a0, a1, (unsigned)t0);
  else if (a0.n_cb == 2)
    launch_pdl(combine_small_pair_kernel<DT, FMT, 1, 2>, grid, dim3(256), smem, st, a0, a1, (unsigned)t0);
  else
    launch_pdl(combine_small_pair_kernel<DT, FMT, 1, 1>, grid, dim3(256), smem, st, a0, a1, (unsigned)t0);
}

template <int DT, int FMT>
void launch_fmt(const CombineArgs& a, dim3 grid, cudaStream_t st) {
  const int64_t nb = a.n_rb * a.n_cb;
  const int tr = nb <= 4 ? 32 : nb <= 8 ? 16 : nb <= 16 ? 8 : nb <= 32 ? 4 : 2;
  // few leaves on a grid that already fills the GPU: the unrolled form
  if (small_ok(a, device_sms()))
    launch_small<DT, FMT>(a, st);
  else if (nb <= kMaxStaged && staged_smem((int)nb, tr, a.t_nnz, a.num_leaves) <= kStagedSmemMax)
    launch_staged<DT, FMT>(a, (int)nb, st);
  else if (!a.between_d)
    launch_pdl(combine_kernel<DT, FMT>, dim3(grid.x, grid.y, leaf_splits(a, kTR, a.num_leaves, 8)), dim3(kThreads), 0,
               st, a);
}

template <int DT>
cudaError_t launch_dt(const CombineArgs& a, dim3 grid, cudaStream_t st) {
  KernelTimer timer("combine", st);
  switch (a.fmt) {
    case FMM_LEAF_BF16: launch_fmt<DT, FMM_LEAF_BF16>(a, grid, st); break;
    case FMM_LEAF_F16: launch_fmt<DT, FMM_LEAF_F16>(a, grid, st); break;
    default: launch_fmt<DT, FMM_LEAF_BF16X3>(a, grid, st); break;
  }
  return cudaGetLastError();
}

// Output combination pass over stored leaf products M_r: one CTA covers a
// TR x 64 position tile of every C block and walks the leaves in order,
// keeping one fp32 accumulator per (C block, position) in shared memory
// (each thread only ever touches its own positions): acc = w M for the
// first leaf touching the block, else acc + w M.  The unscale of Algs. 1-3,
// C = D_A C' D_B, is applied once per element when C is written (the fused
// epilogue's per-term scaling gives the same value, since powers of two
// commute exactly with the sums while no value under- or overflows).  The
// C-side term list sits in shared memory with each term's accumulator
// offset; the M_r loads of a batch of leaves are issued together: four for
// CTAs of 256 or more threads, more for the small CTAs of plans with many C
// blocks (few threads per SM), so that each SM keeps enough loads in flight.
template <int TR>
constexpr int out_batch() { return TR >= 16 ? 4 : (TR >= 8 ? 8 : 16); }

template <int TR>
__device__ __forceinline__ void out_combine_body(const OutArgs& a, int64_t bx, int64_t by, float4* acc4) {
  const EpilogueArgs& c = a.c;
  const int tr = threadIdx.x >> 4, tq = threadIdx.x & 15;
  const int64_t lr = by * TR + tr, lc = bx * kTC + tq * 4;
  const int pn = (int)a.pn;
  const int R = (int)a.num_leaves;
  const int nnz = (int)a.c_nnz;
  int* cw = reinterpret_cast<int*>(acc4 + a.c_blocks * TR * 16);  // accumulator offset | first bit
  float* ccoef = reinterpret_cast<float*>(cw + nnz);
  int* cstart = reinterpret_cast<int*>(ccoef + nnz);
  for (int i = threadIdx.x; i < nnz; i += TR * 16) {
    const int32_t word = __ldg(a.c_blk + i);
    const int bi = (word >> 16) & 0x7FFF, bj = word & 0xFFFF;
    cw[i] = ((bi * pn + bj) * TR * 16) | (word & kFirstBit);
    ccoef[i] = __ldg(a.c_coef + i);
  }
  for (int i = threadIdx.x; i <= R; i += TR * 16) cstart[i] = __ldg(a.c_start + i);
  __syncthreads();
  const int me = tr * 16 + tq;
  const float* mcol = a.mbuf + lr * a.tp_b + lc;
  const int64_t leaf_stride = a.tp_a * a.tp_b;
  int t = 0;
  constexpr int kOutBatch = out_batch<TR>();
  for (int r0 = 0; r0 < R; r0 += kOutBatch) {
    float4 m[kOutBatch];
#pragma unroll
    for (int u = 0; u < kOutBatch; ++u)
      if (r0 + u < R) m[u] = __ldg(reinterpret_cast<const float4*>(mcol + (int64_t)(r0 + u) * leaf_stride));
#pragma unroll
    for (int u = 0; u < kOutBatch; ++u) {
      if (r0 + u >= R) break;
      const int t1 = cstart[r0 + u + 1];
      for (; t < t1; ++t) {
        const int w = cw[t];
        const float coef = ccoef[t];
        float4& acc = acc4[(w & 0x7FFFFFFF) + me];
        const float4 x = make_float4(coef * m[u].x, coef * m[u].y, coef * m[u].z, coef * m[u].w);
        if (w < 0) {
          acc = x;
        } else {
          acc.x += x.x; acc.y += x.y; acc.z += x.z; acc.w += x.w;
        }
      }
    }
  }
  for (int k = 0; k < (int)a.c_blocks && lr < c.bm; ++k) {
    const int bi = k / pn, bj = k % pn;
    const int64_t gi = bi * c.bm + lr, gj = bj * c.bn + lc;
    if (gi >= c.M) continue;
    const float4 v = acc4[k * TR * 16 + me];
    float vv[4] = {v.x, v.y, v.z, v.w};
    if (c.eA) {
      const float fa = exp2i(__ldg(c.eA + gi));
#pragma unroll
      for (int j = 0; j < 4; ++j) vv[j] *= fa;
    }
    if (c.eB) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (gj + j < c.N) vv[j] *= exp2i(__ldg(c.eB + gj + j));
    }
    float* dst = c.C + gi * c.ldc + gj;
    if (c.vec_ok && lc + 4 <= c.bn && gj + 4 <= c.N) {
      *reinterpret_cast<float4*>(dst) = make_float4(vv[0], vv[1], vv[2], vv[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (lc + j < c.bn && gj + j < c.N) dst[j] = vv[j];
    }
  }
}

template <int TR>
__global__ void __launch_bounds__(TR * 16) out_combine_kernel(const OutArgs a) {
  extern __shared__ float4 acc4[];  // [c_blocks][TR][16], then the term list
  pdl_wait();
  pdl_trigger();
  out_combine_body<TR>(a, blockIdx.x, blockIdx.y, acc4);
}

// Output pass with the accumulators in registers, for plans with at most
// NB C blocks: the leaves' W coefficients are laid out densely in shared
// memory (sW[r][k], zero where leaf r does not add into block k).  A CTA
// covers TR rows x TC columns of positions; each thread owns 4 consecutive
// entries of one position row in every C block
// and walks the leaves in order, adding w * M_r with one fused multiply-add
// per nonzero coefficient (w * M_r is exact for the power-of-two
// coefficients of the printed rules, so the sums equal those of the
// shared-memory pass).  The C sums are unscaled once and stored.
constexpr int kDenseBatch = 4;  // leaves whose loads are in flight together

template <int NB, int TR, int TC, int MINB = 1>
__global__ void __launch_bounds__(TR * TC / 4, MINB) out_dense_kernel(const OutArgs a) {
  extern __shared__ float sW[];  // [num_leaves][NB]
  pdl_wait();
  pdl_trigger();
  const EpilogueArgs& c = a.c;
  const int R = (int)a.num_leaves;
  const int pn = (int)a.pn;
  for (int i = threadIdx.x; i < R * NB; i += TR * TC / 4) sW[i] = 0.f;
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += TR * TC / 4) {
    for (int t = __ldg(a.c_start + r); t < __ldg(a.c_start + r + 1); ++t) {
      const int32_t word = __ldg(a.c_blk + t);
      const int bi = (word >> 16) & 0x7FFF, bj = word & 0xFFFF;
      sW[r * NB + bi * pn + bj] = __ldg(a.c_coef + t);
    }
  }
  __syncthreads();
  const int tr = threadIdx.x / (TC / 4), tq = threadIdx.x % (TC / 4);
  const int64_t lr = a.r_begin + (int64_t)blockIdx.y * TR + tr, lc = (int64_t)blockIdx.x * TC + tq * 4;
  if (lr >= (a.r_end ? min(a.r_end, c.bm) : c.bm) || lc >= c.bn) return;
  const float* mpos = a.mbuf + lr * a.tp_b + lc;
  const int64_t leaf_stride = a.tp_a * a.tp_b;
  float4 acc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) acc[b] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int r0 = 0; r0 < R; r0 += kDenseBatch) {
    float4 m[kDenseBatch];
#pragma unroll
    for (int u = 0; u < kDenseBatch; ++u)
      if (r0 + u < R) m[u] = __ldg(reinterpret_cast<const float4*>(mpos + (int64_t)(r0 + u) * leaf_stride));
#pragma unroll
    for (int u = 0; u < kDenseBatch; ++u) {
      if (r0 + u >= R) break;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const float w = sW[(r0 + u) * NB + b];
        if (w != 0.f) {
          acc[b].x = fmaf(w, m[u].x, acc[b].x);
          acc[b].y = fmaf(w, m[u].y, acc[b].y);
          acc[b].z = fmaf(w, m[u].z, acc[b].z);
          acc[b].w = fmaf(w, m[u].w, acc[b].w);
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (b >= (int)a.c_blocks) break;
    const int bi = b / pn, bj = b % pn;
    const int64_t gi = bi * c.bm + lr, gj = bj * c.bn + lc;
    if (gi >= c.M) continue;
    float vv[4] = {acc[b].x, acc[b].y, acc[b].z, acc[b].w};
    if (c.eA) {
      const float fa = exp2i(__ldg(c.eA + gi));
#pragma unroll
      for (int j = 0; j < 4; ++j) vv[j] *= fa;
    }
    if (c.eB) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (gj + j < c.N) vv[j] *= exp2i(__ldg(c.eB + gj + j));
    }
    float* dst = c.C + gi * c.ldc + gj;
    if (c.vec_ok && lc + 4 <= c.bn && gj + 4 <= c.N) {
      *reinterpret_cast<float4*>(dst) = make_float4(vv[0], vv[1], vv[2], vv[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (lc + j < c.bn && gj + j < c.N) dst[j] = vv[j];
    }
  }
}

// Output pass by C block (Eq. 3.2 read per output block): CTA (x, y)
// covers position tile x (kOutGatherRows x 64 entries of the leaf block) of
// C blocks y, y + gridDim.y, ...; each thread forms 4 consecutive entries as
// the sum over the block's terms, in leaf order, of w * M_r (the first term
// assigned, as the stored-products pass does), then unscales once and
// stores.  Every M_r is read once per C block it adds into.
constexpr int kOutGatherRows = 16;

__global__ void __launch_bounds__(kOutGatherRows * 16) out_gather_kernel(const OutArgs a) {
  pdl_wait();
  pdl_trigger();
  const EpilogueArgs& c = a.c;
  const int64_t gx = (c.bn + kTC - 1) / kTC;
  const int64_t bx = blockIdx.x % gx, by = blockIdx.x / gx;
  const int tr = threadIdx.x >> 4, tq = threadIdx.x & 15;
  const int64_t lr = by * kOutGatherRows + tr, lc = bx * kTC + tq * 4;
  if (lr >= c.bm || lc >= c.bn) return;
  const int64_t leaf_stride = a.tp_a * a.tp_b;
  const float* mpos = a.mbuf + lr * a.tp_b + lc;
  const int pn = (int)a.pn;
  for (int64_t k = blockIdx.y; k < a.c_blocks; k += gridDim.y) {
    const int t0 = __ldg(a.g_start + k), t1 = __ldg(a.g_start + k + 1);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int t = t0;
    for (; t + 4 <= t1; t += 4) {
      float4 m[4];
      float w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        w[u] = __ldg(a.g_coef + t + u);
        m[u] = __ldg(reinterpret_cast<const float4*>(mpos + (int64_t)__ldg(a.g_leaf + t + u) * leaf_stride));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 x = make_float4(w[u] * m[u].x, w[u] * m[u].y, w[u] * m[u].z, w[u] * m[u].w);
        if (t + u == t0) {
          acc = x;
        } else {
          acc.x += x.x; acc.y += x.y; acc.z += x.z; acc.w += x.w;
        }
      }
    }
    for (; t < t1; ++t) {
      const float w = __ldg(a.g_coef + t);
      const float4 m = __ldg(reinterpret_cast<const float4*>(mpos + (int64_t)__ldg(a.g_leaf + t) * leaf_stride));
      const float4 x = make_float4(w * m.x, w * m.y, w * m.z, w * m.w);
      if (t == t0) {
        acc = x;
      } else {
        acc.x += x.x; acc.y += x.y; acc.z += x.z; acc.w += x.w;
      }
    }
    const int bi = (int)(k / pn), bj = (int)(k % pn);
    const int64_t gi = bi * c.bm + lr, gj = bj * c.bn + lc;
    if (gi >= c.M) continue;
    float vv[4] = {acc.x, acc.y, acc.z, acc.w};
    if (c.eA) {
      const float fa = exp2i(__ldg(c.eA + gi));
#pragma unroll
      for (int j = 0; j < 4; ++j) vv[j] *= fa;
    }
    if (c.eB) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (gj + j < c.N) vv[j] *= exp2i(__ldg(c.eB + gj + j));
    }
    float* dst = c.C + gi * c.ldc + gj;
    if (c.vec_ok && lc + 4 <= c.bn && gj + 4 <= c.N) {
      *reinterpret_cast<float4*>(dst) = make_float4(vv[0], vv[1], vv[2], vv[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (lc + j < c.bn && gj + j < c.N) dst[j] = vv[j];
    }
  }
}

// Batched form: CTA b belongs to problem p with start[p] <= b < start[p + 1]
// and covers position tile (local mod gx, local / gx), gx = ceil(bn / 64).
template <int TR>
__global__ void __launch_bounds__(TR * 16) out_combine_batched_kernel(const OutArgs* args, const int64_t* start,
                                                                      int count, int64_t total) {
  extern __shared__ float4 acc4[];
  for (int64_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int p = warp_find_problem(start, count, b);
    const OutArgs& a = args[p];
    const int64_t local = b - __ldg(start + p), gx = (a.c.bn + kTC - 1) / kTC;
    out_combine_body<TR>(a, local % gx, local / gx, acc4);
    __syncthreads();  // the next tile reuses the shared memory
  }
}

// Node-exponent pass (scaling between recursive steps): one CTA covers a
// 16 x 64 position tile of the level-1 blocks, stages the (scaled) input
// block tiles as the combination pass does, forms each level-1 product's
// FP32 sum in term order and reduces the frexp exponents of the sums over t
// (over the tile's rows when t runs along memory rows, else over its
// columns) into out[r * k1 + k] with atomicMax.
constexpr int kNodeTR = 16;

template <int DT>
__global__ void __launch_bounds__(kNodeTR * 16) node_exp_kernel(const CombineArgs a, int* out, int64_t k1) {
  extern __shared__ float4 tile4[];  // [block][kNodeTR][16], then colmax [R][64] ints
  const int64_t r0 = (int64_t)blockIdx.y * kNodeTR, c0 = (int64_t)blockIdx.x * kTC;
  const int tr = threadIdx.x >> 4, tq = threadIdx.x & 15, tc = tq * 4;
  const int es = DT == kF32 ? 4 : 2;
  const bool vec_ok = ((uintptr_t)a.src % (4 * es) == 0) && (a.ld % 4 == 0) && (a.b_cols % 4 == 0) &&
                      (!a.ce || (uintptr_t)a.ce % 16 == 0);
  const int n_rb = (int)a.n_rb, n_cb = (int)a.n_cb, nb = n_rb * n_cb;
  const int R = (int)a.num_leaves;
  int* colmax = reinterpret_cast<int*>(tile4 + nb * kNodeTR * 16);
  for (int i = threadIdx.x; i < R * kTC; i += kNodeTR * 16) colmax[i] = kZeroExp;
  const int64_t lr = r0 + tr, lc = c0 + tc;
  for (int rb = 0; rb < n_rb; ++rb) {
    const int64_t nr = min(a.b_rows, a.rows - rb * a.b_rows);
    const int64_t gr = rb * a.b_rows + lr;
    const bool row_in = r0 + kNodeTR <= nr;
    const int er = (a.re && lr < nr) ? a.rs * __ldg(a.re + gr) : 0;
    const char* src_row = static_cast<const char*>(a.src) + gr * a.ld * es;
    for (int cb = 0; cb < n_cb; ++cb) {
      const int64_t nc = min(a.b_cols, a.cols - cb * a.b_cols);
      const int64_t gc = cb * a.b_cols + lc;
      float x[4];
      if (vec_ok && row_in && c0 + kTC <= nc) {
        load4<DT>(src_row, gc, x);
        if (a.re || a.ce) {
          int4 ec = make_int4(0, 0, 0, 0);
          if (a.ce) ec = __ldg(reinterpret_cast<const int4*>(a.ce + gc));
          x[0] = scale_pow2(x[0], er + a.cs * ec.x);
          x[1] = scale_pow2(x[1], er + a.cs * ec.y);
          x[2] = scale_pow2(x[2], er + a.cs * ec.z);
          x[3] = scale_pow2(x[3], er + a.cs * ec.w);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          x[j] = 0.f;
          if (lr < nr && lc + j < nc) {
            const float v = load_elem<DT>(src_row, gc + j);
            x[j] = scale_pow2(v, er + (a.ce ? a.cs * __ldg(a.ce + gc + j) : 0));
          }
        }
      }
      tile4[((rb * n_cb + cb) * kNodeTR + tr) * 16 + tq] = make_float4(x[0], x[1], x[2], x[3]);
    }
  }
  __syncthreads();
  const int me = tr * 16 + tq;
  bool nf = false;
  for (int r = 0; r < R; ++r) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int t1 = __ldg(a.t_start + r + 1);
    for (int t = __ldg(a.t_start + r); t < t1; ++t) {
      const int32_t blk = __ldg(a.t_blk + t);
      const int bt = (blk >> a.blk_t_shift) & 0xFFFF, bk = (blk >> a.blk_k_shift) & 0xFFFF;
      const int b = a.t_rows ? bt * n_cb + bk : bk * n_cb + bt;
      const float coef = __ldg(a.t_coef + t);
      const float4 v = tile4[b * kNodeTR * 16 + me];
      acc[0] = fmaf(coef, v.x, acc[0]);
      acc[1] = fmaf(coef, v.y, acc[1]);
      acc[2] = fmaf(coef, v.z, acc[2]);
      acc[3] = fmaf(coef, v.w, acc[3]);
    }
    int e[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) e[j] = fexp_f32(__float_as_uint(fabsf(acc[j])), &nf);
    if (a.t_rows) {
      // k along memory columns: maximum over the tile's rows
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (e[j] > kZeroExp) atomicMax(&colmax[r * kTC + tc + j], e[j]);
    } else {
      // k along memory rows: maximum over the tile's columns (16 threads)
      int m = max(max(e[0], e[1]), max(e[2], e[3]));
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (tq == 0 && m > kZeroExp && lr < k1) atomicMax(out + (int64_t)r * k1 + lr, m);
    }
  }
  if (a.t_rows) {
    __syncthreads();
    for (int i = threadIdx.x; i < R * kTC; i += kNodeTR * 16) {
      const int r = i / kTC, c = i % kTC;
      if (colmax[i] > kZeroExp && c0 + c < k1) atomicMax(out + (int64_t)r * k1 + c0 + c, colmax[i]);
    }
  }
}

__global__ void between_finalize_kernel(const int* cexp, const int* rexp, int* d, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = cexp[i], r = rexp[i];
  d[i] = (c <= kZeroExp / 2 || r <= kZeroExp / 2) ? 0 : ((r - c) >> 1);  // arithmetic shift = floor
}

}  // namespace

// CTAs of one entry of the conversion above.
int64_t convert_batched_ctas(const CombineArgs& a) {
  return ((a.p_rows + kConvRows - 1) / kConvRows) * ((a.p_cols + kConvCols - 1) / kConvCols);
}

cudaError_t launch_convert_batched(const CombineArgs* args, const int64_t* start, int count, int64_t total, int dt,
                                   int fmt, cudaStream_t st) {
  if (total == 0 || count == 0) return cudaSuccess;
  if (total > 0x7FFFFFFF) return cudaErrorInvalidValue;
  KernelTimer timer("combine", st);
#define FMM_CV(DT)                                                                                              \
  switch (fmt) {                                                                                                \
    case FMM_LEAF_BF16: convert_batched_kernel<DT, FMM_LEAF_BF16><<<(unsigned)total, 256, 0, st>>>(args, start, count); break; \
    case FMM_LEAF_F16: convert_batched_kernel<DT, FMM_LEAF_F16><<<(unsigned)total, 256, 0, st>>>(args, start, count); break;   \
    default: convert_batched_kernel<DT, FMM_LEAF_BF16X3><<<(unsigned)total, 256, 0, st>>>(args, start, count); break;         \
  }
  switch (dt) {
    case kF32: FMM_CV(kF32) break;
    case kBF16: FMM_CV(kBF16) break;
    default: FMM_CV(kF16) break;
  }
#undef FMM_CV
  return cudaGetLastError();
}


// E4M3 combination pass: one CTA covers TT t x 128 k (one scale block) of
// every leaf block (TT = 16, or 4 when the input blocks are too many to
// stage sixteen rows of each); the input block tiles are staged as [t][k] (k
// contiguous, stride kF8Stride) whatever the source's layout; each half of
// warp w forms row t0 + 2w (+ 1) of each leaf's sum, 8 consecutive k per
// lane, reduces the block's max |sum| across its 16 lanes, picks
// s = e(max) - 8 (0 for a zero block; at least -127), rounds sum 2^-s to
// E4M3 (ties to even) and writes the 128 bytes of its row plus its scale.
constexpr int kF8TT = 16;
constexpr int kF8Stride = 132;

// The row's four sums of one leaf (lanes: 4 consecutive k each, 128 k per
// warp): the block's max |sum| across the warp, s = e(max) - 8 (0 for a
// zero block; at least -127, the smallest UE8M0 scale, so blocks whose max
// is below 2^-120 use E4M3 subnormals), sum 2^-s rounded to E4M3 (ties to
// even), the 4 bytes stored, and the block's scale (lane 0): the factor 2^s
// or, with sf_atoms, the UE8M0 byte s + 127 at the row's place in the
// block-scale atom.
__device__ __forceinline__ void e4m3_store_row(const CombineArgs& a, int r, int64_t t, int64_t k0, int lane,
                                               const float (&acc)[4]) {
  float m = fmaxf(fmaxf(fabsf(acc[0]), fabsf(acc[1])), fmaxf(fabsf(acc[2]), fabsf(acc[3])));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  bool nf = false;
  const int e = fexp_f32(__float_as_uint(m), &nf);
  const int sc = m > 0.f ? max(e - 8, -127) : 0;
  uint32_t packed = 0;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float2 pr = make_float2(scale_pow2(acc[2 * j], -sc), scale_pow2(acc[2 * j + 1], -sc));
    const uint32_t q = (uint32_t)__nv_cvt_float2_to_fp8x2(pr, __NV_SATFINITE, __NV_E4M3);
    packed |= q << (16 * j);
  }
  unsigned char* out = static_cast<unsigned char*>(a.out);
  *reinterpret_cast<uint32_t*>(out + ((int64_t)r * a.p_rows + t) * a.p_cols + k0 + 4 * lane) = packed;
  if (lane == 0) {
    const int64_t kb = k0 / 128, nkb = a.p_cols / 128;
    if (a.sf_atoms) {
      const int64_t atom = ((int64_t)r * nkb + kb) * (a.p_rows / 128) + t / 128;
      reinterpret_cast<uint32_t*>(a.scale_out)[atom * 128 + (t % 32) * 4 + (t % 128) / 32] =
          (uint32_t)(sc + 127) * 0x01010101u;
    } else {
      a.scale_out[((int64_t)r * nkb + kb) * a.p_rows + t] = exp2i(sc);
    }
  }
}

// The same for a row held by a half-warp, 8 consecutive k per lane (sub =
// lane within the half): the block max reduced over the 16 lanes, 8 bytes
// stored per lane, the scale by the half's first lane.
__device__ __forceinline__ void e4m3_store_row8(const CombineArgs& a, int r, int64_t t, int64_t k0, int sub,
                                                const float (&acc)[8]) {
  float m = fmaxf(fmaxf(fmaxf(fabsf(acc[0]), fabsf(acc[1])), fmaxf(fabsf(acc[2]), fabsf(acc[3]))),
                  fmaxf(fmaxf(fabsf(acc[4]), fabsf(acc[5])), fmaxf(fabsf(acc[6]), fabsf(acc[7]))));
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  bool nf = false;
  const int e = fexp_f32(__float_as_uint(m), &nf);
  const int sc = m > 0.f ? max(e - 8, -127) : 0;
  uint32_t packed[2] = {0u, 0u};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 pr = make_float2(scale_pow2(acc[2 * j], -sc), scale_pow2(acc[2 * j + 1], -sc));
    const uint32_t q = (uint32_t)__nv_cvt_float2_to_fp8x2(pr, __NV_SATFINITE, __NV_E4M3);
    packed[j >> 1] |= q << (16 * (j & 1));
  }
  unsigned char* out = static_cast<unsigned char*>(a.out);
  *reinterpret_cast<uint2*>(out + ((int64_t)r * a.p_rows + t) * a.p_cols + k0 + 8 * sub) =
      make_uint2(packed[0], packed[1]);
  if (sub == 0) {
    const int64_t kb = k0 / 128, nkb = a.p_cols / 128;
    if (a.sf_atoms) {
      const int64_t atom = ((int64_t)r * nkb + kb) * (a.p_rows / 128) + t / 128;
      reinterpret_cast<uint32_t*>(a.scale_out)[atom * 128 + (t % 32) * 4 + (t % 128) / 32] =
          (uint32_t)(sc + 127) * 0x01010101u;
    } else {
      a.scale_out[((int64_t)r * nkb + kb) * a.p_rows + t] = exp2i(sc);
    }
  }
}

// Threads of the E4M3 combination CTA: two rows per warp in the sums, at
// least four warps for the staging.
template <int TT>
constexpr int e4m3_threads() { return TT * 16 > 128 ? TT * 16 : 128; }

template <int DT, int TT>
__global__ void __launch_bounds__(e4m3_threads<TT>()) combine_e4m3_kernel(const CombineArgs a) {
  extern __shared__ float f8tile[];  // [block][TT][kF8Stride], then the term list
  constexpr int kThr = e4m3_threads<TT>();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t t0 = (int64_t)blockIdx.y * TT, k0 = (int64_t)blockIdx.x * 128;
  const int n_rb = (int)a.n_rb, n_cb = (int)a.n_cb, nb = n_rb * n_cb;
  const int R = (int)a.num_leaves, nnz = (int)a.t_nnz;
  int* toff = reinterpret_cast<int*>(f8tile + nb * TT * kF8Stride);
  float* tcoef = reinterpret_cast<float*>(toff + nnz);
  int* tstart = reinterpret_cast<int*>(tcoef + nnz);
  for (int i = tid; i < nnz; i += kThr) {
    const int32_t blk = __ldg(a.t_blk + i);
    const int bt = (blk >> a.blk_t_shift) & 0xFFFF, bk = (blk >> a.blk_k_shift) & 0xFFFF;
    toff[i] = (a.t_rows ? bt * n_cb + bk : bk * n_cb + bt) * TT * kF8Stride;
    tcoef[i] = __ldg(a.t_coef + i);
  }
  for (int i = tid; i <= R; i += kThr) tstart[i] = __ldg(a.t_start + i);
  // staging: position (t, k) of block (rb, cb) -> memory (t, k) (k
  // contiguous) or (k, t) (t contiguous); each thread loads 4 consecutive
  // memory columns (one vector load where the row allows)
  const int es = DT == kF32 ? 4 : 2;
  const bool vec_ok = ((uintptr_t)a.src % (4 * es) == 0) && (a.ld % 4 == 0) && (a.b_cols % 4 == 0);
  constexpr int kRowThreadsT = 32, kRowThreadsK = TT / 4;  // threads per memory row
  for (int rb = 0; rb < n_rb; ++rb) {
    for (int cb = 0; cb < n_cb; ++cb) {
      float* tile = f8tile + (rb * n_cb + cb) * TT * kF8Stride;
      const int64_t nr = min(a.b_rows, a.rows - rb * a.b_rows), nc = min(a.b_cols, a.cols - cb * a.b_cols);
      const int per_row = a.t_rows ? kRowThreadsT : kRowThreadsK;
      const int n_items = a.t_rows ? TT * kRowThreadsT : 128 * kRowThreadsK;
      for (int i = tid; i < n_items; i += kThr) {
        const int mrow = i / per_row, mcol = 4 * (i % per_row);  // within the CTA's window
        const int64_t lr = (a.t_rows ? t0 : k0) + mrow, lc = (a.t_rows ? k0 : t0) + mcol;
        const int64_t gr = rb * a.b_rows + lr, gc = cb * a.b_cols + lc;
        float x[4];
        const int er = (a.re && lr < nr) ? a.rs * __ldg(a.re + gr) : 0;
        if (vec_ok && lr < nr && lc + 4 <= nc) {
          load4<DT>(a.src, gr * a.ld + gc, x);
#pragma unroll
          for (int j = 0; j < 4; ++j) x[j] = scale_pow2(x[j], er + (a.ce ? a.cs * __ldg(a.ce + gc + j) : 0));
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            x[j] = (lr < nr && lc + j < nc)
                       ? scale_pow2(load_elem<DT>(a.src, gr * a.ld + gc + j),
                                    er + (a.ce ? a.cs * __ldg(a.ce + gc + j) : 0))
                       : 0.f;
        }
        if (a.t_rows) {
          *reinterpret_cast<float4*>(tile + mrow * kF8Stride + mcol) = make_float4(x[0], x[1], x[2], x[3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) tile[(mcol + j) * kF8Stride + mrow] = x[j];
        }
      }
    }
  }
  __syncthreads();
  // half-warp h of warp w forms row 2w + h, 8 consecutive k per lane
  const int row = 2 * warp + (lane >> 4), sub = lane & 15;
  if (row >= TT) return;  // staging-only warps (warp-uniform)
  const int64_t t = t0 + row;
  const float* trow = f8tile + row * kF8Stride + 8 * sub;
  int tt = 0;
  for (int r = 0; r < R; ++r) {
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int t1 = tstart[r + 1];
    for (; tt < t1; ++tt) {
      const float coef = tcoef[tt];
      const float4 v0 = *reinterpret_cast<const float4*>(trow + toff[tt]);
      const float4 v1 = *reinterpret_cast<const float4*>(trow + toff[tt] + 4);
      acc[0] = fmaf(coef, v0.x, acc[0]);
      acc[1] = fmaf(coef, v0.y, acc[1]);
      acc[2] = fmaf(coef, v0.z, acc[2]);
      acc[3] = fmaf(coef, v0.w, acc[3]);
      acc[4] = fmaf(coef, v1.x, acc[4]);
      acc[5] = fmaf(coef, v1.y, acc[5]);
      acc[6] = fmaf(coef, v1.z, acc[6]);
      acc[7] = fmaf(coef, v1.w, acc[7]);
    }
    e4m3_store_row8(a, r, t, k0, sub, acc);
  }
}

// Unstaged form for operands with more input blocks than the staged tiles
// hold: one warp per row t of a 16-row, 128-k window, each term's four
// elements per lane loaded straight from the source (the window's input
// tiles are reused from L1 / L2 across terms and warps), scaled and summed
// in term order as above, so the sums and their rounding are the staged
// kernel's.
template <int DT>
__global__ void __launch_bounds__(kF8TT * 32) combine_e4m3_direct_kernel(const CombineArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t0 = (int64_t)blockIdx.y * kF8TT, k0 = (int64_t)blockIdx.x * 128;
  const int64_t t = t0 + warp;
  const int R = (int)a.num_leaves;
  // this lane's memory positions inside a block: (row, column) offsets of
  // (t, k0 + 4 lane + j), j = 0..3
  const int64_t lt = t0 + warp, lk = k0 + 4 * lane;
  for (int r = 0; r < R; ++r) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int t1 = __ldg(a.t_start + r + 1);
    for (int tt = __ldg(a.t_start + r); tt < t1; ++tt) {
      const int32_t blk = __ldg(a.t_blk + tt);
      const int64_t bt = (blk >> a.blk_t_shift) & 0xFFFF, bk = (blk >> a.blk_k_shift) & 0xFFFF;
      const float coef = __ldg(a.t_coef + tt);
      const int64_t rb = a.t_rows ? bt : bk, cb = a.t_rows ? bk : bt;
      const int64_t nr = min(a.b_rows, a.rows - rb * a.b_rows), nc = min(a.b_cols, a.cols - cb * a.b_cols);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t lr = a.t_rows ? lt : lk + j, lc = a.t_rows ? lk + j : lt;
        float v = 0.f;
        if (lr < nr && lc < nc) {
          const int64_t gr = rb * a.b_rows + lr, gc = cb * a.b_cols + lc;
          const int er = (a.re ? a.rs * __ldg(a.re + gr) : 0) + (a.ce ? a.cs * __ldg(a.ce + gc) : 0);
          v = scale_pow2(load_elem<DT>(a.src, gr * a.ld + gc), er);
        }
        acc[j] = fmaf(coef, v, acc[j]);
      }
    }
    e4m3_store_row(a, r, t, k0, lane, acc);
  }
}

// FMM_E4M3_DIRECT=1 in the environment (read once): the unstaged E4M3
// combination whatever the block count (testing: it must give the staged
// kernel's bytes and scales exactly).
static bool e4m3_direct_forced() {
  static bool on = [] {
    const char* s = std::getenv("FMM_E4M3_DIRECT");
    return s && std::atoi(s) != 0;
  }();
  return on;
}

cudaError_t launch_combine_e4m3(const CombineArgs& a, cudaStream_t st) {
  if (a.p_rows % kF8TT != 0 || a.p_cols % 128 != 0 || (a.sf_atoms && a.p_rows % 128 != 0)) return cudaErrorInvalidValue;
  const int64_t nb = a.n_rb * a.n_cb;
  const size_t list = (size_t)a.t_nnz * 8 + (size_t)(a.num_leaves + 1) * 4;
  // sixteen rows per CTA when the staged tiles fit, else four, else the
  // unstaged kernel (sixteen rows)
  const bool wide = (size_t)nb * kF8TT * kF8Stride * 4 + list <= kStagedSmemMax;
  const int tt = wide ? kF8TT : 4;
  const size_t smem = (size_t)nb * tt * kF8Stride * 4 + list;
  if (a.p_rows / 4 > 65535) return cudaErrorNotSupported;
  if (a.num_leaves == 0 || a.p_rows == 0 || a.p_cols == 0) return cudaSuccess;
  if (smem > kStagedSmemMax || e4m3_direct_forced()) {
    const dim3 grid((unsigned)(a.p_cols / 128), (unsigned)(a.p_rows / kF8TT));
    KernelTimer timer("combine", st);
    switch (a.dtype) {
      case kF32: combine_e4m3_direct_kernel<kF32><<<grid, kF8TT * 32, 0, st>>>(a); break;
      case kBF16: combine_e4m3_direct_kernel<kBF16><<<grid, kF8TT * 32, 0, st>>>(a); break;
      default: combine_e4m3_direct_kernel<kF16><<<grid, kF8TT * 32, 0, st>>>(a); break;
    }
    return cudaGetLastError();
  }
  static bool attr_done[64][6] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  const dim3 grid((unsigned)(a.p_cols / 128), (unsigned)(a.p_rows / tt));
  KernelTimer timer("combine", st);
  auto go = [&](auto kern, int idx) {
    if (!attr_done[dev][idx]) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStagedSmemMax);
      attr_done[dev][idx] = true;
    }
    kern<<<grid, wide ? e4m3_threads<kF8TT>() : e4m3_threads<4>(), smem, st>>>(a);
  };
  switch (a.dtype) {
    case kF32: wide ? go(combine_e4m3_kernel<kF32, kF8TT>, 0) : go(combine_e4m3_kernel<kF32, 4>, 3); break;
    case kBF16: wide ? go(combine_e4m3_kernel<kBF16, kF8TT>, 1) : go(combine_e4m3_kernel<kBF16, 4>, 4); break;
    default: wide ? go(combine_e4m3_kernel<kF16, kF8TT>, 2) : go(combine_e4m3_kernel<kF16, 4>, 5); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_node_exp(const CombineArgs& a, int* out, int64_t k1, cudaStream_t st) {
  const int64_t nb = a.n_rb * a.n_cb;
  const size_t smem = (size_t)nb * kNodeTR * 256 + (size_t)a.num_leaves * kTC * 4;
  if (smem > kStagedSmemMax) return cudaErrorInvalidValue;
  const int64_t rows = a.b_rows, cols = a.b_cols;
  if (rows == 0 || cols == 0 || a.num_leaves == 0) return cudaSuccess;
  static bool attr_done[64][3] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  const dim3 grid((unsigned)((cols + kTC - 1) / kTC), (unsigned)((rows + kNodeTR - 1) / kNodeTR));
  KernelTimer timer("combine", st);
  auto go = [&](auto kern, int idx) {
    if (!attr_done[dev][idx]) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStagedSmemMax);
      attr_done[dev][idx] = true;
    }
    kern<<<grid, kNodeTR * 16, smem, st>>>(a, out, k1);
  };
  switch (a.dtype) {
    case kF32: go(node_exp_kernel<kF32>, 0); break;
    case kBF16: go(node_exp_kernel<kBF16>, 1); break;
    default: go(node_exp_kernel<kF16>, 2); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_between_finalize(const int* cexp, const int* rexp, int* d, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  KernelTimer timer("scale", st);
  between_finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cexp, rexp, d, n);
  return cudaGetLastError();
}

cudaError_t launch_out_gather(const OutArgs& a, cudaStream_t st) {
  if (!a.g_start || a.c.bm > a.tp_a || a.c.bn > a.tp_b || a.tp_b % kTC != 0) return cudaErrorInvalidValue;
  if (a.c.bm == 0 || a.c.bn == 0) return cudaSuccess;
  KernelTimer timer("combine", st);
  const int64_t tiles = ((a.c.bn + kTC - 1) / kTC) * ((a.c.bm + kOutGatherRows - 1) / kOutGatherRows);
  if (tiles > 0x7FFFFFFF) return cudaErrorInvalidValue;
  const unsigned gy = (unsigned)std::min<int64_t>(a.c_blocks, 65535);
  return launch_pdl(out_gather_kernel, dim3((unsigned)tiles, gy), dim3(kOutGatherRows * 16), 0, st, a);
}

cudaError_t launch_out_dense_slim(const OutArgs& a, cudaStream_t st) {
  if (a.c_blocks > 16 || a.num_leaves * 16 * 4 > 48 * 1024 || a.c.bm > a.tp_a || a.c.bn > a.tp_b ||
      a.tp_b % kTC != 0)
    return cudaErrorNotSupported;
  const int64_t rows = (a.r_end ? std::min(a.r_end, a.c.bm) : a.c.bm) - a.r_begin;
  if (rows <= 0 || a.c.bn == 0) return cudaSuccess;
  KernelTimer timer("combine", st);
  constexpr int TR = 16, TC = kTC;  // 256 threads
  const dim3 grid((unsigned)((a.c.bn + TC - 1) / TC), (unsigned)((rows + TR - 1) / TR));
  const size_t smem = (size_t)a.num_leaves * 16 * 4;
  if (a.c_blocks <= 4) return launch_pdl(out_dense_kernel<4, TR, TC, 3>, grid, dim3(TR * TC / 4), smem / 4, st, a);
  if (a.c_blocks <= 9) return launch_pdl(out_dense_kernel<9, TR, TC, 3>, grid, dim3(TR * TC / 4), smem * 9 / 16, st, a);
  return launch_pdl(out_dense_kernel<16, TR, TC, 3>, grid, dim3(TR * TC / 4), smem, st, a);
}

cudaError_t launch_out_combine(const OutArgs& a, cudaStream_t st) {
  if (a.c_blocks > kMaxOutBlocks || a.c.bm > a.tp_a || a.c.bn > a.tp_b || a.tp_b % kTC != 0)
    return cudaErrorInvalidValue;
  if (a.c.bm == 0 || a.c.bn == 0) return cudaSuccess;
  if (a.c_blocks <= 16 && a.num_leaves * 16 * 4 <= 48 * 1024) {
    // register accumulators
    KernelTimer timer("combine", st);
    auto go = [&](auto nb_tag, auto tr_tag) {
      constexpr int NB = decltype(nb_tag)::value, TR = decltype(tr_tag)::value, TC = kTC;
      const int64_t rows = (a.r_end ? std::min(a.r_end, a.c.bm) : a.c.bm) - a.r_begin;
      if (rows <= 0) return;
      const unsigned gy = (unsigned)((rows + TR - 1) / TR);
      launch_pdl(out_dense_kernel<NB, TR, TC>, dim3((unsigned)((a.c.bn + TC - 1) / TC), gy), dim3(TR * TC / 4),
                 (size_t)a.num_leaves * NB * 4, st, a);
    };
    // TR rows of 64 columns (measured: wider rows were no faster)
    if (a.c_blocks <= 4) go(std::integral_constant<int, 4>(), std::integral_constant<int, 32>());
    else if (a.c_blocks <= 9) go(std::integral_constant<int, 9>(), std::integral_constant<int, 16>());
    else go(std::integral_constant<int, 16>(), std::integral_constant<int, 16>());
    return cudaGetLastError();
  }
  const size_t list_bytes = (size_t)a.c_nnz * 8 + (size_t)(a.num_leaves + 1) * 4;
  if (list_bytes > 150 * 1024) return cudaErrorInvalidValue;
  KernelTimer timer("combine", st);
  const unsigned gx = (unsigned)((a.c.bn + kTC - 1) / kTC);
  const int nb = (int)a.c_blocks;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  // TR rows per CTA so that the accumulators take at most 48 KB
  auto go = [&](auto tr_tag) {
    constexpr int TR = decltype(tr_tag)::value;
    static bool attr_done[64] = {};
    if (!attr_done[dev]) {
      cudaFuncSetAttribute(out_combine_kernel<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr_done[dev] = true;
    }
    const unsigned gy = (unsigned)((a.c.bm + TR - 1) / TR);
    launch_pdl(out_combine_kernel<TR>, dim3(gx, gy), dim3(TR * 16), (size_t)nb * TR * 256 + list_bytes, st, a);
  };
  if (nb <= 6) go(std::integral_constant<int, 32>());
  else if (nb <= 12) go(std::integral_constant<int, 16>());
  else if (nb <= 24) go(std::integral_constant<int, 8>());
  else if (nb <= 48) go(std::integral_constant<int, 4>());
  else go(std::integral_constant<int, 2>());
  return cudaGetLastError();
}

// Rows per CTA of the staged combination for a block count (tiles <= 32 KB).
static int staged_tr(int64_t nb) { return nb <= 4 ? 32 : nb <= 8 ? 16 : nb <= 16 ? 8 : nb <= 32 ? 4 : 2; }
// Rows per CTA of the output pass for a C block count (accumulators <= 48 KB).
static int out_tr(int64_t nb) { return nb <= 6 ? 32 : nb <= 12 ? 16 : nb <= 24 ? 8 : nb <= 48 ? 4 : 2; }

int combine_batched_rows(int64_t max_blocks) { return staged_tr(max_blocks); }
int out_batched_rows(int64_t max_c_blocks) { return out_tr(max_c_blocks); }

template <int DT, int FMT, int TR>
static void launch_combine_batched_tr(const CombineArgs* args, const int64_t* start, int count, int64_t total,
                                      size_t smem, cudaStream_t st) {
  constexpr int RPT = TR == 32 ? 2 : 1;
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr_done[dev]) {
    cudaFuncSetAttribute(combine_staged_batched_kernel<DT, FMT, TR, RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kStagedSmemMax);
    attr_done[dev] = true;
  }
  // one CTA per tile (a grid of a few CTAs per SM looping over the tiles
  // measured slower: it loses the overlap of one tile's loads with
  // another's arithmetic that independent CTAs give)
  combine_staged_batched_kernel<DT, FMT, TR, RPT><<<(unsigned)total, TR * 16 / RPT, smem, st>>>(args, start, count,
                                                                                                total);
}

template <int DT, int FMT>
static void launch_combine_batched_fmt(const CombineArgs* args, const int64_t* start, int count, int64_t total,
                                       int tr, size_t smem, cudaStream_t st) {
  switch (tr) {
    case 32: launch_combine_batched_tr<DT, FMT, 32>(args, start, count, total, smem, st); break;
    case 16: launch_combine_batched_tr<DT, FMT, 16>(args, start, count, total, smem, st); break;
    case 8: launch_combine_batched_tr<DT, FMT, 8>(args, start, count, total, smem, st); break;
    case 4: launch_combine_batched_tr<DT, FMT, 4>(args, start, count, total, smem, st); break;
    default: launch_combine_batched_tr<DT, FMT, 2>(args, start, count, total, smem, st); break;
  }
}

cudaError_t launch_combine_batched(const CombineArgs* args, const int64_t* start, int count, int64_t total, int dt,
                                   int fmt, int tr, size_t smem, cudaStream_t st) {
  if (total == 0 || count == 0) return cudaSuccess;
  if (smem > kStagedSmemMax) return cudaErrorInvalidValue;
  KernelTimer timer("combine", st);
#define FMM_CB(DT)                                                                                   \
  switch (fmt) {                                                                                     \
    case FMM_LEAF_BF16: launch_combine_batched_fmt<DT, FMM_LEAF_BF16>(args, start, count, total, tr, smem, st); break; \
    case FMM_LEAF_F16: launch_combine_batched_fmt<DT, FMM_LEAF_F16>(args, start, count, total, tr, smem, st); break;   \
    default: launch_combine_batched_fmt<DT, FMM_LEAF_BF16X3>(args, start, count, total, tr, smem, st); break;         \
  }
  switch (dt) {
    case kF32: FMM_CB(kF32) break;
    case kBF16: FMM_CB(kBF16) break;
    default: FMM_CB(kF16) break;
  }
#undef FMM_CB
  return cudaGetLastError();
}

cudaError_t launch_out_combine_batched(const OutArgs* args, const int64_t* start, int count, int64_t total, int tr,
                                       size_t smem, cudaStream_t st) {
  if (total == 0 || count == 0) return cudaSuccess;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  KernelTimer timer("combine", st);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  auto go = [&](auto tr_tag) {
    constexpr int TR = decltype(tr_tag)::value;
    static bool attr_done[64] = {};
    if (!attr_done[dev]) {
      cudaFuncSetAttribute(out_combine_batched_kernel<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr_done[dev] = true;
    }
    out_combine_batched_kernel<TR><<<(unsigned)total, TR * 16, smem, st>>>(args, start, count, total);
  };
  switch (tr) {
    case 32: go(std::integral_constant<int, 32>()); break;
    case 16: go(std::integral_constant<int, 16>()); break;
    case 8: go(std::integral_constant<int, 8>()); break;
    case 4: go(std::integral_constant<int, 4>()); break;
    default: go(std::integral_constant<int, 2>()); break;
  }
  return cudaGetLastError();
}

size_t combine_staged_smem(int64_t nb, int tr, int64_t nnz, int64_t leaves) { return staged_smem((int)nb, tr, nnz, leaves); }

cudaError_t launch_combine(const CombineArgs& a, cudaStream_t st) {
  if (a.p_rows % kTR != 0 || a.p_cols % kTC != 0 || a.p_rows / kTR > 65535) return cudaErrorInvalidValue;
  if (a.between_d) {
    const int64_t nb = a.n_rb * a.n_cb;
    const int tr = nb <= 4 ? 32 : nb <= 8 ? 16 : nb <= 16 ? 8 : nb <= 32 ? 4 : 2;
    if (nb > kMaxStaged || staged_smem((int)nb, tr, a.t_nnz, a.num_leaves) > kStagedSmemMax)
      return cudaErrorNotSupported;  // the between-steps scale needs the staged form
  }
  if (a.b_rows > a.p_rows || a.b_cols > a.p_cols) return cudaErrorInvalidValue;
  if (a.num_leaves == 0 || a.p_rows == 0 || a.p_cols == 0) return cudaSuccess;
  const dim3 grid((unsigned)(a.p_cols / kTC), (unsigned)(a.p_rows / kTR));
  switch (a.dtype) {
    case kF32: return launch_dt<kF32>(a, grid, st);
    case kBF16: return launch_dt<kBF16>(a, grid, st);
    default: return launch_dt<kF16>(a, grid, st);
  }
}

// ------------------------------------------------------------ streamed form
// The unrolled combination (at most 2 x 2 FP32 source blocks) as a
// persistent kernel that streams the input tiles with bulk tensor copies:
// each CTA walks position tiles t = blockIdx.x, + gridDim.x, ... of both
// operands (a0's tiles first), and one thread keeps kStreamStages tiles of
// every block in flight through an mbarrier ring, so loads no longer wait
// for the previous tile's stores.  Per tile the threads scale their own
// elements in place (2^(re + ce), exactly as the unrolled form does), then
// sum each leaf's terms in term order and store the rounded leaf values:
// the same arithmetic, so the same results.  Every tile of a block lies
// inside the block (b_rows, b_cols multiples of 8 and 256 unless the block
// is the last one along that side, whose rows and columns past the source
// read as zero from the tensor map).  Tiles are 8 rows x 256 columns, so
// every source row piece is 1 KB and every output row piece 512 bytes of
// contiguous memory.
constexpr int kStreamStages = 3;
constexpr int kStreamTR = 8, kStreamTC = 256;  // position tile: 8 rows x 256 columns (1 KB source rows)
constexpr int kStreamBox = kStreamTR * kStreamTC;  // floats per block tile

template <int NB>
constexpr size_t stream_smem_fixed() {
  return (size_t)kStreamStages * NB * kStreamBox * 4 + 64;
}

template <int FMT, int NRB, int NCB>
__global__ void __launch_bounds__(256, 2) combine_stream_kernel(const __grid_constant__ CUtensorMap m0,
                                                                const __grid_constant__ CUtensorMap m1,
                                                                const __grid_constant__ CombineArgs a0,
                                                                const __grid_constant__ CombineArgs a1, int64_t tiles0,
                                                                int64_t tiles, int* status, uint64_t timeout_ns) {
  constexpr int NB = NRB * NCB, TR = kStreamTR, TC = kStreamTC;
  constexpr int kQ = TC / 4;                 // threads across a tile row (4 columns each)
  constexpr int kRowsPer = 256 / kQ;         // rows covered by one pass of the CTA
  constexpr int kPasses = TR / kRowsPer;     // rows per thread
  extern __shared__ __align__(128) uint8_t sm[];
  float4* stages = reinterpret_cast<float4*>(sm);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)kStreamStages * NB * kStreamBox * 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(full + kStreamStages);
  int2* terms = reinterpret_cast<int2*>(sm + stream_smem_fixed<NB>());  // a0's terms, then a1's
  const int nnz0 = (int)a0.t_nnz, nnz1 = (int)a1.t_nnz;
  int* tstart = reinterpret_cast<int*>(terms + nnz0 + nnz1);        // a0's R0 + 1 starts, then a1's
  const int R0 = (int)a0.num_leaves, R1 = (int)a1.num_leaves;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStreamStages; ++s) mbar_init(&full[s], 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  // term lists: (float4 offset of the term's block tile, coefficient bits)
  auto load_terms = [&](const CombineArgs& a, int2* dst, int* ts, int nnz, int R) {
    for (int i = threadIdx.x; i < nnz; i += 256) {
      const int32_t blk = __ldg(a.t_blk + i);
      const int bt = (blk >> a.blk_t_shift) & 0xFFFF, bk = (blk >> a.blk_k_shift) & 0xFFFF;
      dst[i] = make_int2((a.t_rows ? bt * NCB + bk : bk * NCB + bt) * (kStreamBox / 4),
                         __float_as_int(__ldg(a.t_coef + i)));
    }
    for (int i = threadIdx.x; i <= R; i += 256) ts[i] = __ldg(a.t_start + i);
  };
  load_terms(a0, terms, tstart, nnz0, R0);
  load_terms(a1, terms + nnz0, tstart + R0 + 1, nnz1, R1);
  __syncthreads();
  // the sources' exponents (and a source written by the previous kernel)
  // are read from here on
  pdl_wait();
  pdl_trigger();

  auto issue = [&](int64_t t, int s) {
    const bool second = t >= tiles0;
    const CombineArgs& a = second ? a1 : a0;
    const CUtensorMap* m = second ? &m1 : &m0;
    const int64_t lt = second ? t - tiles0 : t, gx = a.p_cols / TC;
    const int64_t r0 = (lt / gx) * TR, c0 = (lt % gx) * TC;
    gemm::mbar_arrive_expect_tx(&full[s], (uint32_t)(NB * kStreamBox * 4));
#pragma unroll
    for (int rb = 0; rb < NRB; ++rb)
#pragma unroll
      for (int cb = 0; cb < NCB; ++cb)
        gemm::tma_load_2d(stages + ((size_t)s * NB + rb * NCB + cb) * (kStreamBox / 4), m,
                          (int32_t)(cb * a.b_cols + c0), (int32_t)(rb * a.b_rows + r0), &full[s]);
  };
  const int64_t G = gridDim.x;
  if (threadIdx.x == 0)
    for (int i = 0; i < kStreamStages - 1; ++i) {
      const int64_t t = blockIdx.x + i * G;
      if (t < tiles) issue(t, i);
    }
  const int tr = threadIdx.x / kQ, tq = threadIdx.x % kQ, tc = tq * 4;
  const int me = tr * kQ + tq;  // float4 slot of row tr; row tr + kRowsPer * q at me + 256 q
  int64_t issued_upto = blockIdx.x + (kStreamStages - 1) * G;  // first tile not yet issued
  int i = 0;
  for (int64_t t = blockIdx.x; t < tiles; t += G, ++i) {
    const int s = i % kStreamStages;
    const uint32_t ph = (uint32_t)(i / kStreamStages) & 1u;
    if (threadIdx.x == 0) {
      // the stage of tile i - 1 was released by the barrier that ended it
      const int64_t tn = t + (kStreamStages - 1) * G;
      if (tn < tiles) {
        fence_proxy_async_smem();
        issue(tn, (i + kStreamStages - 1) % kStreamStages);
        issued_upto = tn + G;
      }
    }
    const bool ok = mbar_wait_bounded(&full[s], ph, abort_flag, timeout_ns);
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
      break;
    }
    const bool second = t >= tiles0;
    const CombineArgs& a = second ? a1 : a0;
    const int2* tm = second ? terms + nnz0 : terms;
    const int* ts = second ? tstart + R0 + 1 : tstart;
    const int R = second ? R1 : R0;
    const int64_t lt = second ? t - tiles0 : t, gx = a.p_cols / TC;
    const int64_t r0 = (lt / gx) * TR, c0 = (lt % gx) * TC, lc = c0 + tc;
    float4* tile4 = stages + (size_t)s * NB * (kStreamBox / 4);
    // scale this thread's elements in place: 2^(rs re[row] + cs ce[col])
    if (a.re || a.ce) {
#pragma unroll
      for (int cb = 0; cb < NCB; ++cb) {
        const int64_t nc = min(a.b_cols, a.cols - cb * a.b_cols);
        int ec[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          ec[j] = (a.ce && lc + j < nc) ? a.cs * __ldg(a.ce + cb * a.b_cols + lc + j) : 0;
#pragma unroll
        for (int rb = 0; rb < NRB; ++rb) {
          const int64_t nr = min(a.b_rows, a.rows - rb * a.b_rows);
#pragma unroll
          for (int q = 0; q < kPasses; ++q) {
            const int64_t lr = r0 + tr + kRowsPer * q;
            const int er = (a.re && lr < nr) ? a.rs * __ldg(a.re + rb * a.b_rows + lr) : 0;
            float4& v = tile4[(rb * NCB + cb) * (kStreamBox / 4) + me + 256 * q];
            v = make_float4(scale_fast(v.x, er + ec[0]), scale_fast(v.y, er + ec[1]), scale_fast(v.z, er + ec[2]),
                            scale_fast(v.w, er + ec[3]));
          }
        }
      }
    }
    unsigned short* out = static_cast<unsigned short*>(a.out);
    const int64_t leaf_stride = a.p_rows * a.p_cols;
    const int64_t plane = (int64_t)R * leaf_stride;
    unsigned short* orow = out + (r0 + tr) * a.p_cols + lc;
    const int64_t qstride = (int64_t)kRowsPer * a.p_cols;
    int k = 0;
    for (int r = 0; r < R; ++r, orow += leaf_stride) {
      const int k1 = ts[r + 1];
      float acc[kPasses][4];
#pragma unroll
      for (int q = 0; q < kPasses; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
      for (; k < k1; ++k) {
        const int2 term = tm[k];
        const float coef = __int_as_float(term.y);
#pragma unroll
        for (int q = 0; q < kPasses; ++q) {
          const float4 v = tile4[term.x + me + 256 * q];
          acc[q][0] = fmaf(coef, v.x, acc[q][0]);
          acc[q][1] = fmaf(coef, v.y, acc[q][1]);
          acc[q][2] = fmaf(coef, v.z, acc[q][2]);
          acc[q][3] = fmaf(coef, v.w, acc[q][3]);
        }
      }
#pragma unroll
      for (int q = 0; q < kPasses; ++q) store4<FMT>(orow + q * qstride, orow + q * qstride + plane, acc[q]);
    }
    __syncthreads();  // stage s is free again
  }
  // no copy may still be writing shared memory when the CTA exits (only
  // after a timeout can one be outstanding): wait for each issued stage
  if (threadIdx.x == 0) {
    for (int64_t tt = blockIdx.x + (int64_t)i * G, j = i; tt < issued_upto && tt < tiles; tt += G, ++j) {
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(&full[j % kStreamStages], (uint32_t)(j / kStreamStages) & 1u) &&
             globaltimer_ns() - t0 < 1000000000ull) {
      }
    }
  }
  __syncthreads();
}

// Whether the streamed form applies to one operand (see above).
bool stream_ok(const CombineArgs& a) {
  const int64_t nb = a.n_rb * a.n_cb;
  return a.dtype == kF32 && a.n_rb <= 2 && a.n_cb <= 2 && !a.between_d && a.fmt != FMM_LEAF_E4M3B128 &&
         a.p_rows % kStreamTR == 0 && a.p_cols % kStreamTC == 0 && (a.n_rb == 1 || a.b_rows % kStreamTR == 0) &&
         (a.n_cb == 1 || a.b_cols % kStreamTC == 0) && a.b_rows <= a.p_rows && a.b_cols <= a.p_cols &&
         (uintptr_t)a.src % 16 == 0 && (a.ld * 4) % 16 == 0 && (!a.ce || (uintptr_t)a.ce % 16 == 0) && nb >= 1 &&
         a.num_leaves > 0 && a.rows < 0x7FFFFFFF && a.cols < 0x7FFFFFFF;
}

cudaError_t launch_combine_pair_stream(const CombineArgs& a0, const CUtensorMap& m0, const CombineArgs& a1,
                                       const CUtensorMap& m1, uint64_t timeout_ns, int* status, cudaStream_t st) {
  if (!stream_ok(a0) || !stream_ok(a1) || a0.fmt != a1.fmt || a0.n_rb != a1.n_rb || a0.n_cb != a1.n_cb)
    return cudaErrorNotSupported;
  const int64_t tiles0 = (a0.p_cols / kStreamTC) * (a0.p_rows / kStreamTR),
                tiles = tiles0 + (a1.p_cols / kStreamTC) * (a1.p_rows / kStreamTR);
  const size_t list = (size_t)(a0.t_nnz + a1.t_nnz) * 8 + (size_t)(a0.num_leaves + a1.num_leaves + 2) * 4;
  if (tiles == 0 || list > 16384) return cudaErrorNotSupported;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)device_sms() * 2);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  KernelTimer timer("combine", st);
  auto go = [&](auto fmt_tag, auto nrb_tag, auto ncb_tag) {
    constexpr int FMT = decltype(fmt_tag)::value, NRB = decltype(nrb_tag)::value, NCB = decltype(ncb_tag)::value;
    auto kern = combine_stream_kernel<FMT, NRB, NCB>;
    const size_t smem = stream_smem_fixed<NRB * NCB>() + list;
    static bool attr[64] = {};
    if (!attr[dev]) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 110 * 1024);
      attr[dev] = true;
    }
    return launch_pdl(kern, dim3((unsigned)grid), dim3(256), smem, st, m0, m1, a0, a1, tiles0, tiles, status,
                      timeout_ns);
  };
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  auto by_blocks = [&](auto fmt_tag) {
    if (a0.n_rb == 2 && a0.n_cb == 2) return go(fmt_tag, I2(), I2());
    if (a0.n_rb == 2) return go(fmt_tag, I2(), I1());
    if (a0.n_cb == 2) return go(fmt_tag, I1(), I2());
    return go(fmt_tag, I1(), I1());
  };
  switch (a0.fmt) {
    case FMM_LEAF_BF16: return by_blocks(std::integral_constant<int, FMM_LEAF_BF16>());
    case FMM_LEAF_F16: return by_blocks(std::integral_constant<int, FMM_LEAF_F16>());
    default: return by_blocks(std::integral_constant<int, FMM_LEAF_BF16X3>());
  }
}

cudaError_t launch_combine_pair(const CombineArgs& a0, const CombineArgs& a1, cudaStream_t st) {
  const int sms = device_sms();
  const bool pair = small_ok(a0, sms) && small_ok(a1, sms) && a0.dtype == a1.dtype && a0.fmt == a1.fmt &&
                    a0.n_rb == a1.n_rb && a0.n_cb == a1.n_cb && a0.num_leaves > 0 && a1.num_leaves > 0 &&
                    a0.b_rows <= a0.p_rows && a0.b_cols <= a0.p_cols && a1.b_rows <= a1.p_rows &&
                    a1.b_cols <= a1.p_cols &&
                    (a0.p_cols / kTC) * (a0.p_rows / 32) + (a1.p_cols / kTC) * (a1.p_rows / 32) < 0x7FFFFFFF;
  if (!pair) {
    const cudaError_t e = launch_combine(a0, st);
    return e != cudaSuccess ? e : launch_combine(a1, st);
  }
  KernelTimer timer("combine", st);
#define FMM_PAIR(DT)                                                              \
  switch (a0.fmt) {                                                               \
    case FMM_LEAF_BF16: launch_small_pair<DT, FMM_LEAF_BF16>(a0, a1, st); break;  \
    case FMM_LEAF_F16: launch_small_pair<DT, FMM_LEAF_F16>(a0, a1, st); break;    \
    default: launch_small_pair<DT, FMM_LEAF_BF16X3>(a0, a1, st); break;          \
  }
  switch (a0.dtype) {
    case kF32: FMM_PAIR(kF32) break;
    case kBF16: FMM_PAIR(kBF16) break;
    default: FMM_PAIR(kF16) break;
  }
#undef FMM_PAIR
  return cudaGetLastError();
}

}  // namespace fmm
