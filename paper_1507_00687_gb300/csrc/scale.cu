// Power-of-two diagonal scaling (Sec. 6, Algs. 1-3): row / column max-abs
// reductions done entirely in exponent arithmetic.
//
// For a scaled operand X' = 2^(rs*re_i) X_ij 2^(cs*ce_j) the frexp exponent
// of an entry is e(X_ij) + rs*re_i + cs*ce_j, and the exponent of a row's
// (column's) max-abs is the max of its entries' exponents, because e() is
// monotone in |x|.  So no mantissa is ever multiplied and the scale factors
// are exact by construction.  Both kernels are single passes over the
// matrix, HBM-bound: 4 (fp32) or 2 (bf16/fp16) bytes read per element.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace fmm {

// ---------------------------------------------------------------- decoding

// Four consecutive raw encodings (16 bytes for fp32, 8 for 16-bit types),
// loaded without using them so that several loads can be in flight.
template <int DT>
__device__ __forceinline__ uint4 raw4(const void* base, int64_t idx) {
  if constexpr (DT == kF32) {
    return __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const uint32_t*>(base) + idx));
  } else {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const unsigned short*>(base) + idx));
    return make_uint4(v.x, v.y, 0u, 0u);
  }
}

template <int DT>
__device__ __forceinline__ uint32_t raw1(const void* base, int64_t idx) {
  if constexpr (DT == kF32) return __ldg(reinterpret_cast<const uint32_t*>(base) + idx);
  else return __ldg(reinterpret_cast<const unsigned short*>(base) + idx);
}

// raw4 for columns c .. c + 3 of row offset `row` when some may lie at or
// beyond C: those read as the encoding 0 (a zero, which never raises a
// maximum).  Vector load when all four exist and alignment allows.
template <int DT>
__device__ __forceinline__ uint4 raw4_guarded(const void* base, int64_t row, int64_t c, int64_t C, bool vec) {
  if (vec && c + 4 <= C) return raw4<DT>(base, row + c);
  uint32_t b[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) b[t] = (c + t < C) ? raw1<DT>(base, row + c + t) : 0u;
  if constexpr (DT == kF32) return make_uint4(b[0], b[1], b[2], b[3]);
  else return make_uint4(b[0] | (b[1] << 16), b[2] | (b[3] << 16), 0u, 0u);
}

// The four encodings held in a raw4 result.
template <int DT>
__device__ __forceinline__ void unpack4(uint4 v, uint32_t (&b)[4]) {
  if constexpr (DT == kF32) {
    b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
  } else {
    b[0] = v.x & 0xFFFFu; b[1] = v.x >> 16; b[2] = v.y & 0xFFFFu; b[3] = v.y >> 16;
  }
}

// frexp exponent of one encoding, with the common case (a normal number:
// biased exponent field minus the bias, minus one) inline and zero,
// subnormals and Inf/NaN through the exact decoders.
template <int DT>
__device__ __forceinline__ int fexp_fast(uint32_t bits, bool* nf) {
  if constexpr (DT == kF32) {
    const uint32_t be = (bits >> 23) & 0xFFu;
    if (be - 1u < 254u) return (int)be - 126;
    return fexp_f32(bits, nf);
  } else if constexpr (DT == kBF16) {
    const uint32_t be = (bits >> 7) & 0xFFu;
    if (be - 1u < 254u) return (int)be - 126;
    return fexp_bf16(bits, nf);
  } else {
    const uint32_t be = (bits >> 10) & 0x1Fu;
    if (be - 1u < 30u) return (int)be - 14;
    return fexp_f16(bits, nf);
  }
}

// The biased exponent field of an encoding, minus one (so that a normal
// number gives a value below kNormalSpan), and the frexp exponent of a
// normal number from its field.  Shifted maxima over a group of encodings
// test the whole group once (one branch instead of one per element) and
// send it through fexp_fast only when some member is zero, subnormal or not
// finite.
template <int DT>
__device__ __forceinline__ uint32_t field_m1(uint32_t bits) {
  if constexpr (DT == kF32) return ((bits >> 23) & 0xFFu) - 1u;
  else if constexpr (DT == kBF16) return ((bits >> 7) & 0xFFu) - 1u;
  else return ((bits >> 10) & 0x1Fu) - 1u;
}
template <int DT>
constexpr uint32_t kNormalSpan = DT == kF16 ? 30u : 254u;
template <int DT>
__device__ __forceinline__ int fexp_normal(uint32_t bits) {
  return (int)field_m1<DT>(bits) + (DT == kF16 ? -13 : -125);
}
// The largest field_m1 of the four encodings of a raw4 result.
template <int DT>
__device__ __forceinline__ uint32_t worst4(uint4 v) {
  uint32_t b[4];
  unpack4<DT>(v, b);
  return max(max(field_m1<DT>(b[0]), field_m1<DT>(b[1])), max(field_m1<DT>(b[2]), field_m1<DT>(b[3])));
}

// |x| as an integer: for finite values its order is the order of |x|, so
// the exponent of a max-abs is the exponent of the max of these keys.
template <int DT>
__device__ __forceinline__ uint32_t abs_bits(uint32_t bits) {
  return DT == kF32 ? (bits & 0x7FFFFFFFu) : (bits & 0x7FFFu);
}
template <int DT>
__device__ __forceinline__ int fexp_of_abs_max(uint32_t m, bool* nf) {
  if constexpr (DT == kF32) return fexp_f32(m, nf);
  else if constexpr (DT == kBF16) return fexp_bf16(m, nf);
  else return fexp_f16(m, nf);
}

// Any value at or below this is "no nonzero entry": shifted exponents of
// zeros (kZeroExp + a small shift) stay far below it.
constexpr int kZeroThreshold = kZeroExp / 2;

// ---------------------------------------------------------------- row reduction

// Row reduction.  For each row i of the R x C matrix X:
//   m_i = max_j ( e(X_ij) + cs * ce_j )          (no nonzero entry: zero row)
// mode kRowOStep:  out[i] = m_i, or 0 for a zero row          (O step)
// mode kRowIStep:  out[i] holds e_x (a column max of the other operand, from
//   col_exp_kernel); out[i] = floor((m_i - e_x) / 2), 0 if either is zero
//   (the I-step exponent of Eq. 6.6).
// One warp per row, kRowBatch 16-byte loads in flight per lane, and the row
// maximum a warp shuffle reduction.  Without column shifts (SHIFT false) the
// row max is taken over |x| as integers and decoded once.
constexpr int kRowWarps = 8;
constexpr int kRowBatch = 8;

// Row i, one warp (lane = its lane index).
template <int DT, bool SHIFT, int kRowBatch = kRowBatch, bool kGroup = false>
__device__ __forceinline__ void row_exp_one(const void* X, int64_t C, int64_t ld, const int* ce, int cs, int* out,
                                            int mode, bool vec_ok, int64_t i, int lane, bool* nf) {
  // the vector path also needs the column exponents 16-byte aligned
  const bool vec = vec_ok && (!SHIFT || ((uintptr_t)ce % 16 == 0));
  int m = kZeroExp;       // SHIFT: max shifted exponent
  uint32_t mb = 0;        // !SHIFT: max |x| key
  const int64_t rowoff = i * ld;
  auto take = [&](uint32_t bits, int c) {
    if constexpr (SHIFT) m = max(m, fexp_fast<DT>(bits, nf) + cs * c);
    else mb = max(mb, abs_bits<DT>(bits));
  };
  int64_t jdone = 0;
  if (vec) {
    const int64_t C4 = C >> 2;
    int64_t j4 = lane;
    // kGroup: every batch is issued whole, the positions past the row's end
    // clamped to its last group of four (re-reading an element of the row
    // never changes a maximum), so a row ends without single-load rounds
    for (; kGroup ? j4 < C4 : j4 + 32 * (kRowBatch - 1) < C4; j4 += 32 * kRowBatch) {
      uint4 v[kRowBatch];
      int4 c[kRowBatch];
      int64_t jj[kRowBatch];
#pragma unroll
      for (int u = 0; u < kRowBatch; ++u) jj[u] = kGroup ? min(j4 + 32 * u, C4 - 1) : j4 + 32 * u;
#pragma unroll
      for (int u = 0; u < kRowBatch; ++u) v[u] = raw4<DT>(X, rowoff + 4 * jj[u]);
#pragma unroll
      for (int u = 0; u < kRowBatch; ++u)
        c[u] = SHIFT ? __ldg(reinterpret_cast<const int4*>(ce + 4 * jj[u])) : make_int4(0, 0, 0, 0);
      if constexpr (SHIFT && kGroup) {
        uint32_t worst = 0u;
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) worst = max(worst, worst4<DT>(v[u]));
        if (worst < kNormalSpan<DT>) {
#pragma unroll
          for (int u = 0; u < kRowBatch; ++u) {
            uint32_t b[4];
            unpack4<DT>(v[u], b);
            m = max(m, fexp_normal<DT>(b[0]) + cs * c[u].x);
            m = max(m, fexp_normal<DT>(b[1]) + cs * c[u].y);
            m = max(m, fexp_normal<DT>(b[2]) + cs * c[u].z);
            m = max(m, fexp_normal<DT>(b[3]) + cs * c[u].w);
          }
        } else {
#pragma unroll
          for (int u = 0; u < kRowBatch; ++u) {
            uint32_t b[4];
            unpack4<DT>(v[u], b);
            take(b[0], c[u].x); take(b[1], c[u].y); take(b[2], c[u].z); take(b[3], c[u].w);
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) {
          uint32_t b[4];
          unpack4<DT>(v[u], b);
          take(b[0], c[u].x); take(b[1], c[u].y); take(b[2], c[u].z); take(b[3], c[u].w);
        }
      }
    }
    for (; j4 < C4; j4 += 32) {
      const uint4 v = raw4<DT>(X, rowoff + 4 * j4);
      const int4 c = SHIFT ? __ldg(reinterpret_cast<const int4*>(ce + 4 * j4)) : make_int4(0, 0, 0, 0);
      uint32_t b[4];
      unpack4<DT>(v, b);
      take(b[0], c.x); take(b[1], c.y); take(b[2], c.z); take(b[3], c.w);
    }
    jdone = 4 * C4;
  }
  for (int64_t j = jdone + lane; j < C; j += 32) take(raw1<DT>(X, rowoff + j), SHIFT ? __ldg(ce + j) : 0);
  if constexpr (!SHIFT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    m = fexp_of_abs_max<DT>(mb, nf);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if (lane == 0) {
    const bool zero = m <= kZeroThreshold;
    if (mode == kRowOStep) {
      out[i] = zero ? 0 : m;
    } else {
      const int ex = out[i];
      out[i] = (zero || ex <= kZeroThreshold) ? 0 : ((m - ex) >> 1);  // arithmetic shift = floor
    }
  }
}

template <int DT, bool SHIFT>
__global__ void __launch_bounds__(kRowWarps * 32) row_exp_kernel(const void* X, int64_t R, int64_t C, int64_t ld,
                                                                 const int* ce, int cs, int* out, int mode,
                                                                 int vec_ok, int* status, const int* skip) {
  if (skip && *skip) return;  // an adaptive iteration that has stopped
  bool nf = false;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * kRowWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kRowWarps;
  for (int64_t i = w0; i < R; i += nw) row_exp_one<DT, SHIFT>(X, C, ld, ce, cs, out, mode, vec_ok != 0, i, lane, &nf);
  if (nf) atomicOr(status, kStatusNonfinite);
}

// Batched row reduction: warp w of the launch takes global row w; rows of
// problem p are [start[p], start[p + 1]).
template <int DT, bool SHIFT>
__global__ void __launch_bounds__(kRowWarps * 32) row_exp_batched_kernel(const ReduceArgs* args,
                                                                         const int64_t* start, int count, int mode,
                                                                         int* status) {
  bool nf = false;
  const int64_t g = (int64_t)blockIdx.x * kRowWarps + (threadIdx.x >> 5);
  if (g >= __ldg(start + count)) return;
  const int p = warp_find_problem(start, count, g);
  const ReduceArgs a = args[p];
  row_exp_one<DT, SHIFT, kRowBatch, true>(a.X, a.C, a.ld, a.shift, a.sign, a.out, mode, a.vec != 0,
                                          g - __ldg(start + p), threadIdx.x & 31, &nf);
  if (nf) atomicOr(status, kStatusNonfinite);
}

// ---------------------------------------------------------------- column reduction

// Column reduction: out[j] = max(out[j], max_i (e(X_ij) + rs * re_i)) over
// a chunk of rows per CTA (out pre-filled with kZeroExp; nothing is written
// for a column with no nonzero entry in the chunk).  A CTA covers a span of
// kColSpan columns with kColGroups groups of 256 threads, each group
// streaming whole rows of its share of the chunk (4 elements x kColVec per
// thread per row: 16-byte loads for fp32, 8-byte for 16-bit types, so DRAM
// sees long contiguous runs) with kColRows rows' loads in flight; the
// groups' maxima meet in shared memory, so one
// atomicMax per column covers the CTA's rows.  Without row shifts (SHIFT
// false) the maximum is taken over |x| as integers and decoded once.
constexpr int kColVec = 2;
constexpr int kColSpan = 256 * 4 * kColVec;  // 2048 columns
// rows of loads in flight per thread: 4 for 16-bit types (8-byte loads), 2
// for fp32
template <int DT>
constexpr int kColRows = DT == kF32 ? 2 : 4;
constexpr int kColGroups = 4;
constexpr int kColThreads = 256 * kColGroups;
constexpr int kColSmem = kColGroups * kColSpan * 4;

// One CTA of the column reduction: column span bx, row chunk by.
template <int DT, bool SHIFT>
__device__ __forceinline__ void col_exp_cta(const void* X, int64_t R, int64_t C, int64_t ld, const int* re, int rs,
                                            int* out, int rows_per_cta, bool vec, int64_t bx, int64_t by, int* red,
                                            bool* nf) {
  const int group = threadIdx.x >> 8, lt = threadIdx.x & 255;
  const int64_t span0 = bx * kColSpan;
  const int rows_g = rows_per_cta / kColGroups;
  const int64_t r0 = by * rows_per_cta + (int64_t)group * rows_g;
  const int64_t r1 = min(R, r0 + rows_g);
  int m[kColVec][4];
  uint32_t mb[kColVec][4];
#pragma unroll
  for (int q = 0; q < kColVec; ++q)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      m[q][t] = kZeroExp;
      mb[q][t] = 0u;
    }
  auto take = [&](int q, int t, uint32_t bits, int sh) {
    if constexpr (SHIFT) m[q][t] = max(m[q][t], fexp_fast<DT>(bits, nf) + sh);
    else mb[q][t] = max(mb[q][t], abs_bits<DT>(bits));
  };
  // column of (q, t): span0 + 1024 q + 4 lt + t
  const int64_t cbase = span0 + 4 * (int64_t)lt;
  int64_t i = r0;
  for (; i + kColRows<DT> <= r1; i += kColRows<DT>) {
    uint4 v[kColRows<DT>][kColVec];
    int sh[kColRows<DT>];
#pragma unroll
    for (int u = 0; u < kColRows<DT>; ++u)
#pragma unroll
      for (int q = 0; q < kColVec; ++q) v[u][q] = raw4_guarded<DT>(X, (i + u) * ld, cbase + 1024 * q, C, vec);
#pragma unroll
    for (int u = 0; u < kColRows<DT>; ++u) sh[u] = SHIFT ? rs * __ldg(re + i + u) : 0;
#pragma unroll
    for (int u = 0; u < kColRows<DT>; ++u)
#pragma unroll
      for (int q = 0; q < kColVec; ++q) {
        uint32_t b[4];
        unpack4<DT>(v[u][q], b);
#pragma unroll
        for (int t = 0; t < 4; ++t) take(q, t, b[t], sh[u]);
      }
  }
  for (; i < r1; ++i) {
    const int sh = SHIFT ? rs * __ldg(re + i) : 0;
#pragma unroll
    for (int q = 0; q < kColVec; ++q) {
      uint32_t b[4];
      unpack4<DT>(raw4_guarded<DT>(X, i * ld, cbase + 1024 * q, C, vec), b);
#pragma unroll
      for (int t = 0; t < 4; ++t) take(q, t, b[t], sh);
    }
  }
#pragma unroll
  for (int q = 0; q < kColVec; ++q)
#pragma unroll
    for (int t = 0; t < 4; ++t)
      red[group * kColSpan + 1024 * q + 4 * lt + t] = SHIFT ? m[q][t] : fexp_of_abs_max<DT>(mb[q][t], nf);
  __syncthreads();
  for (int c = threadIdx.x; c < kColSpan; c += kColThreads) {
    int e = red[c];
#pragma unroll
    for (int g = 1; g < kColGroups; ++g) e = max(e, red[g * kColSpan + c]);
    if (span0 + c < C && e > kZeroThreshold) atomicMax(out + span0 + c, e);
  }
}

template <int DT, bool SHIFT>
__global__ void __launch_bounds__(kColThreads) col_exp_kernel(const void* X, int64_t R, int64_t C, int64_t ld,
                                                              const int* re, int rs, int* out, int rows_per_cta,
                                                              int vec_ok, int* status, const int* skip) {
  if (skip && *skip) return;  // an adaptive iteration that has stopped
  extern __shared__ int red[];  // [kColGroups][kColSpan]
  bool nf = false;
  col_exp_cta<DT, SHIFT>(X, R, C, ld, re, rs, out, rows_per_cta, vec_ok != 0, blockIdx.x, blockIdx.y, red, &nf);
  if (nf) atomicOr(status, kStatusNonfinite);
}

// Batched column reduction: CTA b of the launch belongs to the problem whose
// [start[p], start[p + 1]) holds b; within it, CTAs run over
// (column span, row chunk) with args[p].gx spans.
template <int DT, bool SHIFT>
__global__ void __launch_bounds__(kColThreads) col_exp_batched_kernel(const ReduceArgs* args, const int64_t* start,
                                                                      int count, int* status) {
  extern __shared__ int red[];
  bool nf = false;
  const int p = warp_find_problem(start, count, blockIdx.x);
  const ReduceArgs a = args[p];
  const int64_t local = blockIdx.x - __ldg(start + p);
  col_exp_cta<DT, SHIFT>(a.X, a.R, a.C, a.ld, a.shift, a.sign, a.out, a.rows_per_cta, a.vec != 0, local % a.gx,
                         local / a.gx, red, &nf);
  if (nf) atomicOr(status, kStatusNonfinite);
}

// ---------------------------------------------------------------- fused O-then-I from no scaling
//
// The step pair O, I of Alg. 3 on unscaled operands, in two launches with
// no atomics and no initialisation of the outputs:
//   oi_outside_kernel: CTAs [0, row_ctas) take rows of A, a warp per row
//     (eA_i = e(max_k |A_ik|)); the others take 32-column panels of B over
//     all K rows (eB_j = e(max_k |B_kj|)), the row groups meeting in shared
//     memory.
//   oi_inside_kernel: CTA p takes k in [16 p, 16 p + 16): the column maxima
//     e(max_i 2^-eA_i |A_ik|) over all M rows of A, then the row maxima
//     e(max_j |B_kj| 2^-eB_j) over all N columns of B, then d_k (Eq. 6.6).
// The same exponents as the four separate reductions; each operand is read
// twice, the second time mostly from L2.
constexpr int kOIThreads = 512;
constexpr int kOIBatch = 8;  // rows of loads in flight per thread

// Running maxima of columns c0 + 4 tq .. + 3 (tq = thread mod P/4) over the
// rows tr, tr + G, ... (tr = thread / (P/4), G = 512 / (P/4)) of the R x C
// matrix X; with SHIFT each row's entries are shifted by -re[row].
template <int DT, bool SHIFT, int P, int kOIBatch = kOIBatch>
__device__ __forceinline__ void panel_max(const void* X, int64_t R, int64_t C, int64_t ld, int64_t c0, const int* re,
                                          bool vec, int (&m)[4], uint32_t (&mb)[4], bool* nf) {
  constexpr int kTq = P / 4, kG = kOIThreads / kTq;
  const int tq = threadIdx.x % kTq, tr = threadIdx.x / kTq;
  const int64_t c = c0 + 4 * tq;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    m[t] = kZeroExp;
    mb[t] = 0u;
  }
  auto take = [&](uint4 v, int sh) {
    uint32_t b[4];
    unpack4<DT>(v, b);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if constexpr (SHIFT) m[t] = max(m[t], fexp_fast<DT>(b[t], nf) + sh);
      else mb[t] = max(mb[t], abs_bits<DT>(b[t]));
    }
  };
  int64_t i = tr;
  for (; i + (int64_t)kG * (kOIBatch - 1) < R; i += (int64_t)kG * kOIBatch) {
    uint4 v[kOIBatch];
    int sh[kOIBatch];
#pragma unroll
    for (int u = 0; u < kOIBatch; ++u) v[u] = raw4_guarded<DT>(X, (i + (int64_t)kG * u) * ld, c, C, vec);
#pragma unroll
    for (int u = 0; u < kOIBatch; ++u) sh[u] = SHIFT ? -__ldg(re + i + (int64_t)kG * u) : 0;
#pragma unroll
    for (int u = 0; u < kOIBatch; ++u) take(v[u], sh[u]);
  }
  for (; i < R; i += kG) take(raw4_guarded<DT>(X, i * ld, c, C, vec), SHIFT ? -__ldg(re + i) : 0);
}

// Combine the per-thread maxima of panel_max over the row groups: returns,
// for threads 0 .. P-1, the maximum of column c0 + threadIdx.x (as an
// unshifted |x| key decoded to an exponent, or as a shifted exponent).
template <int DT, bool SHIFT, int P>
__device__ __forceinline__ int panel_reduce(const int (&m)[4], const uint32_t (&mb)[4], int* red, bool* nf) {
  constexpr int kTq = P / 4, kG = kOIThreads / kTq;
  const int tq = threadIdx.x % kTq, tr = threadIdx.x / kTq;
#pragma unroll
  for (int t = 0; t < 4; ++t) red[tr * P + 4 * tq + t] = SHIFT ? m[t] : (int)mb[t];
  __syncthreads();
  int e = kZeroExp;
  if (threadIdx.x < P) {
    if constexpr (SHIFT) {
      for (int g = 0; g < kG; ++g) e = max(e, red[g * P + threadIdx.x]);
    } else {
      uint32_t k = 0;
      for (int g = 0; g < kG; ++g) k = max(k, (uint32_t)red[g * P + threadIdx.x]);
      e = fexp_of_abs_max<DT>(k, nf);
    }
  }
  return e;
}

constexpr int kOIPanelB = 32;  // columns of B per panel CTA of the O step
constexpr int kOIPanelK = 16;  // k per CTA of the I step

template <int DT>
__global__ void __launch_bounds__(kOIThreads) oi_outside_kernel(const void* A, const void* B, int64_t M, int64_t K,
                                                                int64_t N, int64_t lda, int64_t ldb, int* eA, int* eB,
                                                                int row_ctas, int vec_a, int vec_b, int* status) {
  __shared__ int red[(kOIThreads / (kOIPanelB / 4)) * kOIPanelB];
  pdl_wait();
  pdl_trigger();
  bool nf = false;
  if ((int)blockIdx.x < row_ctas) {
    constexpr int kWarps = kOIThreads / 32;
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); i < M; i += (int64_t)row_ctas * kWarps)
      row_exp_one<DT, false>(A, K, lda, nullptr, 0, eA, kRowOStep, vec_a != 0, i, lane, &nf);
  } else {
    const int64_t c0 = (int64_t)(blockIdx.x - row_ctas) * kOIPanelB;
    int m[4];
    uint32_t mb[4];
    panel_max<DT, false, kOIPanelB>(B, K, N, ldb, c0, nullptr, vec_b != 0, m, mb, &nf);
    const int e = panel_reduce<DT, false, kOIPanelB>(m, mb, red, &nf);
    if (threadIdx.x < kOIPanelB && c0 + threadIdx.x < N) eB[c0 + threadIdx.x] = e <= kZeroThreshold ? 0 : e;
  }
  if (nf) atomicOr(status, kStatusNonfinite);
}

template <int DT>
__global__ void __launch_bounds__(kOIThreads, 2) oi_inside_kernel(const void* A, const void* B, int64_t M, int64_t K,
                                                               int64_t N, int64_t lda, int64_t ldb, const int* eA,
                                                               const int* eB, int* d, int vec_a, int vec_b,
                                                               int* status) {
  __shared__ int red[(kOIThreads / (kOIPanelK / 4)) * kOIPanelK];
  pdl_wait();
  pdl_trigger();
  bool nf = false;
  const int64_t k0 = (int64_t)blockIdx.x * kOIPanelK;
  // e(max_i 2^-eA_i |A_ik|) for the CTA's k, parked in d until the row pass
  int m[4];
  uint32_t mb[4];
  panel_max<DT, true, kOIPanelK>(A, M, K, lda, k0, eA, vec_a != 0, m, mb, &nf);
  const int ea = panel_reduce<DT, true, kOIPanelK>(m, mb, red, &nf);
  if (threadIdx.x < kOIPanelK && k0 + threadIdx.x < K) d[k0 + threadIdx.x] = ea;
  __syncthreads();
  // d_k = floor((e(max_j |B_kj| 2^-eB_j) - e_A) / 2): a warp per row of B
  constexpr int kWarps = kOIThreads / 32;
  const int lane = threadIdx.x & 31;
  for (int64_t k = k0 + (threadIdx.x >> 5); k < min(K, k0 + kOIPanelK); k += kWarps)
    row_exp_one<DT, true, 4>(B, N, ldb, eB, -1, d, kRowIStep, vec_b != 0, k, lane, &nf);
  if (nf) atomicOr(status, kStatusNonfinite);
}

// Operand preparation (the apply pass of Algs. 1-3, plus blocking): each
// thread writes 4 consecutive output columns of one output row (row_pad and
// col_pad are multiples of 4, so a group never straddles two blocks), reading
// the matching source elements (zero outside the source) and scaling them by
// 2^(rs re[row] + cs ce[col]).  One HBM-bound pass.
template <int DT, bool OUT_BF16>
__global__ void __launch_bounds__(256) prepare_kernel(const void* X, int64_t R, int64_t C, int64_t ld,
                                                      int64_t row_blk, int64_t row_pad, int64_t col_blk,
                                                      int64_t col_pad, const int* re, int rs, const int* ce, int cs,
                                                      void* Y, int64_t Rp, int64_t Cp, int64_t ldy) {
  const int64_t C4 = Cp / 4;
  const int64_t total = Rp * C4;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rp = idx / C4, cp0 = (idx % C4) * 4;
    const int64_t rb = rp / row_pad, rr = rp % row_pad;
    const int64_t src_r = rb * row_blk + rr;
    const bool row_ok = rr < row_blk && src_r < R;
    const int er = (row_ok && re) ? rs * __ldg(re + src_r) : 0;
    float y[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t cp = cp0 + t, cb = cp / col_pad, cc = cp % col_pad;
      const int64_t src_c = cb * col_blk + cc;
      float x = 0.f;
      if (row_ok && cc < col_blk && src_c < C) {
        const int64_t i = src_r * ld + src_c;
        if constexpr (DT == kF32) x = __ldg(reinterpret_cast<const float*>(X) + i);
        else if constexpr (DT == kBF16)
          x = __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(X) + i) << 16);
        else x = __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(X) + i)));
        x = scale_pow2(x, er + (ce ? cs * __ldg(ce + src_c) : 0));
      }
      y[t] = x;
    }
    if constexpr (OUT_BF16) {
      // exact: a power-of-two multiple of a bf16 value in range is a bf16 value
      const uint32_t b0 = __float_as_uint(y[0]) >> 16, b1 = __float_as_uint(y[1]) >> 16;
      const uint32_t b2 = __float_as_uint(y[2]) >> 16, b3 = __float_as_uint(y[3]) >> 16;
      *reinterpret_cast<uint2*>(reinterpret_cast<unsigned short*>(Y) + rp * ldy + cp0) =
          make_uint2(b0 | (b1 << 16), b2 | (b3 << 16));
    } else {
      *reinterpret_cast<float4*>(reinterpret_cast<float*>(Y) + rp * ldy + cp0) = make_float4(y[0], y[1], y[2], y[3]);
    }
  }
}

__global__ void fill_kernel(int* p, int64_t n, int v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// kZeroExp (an all-zero column) -> 0.
__global__ void zero_sentinel_kernel(int* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (p[i] == kZeroExp) p[i] = 0;
}

static int esize(int dt) { return dt == kF32 ? 4 : 2; }

static bool vec_aligned(const void* X, int64_t ld, int dt) {
  return ((uintptr_t)X % 16 == 0) && ((ld * esize(dt)) % 16 == 0);
}

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 132;
  }
  return n;
}

cudaError_t launch_row_exp(const void* X, int dt, int64_t R, int64_t C, int64_t ld, const int* ce, int cs,
                           int* out, int mode, int* status, cudaStream_t st, const int* skip) {
  if (R == 0) return cudaSuccess;
  const int vec = vec_aligned(X, ld, dt) ? 1 : 0;
  const int64_t grid = std::min<int64_t>((R + kRowWarps - 1) / kRowWarps, (int64_t)sm_count() * 8);
  dim3 g((unsigned)grid);
  const int nt = kRowWarps * 32;
  KernelTimer timer("scale", st);
  switch (dt) {
#define FMM_ROW(DT)                                                                              \
  (ce ? row_exp_kernel<DT, true><<<g, nt, 0, st>>>(X, R, C, ld, ce, cs, out, mode, vec, status, skip)   \
      : row_exp_kernel<DT, false><<<g, nt, 0, st>>>(X, R, C, ld, ce, cs, out, mode, vec, status, skip))
    case kF32: FMM_ROW(kF32); break;
    case kBF16: FMM_ROW(kBF16); break;
    default: FMM_ROW(kF16); break;
#undef FMM_ROW
  }
  return cudaGetLastError();
}

cudaError_t launch_col_exp(const void* X, int dt, int64_t R, int64_t C, int64_t ld, const int* re, int rs,
                           int* out, int* status, cudaStream_t st, const int* skip) {
  if (C == 0) return cudaSuccess;
  {
    KernelTimer fill_timer("scale", st);
    fill_kernel<<<(unsigned)std::min<int64_t>((C + 255) / 256, 4096), 256, 0, st>>>(out, C, kZeroExp);
  }
  if (R == 0) return cudaGetLastError();
  const int vec = vec_aligned(X, ld, dt) ? 1 : 0;
  const int64_t gx = (C + kColSpan - 1) / kColSpan;
  // about one CTA per SM in all; each group's rows a multiple of the batch
  const int64_t target = (int64_t)sm_count();
  const int64_t unit = (int64_t)kColRows<kBF16> * kColGroups;  // a multiple of every type's batch
  int64_t gy = std::max<int64_t>(1, std::min<int64_t>((target + gx - 1) / gx, (R + unit - 1) / unit));
  gy = std::min<int64_t>(gy, 65535);
  const int rows = (int)(((R + gy - 1) / gy + unit - 1) / unit * unit);
  gy = (R + rows - 1) / rows;
  dim3 g((unsigned)gx, (unsigned)gy);
  static bool attr_done[64][6] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  KernelTimer timer("scale", st);
  switch (dt) {
#define FMM_COL(DT, I)                                                                                       \
  if (!attr_done[dev][2 * I]) {                                                                             \
    cudaFuncSetAttribute(col_exp_kernel<DT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kColSmem);   \
    cudaFuncSetAttribute(col_exp_kernel<DT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kColSmem);  \
    attr_done[dev][2 * I] = true;                                                                           \
  }                                                                                                          \
  if (re) col_exp_kernel<DT, true><<<g, kColThreads, kColSmem, st>>>(X, R, C, ld, re, rs, out, rows, vec, status,  \
                                                                     skip);                                    \
  else col_exp_kernel<DT, false><<<g, kColThreads, kColSmem, st>>>(X, R, C, ld, re, rs, out, rows, vec, status, skip);
    case kF32: { FMM_COL(kF32, 0) break; }
    case kBF16: { FMM_COL(kBF16, 1) break; }
    default: { FMM_COL(kF16, 2) break; }
#undef FMM_COL
  }
  return cudaGetLastError();
}

cudaError_t launch_row_exp_batched(const ReduceArgs* args, const int64_t* start, int count, int64_t total, int dt,
                                   bool shift, int mode, int* status, cudaStream_t st) {
  if (total == 0 || count == 0) return cudaSuccess;
  const unsigned g = (unsigned)((total + kRowWarps - 1) / kRowWarps);
  const int nt = kRowWarps * 32;
  KernelTimer timer("scale", st);
#define FMM_ROWB(DT)                                                                                   \
  (shift ? row_exp_batched_kernel<DT, true><<<g, nt, 0, st>>>(args, start, count, mode, status)        \
         : row_exp_batched_kernel<DT, false><<<g, nt, 0, st>>>(args, start, count, mode, status))
  switch (dt) {
    case kF32: FMM_ROWB(kF32); break;
    case kBF16: FMM_ROWB(kBF16); break;
    default: FMM_ROWB(kF16); break;
  }
#undef FMM_ROWB
  return cudaGetLastError();
}

cudaError_t launch_col_exp_batched(const ReduceArgs* args, const int64_t* start, int count, int64_t total, int dt,
                                   bool shift, int* status, cudaStream_t st) {
  static_assert(kBatchColRows % (kColRows<kBF16> * kColGroups) == 0, "row chunk must be whole batches");
  static_assert(kBatchColSpan == kColSpan, "column span");
  if (total == 0 || count == 0) return cudaSuccess;
  static bool attr_done[64][6] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  KernelTimer timer("scale", st);
  const unsigned g = (unsigned)total;
#define FMM_COLB(DT, I)                                                                                          \
  if (!attr_done[dev][I]) {                                                                                      \
    cudaFuncSetAttribute(col_exp_batched_kernel<DT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kColSmem); \
    cudaFuncSetAttribute(col_exp_batched_kernel<DT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                         kColSmem);                                                                              \
    attr_done[dev][I] = true;                                                                                    \
  }                                                                                                              \
  if (shift) col_exp_batched_kernel<DT, true><<<g, kColThreads, kColSmem, st>>>(args, start, count, status);   \
  else col_exp_batched_kernel<DT, false><<<g, kColThreads, kColSmem, st>>>(args, start, count, status);
  switch (dt) {
    case kF32: { FMM_COLB(kF32, 0) break; }
    case kBF16: { FMM_COLB(kBF16, 1) break; }
    default: { FMM_COLB(kF16, 2) break; }
  }
#undef FMM_COLB
  return cudaGetLastError();
}

cudaError_t launch_oi_from_zero(const void* A, const void* B, int dt, int64_t M, int64_t K, int64_t N, int64_t lda,
                                int64_t ldb, int* eA, int* d, int* eB, int* status, cudaStream_t st) {
  if (M == 0 || K == 0 || N == 0) return cudaErrorInvalidValue;
  const int vec_a = vec_aligned(A, lda, dt) ? 1 : 0, vec_b = vec_aligned(B, ldb, dt) ? 1 : 0;
  const int64_t row_ctas = std::min<int64_t>((M + 15) / 16, (int64_t)sm_count() * 4);
  const int64_t panels = (N + kOIPanelB - 1) / kOIPanelB;
  const int64_t kctas = (K + kOIPanelK - 1) / kOIPanelK;
  if (row_ctas + panels > 0x7FFFFFFF || kctas > 0x7FFFFFFF) return cudaErrorInvalidValue;
  {
    KernelTimer timer("scale", st);
    switch (dt) {
      case kF32:
        launch_pdl(oi_outside_kernel<kF32>, dim3((unsigned)(row_ctas + panels)), dim3(kOIThreads), 0, st, A, B, M, K, N, lda, ldb, eA, eB, (int)row_ctas, vec_a, vec_b, status);
        break;
      case kBF16:
        launch_pdl(oi_outside_kernel<kBF16>, dim3((unsigned)(row_ctas + panels)), dim3(kOIThreads), 0, st, A, B, M, K, N, lda, ldb, eA, eB, (int)row_ctas, vec_a, vec_b, status);
        break;
      default:
        launch_pdl(oi_outside_kernel<kF16>, dim3((unsigned)(row_ctas + panels)), dim3(kOIThreads), 0, st, A, B, M, K, N, lda, ldb, eA, eB, (int)row_ctas, vec_a, vec_b, status);
        break;
    }
  }
  KernelTimer timer("scale", st);
  switch (dt) {
    case kF32:
      launch_pdl(oi_inside_kernel<kF32>, dim3((unsigned)kctas), dim3(kOIThreads), 0, st, A, B, M, K, N, lda, ldb, (const int*)eA, (const int*)eB, d, vec_a, vec_b, status);
      break;
    case kBF16:
      launch_pdl(oi_inside_kernel<kBF16>, dim3((unsigned)kctas), dim3(kOIThreads), 0, st, A, B, M, K, N, lda, ldb, (const int*)eA, (const int*)eB, d, vec_a, vec_b, status);
      break;
    default:
      launch_pdl(oi_inside_kernel<kF16>, dim3((unsigned)kctas), dim3(kOIThreads), 0, st, A, B, M, K, N, lda, ldb, (const int*)eA, (const int*)eB, d, vec_a, vec_b, status);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_zero_sentinel(int* p, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  KernelTimer timer("scale", st);
  zero_sentinel_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(p, n);
  return cudaGetLastError();
}

cudaError_t launch_prepare(const void* X, int dt, int64_t R, int64_t C, int64_t ld, int64_t row_blk,
                           int64_t row_pad, int64_t col_blk, int64_t col_pad, const int* re, int rs, const int* ce,
                           int cs, void* Y, int64_t Rp, int64_t Cp, int64_t ldy, cudaStream_t st) {
  if (Rp == 0 || Cp == 0) return cudaSuccess;
  const int64_t total = Rp * (Cp / 4);
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count() * 16);
  KernelTimer timer("prepare", st);
  switch (dt) {
    case kF32:
      prepare_kernel<kF32, false><<<grid, 256, 0, st>>>(X, R, C, ld, row_blk, row_pad, col_blk, col_pad, re, rs, ce,
                                                         cs, Y, Rp, Cp, ldy);
      break;
    case kBF16:
      prepare_kernel<kBF16, true><<<grid, 256, 0, st>>>(X, R, C, ld, row_blk, row_pad, col_blk, col_pad, re, rs, ce,
                                                         cs, Y, Rp, Cp, ldy);
      break;
    default:
      prepare_kernel<kF16, false><<<grid, 256, 0, st>>>(X, R, C, ld, row_blk, row_pad, col_blk, col_pad, re, rs, ce,
                                                         cs, Y, Rp, Cp, ldy);
      break;
  }
  return cudaGetLastError();
}

// Adaptive Alg. 3 (Sec. 6.3).  ctl[0]: stopped; ctl[1]: some factor of the
// current step failed its test; ctl[2]: steps applied.  One step's accept
// pass compares the exponents the step computed (next) with the current
// ones (cur): the step's factor is 2^(next - cur), tested against
// [lo, hi]; then cur <- next.  Nothing happens once stopped.
__global__ void scale_accept_kernel(const int* next, int* cur, int64_t n, int lo, int hi, int* ctl) {
  if (*(volatile int*)ctl) return;
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int g = next[i] - cur[i];
    bad |= g < lo || g > hi;
    cur[i] = next[i];
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(ctl + 1, 1);
}

// After step t: count it, and stop if it was tested and passed.
__global__ void scale_stop_kernel(int* ctl, int tested, int t, int* steps_out) {
  if (ctl[0] == 0) {
    ctl[2] = t;
    if (tested && ctl[1] == 0) ctl[0] = 1;
  }
  ctl[1] = 0;
  if (steps_out) *steps_out = ctl[2];
}

cudaError_t launch_scale_accept(const int* next, int* cur, int64_t n, int lo, int hi, int* ctl, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  KernelTimer timer("scale", st);
  scale_accept_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(next, cur, n, lo, hi, ctl);
  return cudaGetLastError();
}

cudaError_t launch_scale_stop(int* ctl, int tested, int t, int* steps_out, cudaStream_t st) {
  KernelTimer timer("scale", st);
  scale_stop_kernel<<<1, 1, 0, st>>>(ctl, tested, t, steps_out);
  return cudaGetLastError();
}

// Block max-abs for the matrix-dependent variant selection: CTA (p, c)
// takes up to kBlockMaxRows rows of block row p; for each column block q its
// threads stride the block's columns (coalesced), a warp reduction and one
// shared-memory atomic per warp combine them, and one global atomic per
// (CTA, q) writes the result.  Non-negative floats order like their bits.
constexpr int kBlockMaxRows = 32;

__global__ void __launch_bounds__(256) block_max_kernel(const void* X, int dt, int64_t R, int64_t C, int64_t ld,
                                                        int64_t br, int64_t bc, int ncb, float* out, int* status) {
  __shared__ unsigned smax[64];
  if (threadIdx.x < 64) smax[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t p = blockIdx.x;
  const int64_t r0 = p * br + (int64_t)blockIdx.y * kBlockMaxRows;
  const int64_t r1 = min(min(r0 + kBlockMaxRows, (p + 1) * br), R);
  bool nonfinite = false;
  const int lane = threadIdx.x & 31;
  for (int q = 0; q < ncb; ++q) {
    const int64_t c0 = (int64_t)q * bc, c1 = min(c0 + bc, C);
    unsigned m = 0u;
    for (int64_t r = r0; r < r1; ++r)
      for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        float x;
        if (dt == kF32) x = static_cast<const float*>(X)[r * ld + c];
        else {
          const uint16_t h = static_cast<const uint16_t*>(X)[r * ld + c];
          x = dt == kBF16 ? __uint_as_float((uint32_t)h << 16) : __half2float(__ushort_as_half(h));
        }
        const unsigned b = __float_as_uint(x) & 0x7FFFFFFFu;
        if (b >= 0x7F800000u) nonfinite = true;
        else m = max(m, b);
      }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && m) atomicMax(&smax[q], m);
  }
  if (nonfinite) atomicOr(status, kStatusNonfinite);
  __syncthreads();
  if (threadIdx.x < ncb && smax[threadIdx.x])
    atomicMax(reinterpret_cast<unsigned*>(out) + p * ncb + threadIdx.x, smax[threadIdx.x]);
}

cudaError_t launch_block_max(const void* X, int dt, int64_t R, int64_t C, int64_t ld, int nrb, int ncb, float* out,
                             int* status, cudaStream_t st) {
  cudaError_t e = launch_fill(reinterpret_cast<int*>(out), (int64_t)nrb * ncb, 0, st);
  if (e != cudaSuccess || R == 0 || C == 0) return e;
  const int64_t br = (R + nrb - 1) / nrb, bc = (C + ncb - 1) / ncb;
  const int64_t chunks = (br + kBlockMaxRows - 1) / kBlockMaxRows;
  if (chunks > 65535) return cudaErrorInvalidValue;
  KernelTimer timer("scale", st);
  block_max_kernel<<<dim3((unsigned)nrb, (unsigned)chunks), 256, 0, st>>>(X, dt, R, C, ld, br, bc, ncb, out, status);
  return cudaGetLastError();
}

cudaError_t launch_fill(int* p, int64_t n, int v, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  KernelTimer timer("scale", st);
  fill_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

}  // namespace fmm
