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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/fmm.h"
#include "device.cuh"
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

template <int DT, int FMT>
__global__ void __launch_bounds__(kThreads) combine_kernel(const CombineArgs a) {
  const int64_t r0 = (int64_t)blockIdx.y * kTR, c0 = (int64_t)blockIdx.x * kTC;
  const int tid = threadIdx.x;
  const int tr = tid >> 4, tc = (tid & 15) * 4;  // rows tr, tr + 16; columns tc .. tc + 3
  const int64_t R = a.num_leaves;
  const int es = DT == kF32 ? 4 : 2;
  const bool vec_ok = ((uintptr_t)a.src % (4 * es) == 0) && (a.ld % 4 == 0) && (a.b_cols % 4 == 0);
  unsigned short* out = static_cast<unsigned short*>(a.out);
  const int64_t plane = R * a.p_rows * a.p_cols;
  for (int64_t r = 0; r < R; ++r) {
    const LeafDesc* L = a.leaves + r;
    const int n = a.side == 0 ? __ldg(&L->na) : __ldg(&L->nb);
    float acc[kRowsPerThread][4];
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int t = 0; t < n; ++t) {
      const int32_t blk = a.side == 0 ? __ldg(&L->a_blk[t]) : __ldg(&L->b_blk[t]);
      const float coef = a.side == 0 ? __ldg(&L->a_coef[t]) : __ldg(&L->b_coef[t]);
      const int64_t bt = (blk >> a.blk_t_shift) & 0xFFFF, bk = (blk >> a.blk_k_shift) & 0xFFFF;
      const int64_t rb = a.t_rows ? bt : bk, cb = a.t_rows ? bk : bt;
      // rows / columns of this block that exist in the source
      const int64_t nr = min(a.b_rows, a.rows - rb * a.b_rows), nc = min(a.b_cols, a.cols - cb * a.b_cols);
      const int64_t grow0 = rb * a.b_rows, gcol0 = cb * a.b_cols;
      const bool interior = vec_ok && r0 + kTR <= nr && c0 + kTC <= nc;
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i) {
        const int64_t lr = r0 + tr + 16 * i, lc = c0 + tc;
        float x[4];
        if (interior) {
          const int64_t gr = grow0 + lr, gc = gcol0 + lc;
          load4<DT>(a.src, gr * a.ld + gc, x);
          if (a.re || a.ce) {
            const int er = a.re ? a.rs * __ldg(a.re + gr) : 0;
            int ec[4] = {0, 0, 0, 0};
            if (a.ce) {
#pragma unroll
              for (int j = 0; j < 4; ++j) ec[j] = a.cs * __ldg(a.ce + gc + j);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = scale_pow2(x[j], er + ec[j]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            x[j] = 0.f;
            if (lr < nr && lc + j < nc) {
              const int64_t gr = grow0 + lr, gc = gcol0 + lc + j;
              const float v = load_elem<DT>(a.src, gr * a.ld + gc);
              const int e = (a.re ? a.rs * __ldg(a.re + gr) : 0) + (a.ce ? a.cs * __ldg(a.ce + gc) : 0);
              x[j] = scale_pow2(v, e);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(coef, x[j], acc[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i) {
      const int64_t off = (r * a.p_rows + r0 + tr + 16 * i) * a.p_cols + c0 + tc;
      store4<FMT>(out + off, out + off + plane, acc[i]);
    }
  }
}

// Staged form for plans with few input blocks (at most kMaxStaged): every
// input block's TR x 64 tile is loaded and scaled once into shared memory
// (in block order), then each leaf's terms are summed from there in term
// order -- the same arithmetic as above with each element scaled once
// instead of once per use.  TR * 16 threads, one row of 4 columns each.
constexpr int kMaxStaged = 16;

template <int DT, int FMT, int TR>
__global__ void __launch_bounds__(TR * 16) combine_staged_kernel(const CombineArgs a) {
  extern __shared__ float4 tile4[];  // [block][TR][16]
  const int64_t r0 = (int64_t)blockIdx.y * TR, c0 = (int64_t)blockIdx.x * kTC;
  const int tr = threadIdx.x >> 4, tq = threadIdx.x & 15, tc = tq * 4;
  const int es = DT == kF32 ? 4 : 2;
  const bool vec_ok = ((uintptr_t)a.src % (4 * es) == 0) && (a.ld % 4 == 0) && (a.b_cols % 4 == 0) &&
                      (!a.ce || (uintptr_t)a.ce % 16 == 0);
  const int n_rb = (int)a.n_rb, n_cb = (int)a.n_cb;
  const int64_t lr = r0 + tr, lc = c0 + tc;
  for (int rb = 0; rb < n_rb; ++rb) {
    const int64_t nr = min(a.b_rows, a.rows - rb * a.b_rows);
    const int64_t gr = rb * a.b_rows + lr;
    const bool row_in = r0 + TR <= nr;
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
      tile4[((rb * n_cb + cb) * TR + tr) * 16 + tq] = make_float4(x[0], x[1], x[2], x[3]);
    }
  }
  __syncthreads();
  const int64_t R = a.num_leaves;
  unsigned short* out = static_cast<unsigned short*>(a.out);
  const int64_t plane = R * a.p_rows * a.p_cols;
  for (int64_t r = 0; r < R; ++r) {
    const LeafDesc* L = a.leaves + r;
    const int n = a.side == 0 ? __ldg(&L->na) : __ldg(&L->nb);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = 0; t < n; ++t) {
      const int32_t blk = a.side == 0 ? __ldg(&L->a_blk[t]) : __ldg(&L->b_blk[t]);
      const float coef = a.side == 0 ? __ldg(&L->a_coef[t]) : __ldg(&L->b_coef[t]);
      const int bt = (blk >> a.blk_t_shift) & 0xFFFF, bk = (blk >> a.blk_k_shift) & 0xFFFF;
      const int b = a.t_rows ? bt * n_cb + bk : bk * n_cb + bt;
      const float4 v = tile4[(b * TR + tr) * 16 + tq];
      acc[0] = fmaf(coef, v.x, acc[0]);
      acc[1] = fmaf(coef, v.y, acc[1]);
      acc[2] = fmaf(coef, v.z, acc[2]);
      acc[3] = fmaf(coef, v.w, acc[3]);
    }
    const int64_t off = (r * a.p_rows + lr) * a.p_cols + lc;
    store4<FMT>(out + off, out + off + plane, acc);
  }
}

template <int DT, int FMT>
void launch_staged(const CombineArgs& a, int nb, cudaStream_t st) {
  // TR rows per CTA so that the staged tiles take at most 48 KB
  if (nb <= 6) {
    combine_staged_kernel<DT, FMT, 32><<<dim3((unsigned)(a.p_cols / kTC), (unsigned)(a.p_rows / 32)), 512,
                                         nb * 32 * 256, st>>>(a);
  } else if (nb <= 12) {
    combine_staged_kernel<DT, FMT, 16><<<dim3((unsigned)(a.p_cols / kTC), (unsigned)(a.p_rows / 16)), 256,
                                         nb * 16 * 256, st>>>(a);
  } else {
    combine_staged_kernel<DT, FMT, 8><<<dim3((unsigned)(a.p_cols / kTC), (unsigned)(a.p_rows / 8)), 128,
                                        nb * 8 * 256, st>>>(a);
  }
}

template <int DT, int FMT>
void launch_fmt(const CombineArgs& a, dim3 grid, cudaStream_t st) {
  const int64_t nb = a.n_rb * a.n_cb;
  if (nb <= kMaxStaged) launch_staged<DT, FMT>(a, (int)nb, st);
  else combine_kernel<DT, FMT><<<grid, kThreads, 0, st>>>(a);
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

}  // namespace

cudaError_t launch_combine(const CombineArgs& a, cudaStream_t st) {
  if (a.p_rows % kTR != 0 || a.p_cols % kTC != 0 || a.p_rows / kTR > 65535) return cudaErrorInvalidValue;
  if (a.b_rows > a.p_rows || a.b_cols > a.p_cols) return cudaErrorInvalidValue;
  if (a.num_leaves == 0 || a.p_rows == 0 || a.p_cols == 0) return cudaSuccess;
  const dim3 grid((unsigned)(a.p_cols / kTC), (unsigned)(a.p_rows / kTR));
  switch (a.dtype) {
    case kF32: return launch_dt<kF32>(a, grid, st);
    case kBF16: return launch_dt<kBF16>(a, grid, st);
    default: return launch_dt<kF16>(a, grid, st);
  }
}

}  // namespace fmm
