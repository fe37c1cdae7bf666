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

template <int DT>
__device__ __forceinline__ int elem_fexp(const void* base, int64_t idx, bool* nf) {
  if constexpr (DT == kF32) {
    return fexp_f32(__ldg(reinterpret_cast<const uint32_t*>(base) + idx), nf);
  } else {
    uint32_t b = __ldg(reinterpret_cast<const unsigned short*>(base) + idx);
    return DT == kBF16 ? fexp_bf16(b, nf) : fexp_f16(b, nf);
  }
}

template <int DT>
__device__ __forceinline__ void elem_fexp4(const void* base, int64_t idx, bool* nf, int (&e)[4]) {
  if constexpr (DT == kF32) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const uint32_t*>(base) + idx));
    e[0] = fexp_f32(v.x, nf); e[1] = fexp_f32(v.y, nf); e[2] = fexp_f32(v.z, nf); e[3] = fexp_f32(v.w, nf);
  } else {
    uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const unsigned short*>(base) + idx));
    uint32_t h[4] = {v.x & 0xFFFFu, v.x >> 16, v.y & 0xFFFFu, v.y >> 16};
#pragma unroll
    for (int t = 0; t < 4; ++t) e[t] = DT == kBF16 ? fexp_bf16(h[t], nf) : fexp_f16(h[t], nf);
  }
}

__device__ __forceinline__ int block_max(int v, int* red) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : kZeroExp;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

// Row reduction.  For each row i of the R x C matrix X:
//   m_i = max_j ( e(X_ij) + cs * ce_j )          (kZeroExp if the row is 0)
// mode kRowOStep:  out[i] = m_i, or 0 for a zero row          (O step)
// mode kRowIStep:  out[i] holds e_x (a column max of the other operand, from
//   col_exp_kernel); out[i] = floor((m_i - e_x) / 2), 0 if either is zero
//   (the I-step exponent of Eq. 6.6).
template <int DT>
__global__ void __launch_bounds__(256) row_exp_kernel(const void* X, int64_t R, int64_t C, int64_t ld,
                                                      const int* ce, int cs, int* out, int mode,
                                                      int vec_ok, int* status) {
  __shared__ int red[32];
  bool nf = false;
  for (int64_t i = blockIdx.x; i < R; i += gridDim.x) {
    int m = kZeroExp;
    const int64_t rowoff = i * ld;
    if (vec_ok) {
      const int64_t C4 = C >> 2;
      for (int64_t j4 = threadIdx.x; j4 < C4; j4 += blockDim.x) {
        int e[4];
        elem_fexp4<DT>(X, rowoff + 4 * j4, &nf, e);
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (e[t] != kZeroExp) m = max(m, e[t] + (ce ? cs * __ldg(ce + 4 * j4 + t) : 0));
      }
      for (int64_t j = 4 * C4 + threadIdx.x; j < C; j += blockDim.x) {
        int e = elem_fexp<DT>(X, rowoff + j, &nf);
        if (e != kZeroExp) m = max(m, e + (ce ? cs * __ldg(ce + j) : 0));
      }
    } else {
      for (int64_t j = threadIdx.x; j < C; j += blockDim.x) {
        int e = elem_fexp<DT>(X, rowoff + j, &nf);
        if (e != kZeroExp) m = max(m, e + (ce ? cs * __ldg(ce + j) : 0));
      }
    }
    m = block_max(m, red);
    if (threadIdx.x == 0) {
      if (mode == kRowOStep) {
        out[i] = (m == kZeroExp) ? 0 : m;
      } else {
        const int ex = out[i];
        out[i] = (m == kZeroExp || ex == kZeroExp) ? 0 : ((m - ex) >> 1);  // arithmetic shift = floor
      }
    }
  }
  if (nf) atomicOr(status, kStatusNonfinite);
}

// Column reduction: out[j] = max(out[j], max_i (e(X_ij) + rs * re_i)) over
// a chunk of rows per CTA (out pre-filled with kZeroExp).  Each thread owns
// 4 adjacent columns; a warp reads 512 contiguous bytes (fp32) per row.
template <int DT>
__global__ void __launch_bounds__(256) col_exp_kernel(const void* X, int64_t R, int64_t C, int64_t ld,
                                                      const int* re, int rs, int* out, int rows_per_cta,
                                                      int vec_ok, int* status) {
  bool nf = false;
  const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = min(R, r0 + rows_per_cta);
  if (c0 < C) {
    int m[4] = {kZeroExp, kZeroExp, kZeroExp, kZeroExp};
    const bool full = vec_ok && (c0 + 4 <= C);
    for (int64_t i = r0; i < r1; ++i) {
      const int sh = re ? rs * __ldg(re + i) : 0;
      int e[4];
      if (full) {
        elem_fexp4<DT>(X, i * ld + c0, &nf, e);
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) e[t] = (c0 + t < C) ? elem_fexp<DT>(X, i * ld + c0 + t, &nf) : kZeroExp;
      }
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (e[t] != kZeroExp) m[t] = max(m[t], e[t] + sh);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (c0 + t < C && m[t] != kZeroExp) atomicMax(out + c0 + t, m[t]);
  }
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
                           int* out, int mode, int* status, cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  const int vec = vec_aligned(X, ld, dt) ? 1 : 0;
  const int64_t grid = std::min<int64_t>(R, (int64_t)sm_count() * 16);
  dim3 g((unsigned)grid);
  switch (dt) {
    case kF32: row_exp_kernel<kF32><<<g, 256, 0, st>>>(X, R, C, ld, ce, cs, out, mode, vec, status); break;
    case kBF16: row_exp_kernel<kBF16><<<g, 256, 0, st>>>(X, R, C, ld, ce, cs, out, mode, vec, status); break;
    default: row_exp_kernel<kF16><<<g, 256, 0, st>>>(X, R, C, ld, ce, cs, out, mode, vec, status); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_col_exp(const void* X, int dt, int64_t R, int64_t C, int64_t ld, const int* re, int rs,
                           int* out, int* status, cudaStream_t st) {
  if (C == 0) return cudaSuccess;
  fill_kernel<<<(unsigned)std::min<int64_t>((C + 255) / 256, 4096), 256, 0, st>>>(out, C, kZeroExp);
  if (R == 0) return cudaGetLastError();
  const int vec = vec_aligned(X, ld, dt) ? 1 : 0;
  const int64_t gx = (C + 1023) / 1024;
  // enough CTAs to cover ~8 per SM; at least 16 rows per CTA
  int64_t target = (int64_t)sm_count() * 8;
  int64_t gy = std::max<int64_t>(1, std::min<int64_t>((target + gx - 1) / gx, (R + 15) / 16));
  gy = std::min<int64_t>(gy, 65535);
  const int rows = (int)((R + gy - 1) / gy);
  gy = (R + rows - 1) / rows;
  dim3 g((unsigned)gx, (unsigned)gy);
  switch (dt) {
    case kF32: col_exp_kernel<kF32><<<g, 256, 0, st>>>(X, R, C, ld, re, rs, out, rows, vec, status); break;
    case kBF16: col_exp_kernel<kBF16><<<g, 256, 0, st>>>(X, R, C, ld, re, rs, out, rows, vec, status); break;
    default: col_exp_kernel<kF16><<<g, 256, 0, st>>>(X, R, C, ld, re, rs, out, rows, vec, status); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_zero_sentinel(int* p, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  zero_sentinel_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(p, n);
  return cudaGetLastError();
}

cudaError_t launch_prepare(const void* X, int dt, int64_t R, int64_t C, int64_t ld, int64_t row_blk,
                           int64_t row_pad, int64_t col_blk, int64_t col_pad, const int* re, int rs, const int* ce,
                           int cs, void* Y, int64_t Rp, int64_t Cp, int64_t ldy, cudaStream_t st) {
  if (Rp == 0 || Cp == 0) return cudaSuccess;
  const int64_t total = Rp * (Cp / 4);
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count() * 16);
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

cudaError_t launch_fill(int* p, int64_t n, int v, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  fill_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

}  // namespace fmm
