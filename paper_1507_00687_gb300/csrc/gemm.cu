// Fused recursive fast matrix multiplication kernel (sm_103a, tcgen05).
//
// One launch runs every leaf of a flattened plan (Eq. 4.4):
//   S_r = sum_t a_coef[t] A'(a_blk[t]),  T_r = sum_t b_coef[t] B'(b_blk[t]),
//   M_r = S_r T_r,                       C(c_blk[t]) += c_coef[t] M_r,
// with A' = 2^-eA A 2^d and B' = 2^-d B 2^-eB (the scaled operands of
// Algs. 1-3) and the unscale C = 2^eA C' 2^eB folded into the last step.
//
// CTA roles (416 threads, one CTA per SM, persistent over output tiles):
//   warps 0-3   epilogue: TMEM -> registers, C(blk) = / += coef 2^(eA+eB) M_r
//   warp  4     TMEM allocator and single-thread tcgen05.mma issuer
//   warps 5-12  producers: load the terms of S_r / T_r from global memory,
//               apply the power-of-two scales, sum in FP32 in index order,
//               round to the leaf format (bf16 / fp16 / bf16 hi+lo) and
//               store the tile in the 128-byte-swizzled K-major layout the
//               tensor core reads.
// A CTA owns one BM x BN tile coordinate of the leaf block grid and visits
// every leaf for it in leaf order, so each C element is updated by one
// thread in a fixed order: the result is deterministic.
//
// Every mbarrier wait is bounded (globaltimer); on expiry the kernel sets the
// timeout bit of the status word, stops all roles, drains its MMAs and frees
// its TMEM before returning.
#include <cmath>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace fmm {

namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kProdWarp0 = 5;
constexpr int kProdWarps = 8;
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kThreads = (kEpiWarps + 1 + kProdWarps) * 32;

constexpr int kModeBF16 = 0, kModeF16 = 1, kModeBF16x3 = 2;

template <int BN, int MODE>
struct Cfg {
  static constexpr int kSplit = MODE == kModeBF16x3 ? 2 : 1;
  static constexpr int kATile = BM * BK * 2;
  static constexpr int kBTile = BN * BK * 2;
  static constexpr int kStage = kSplit * (kATile + kBTile);
  static constexpr int kStages = (200 * 1024) / kStage > 8 ? 8 : (200 * 1024) / kStage;
  static constexpr int kTmemCols = 2 * BN;  // double-buffered fp32 accumulator
  static constexpr int kBarBytes = 256;
  static constexpr int kSmem = kStages * kStage + kBarBytes + 1024;  // + alignment slack
};

// ------------------------------------------------------------ producer side

template <int DT>
__device__ __forceinline__ float load1(const void* p, int64_t idx) {
  if constexpr (DT == kF32) {
    return __ldg(reinterpret_cast<const float*>(p) + idx);
  } else if constexpr (DT == kBF16) {
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(p) + idx));
  } else {
    return __half2float(__ldg(reinterpret_cast<const __half*>(p) + idx));
  }
}

template <int DT>
__device__ __forceinline__ void load8(const void* p, int64_t idx, float (&v)[8]) {
  if constexpr (DT == kF32) {
    const float4* q = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(p) + idx);
    float4 x = __ldg(q), y = __ldg(q + 1);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
  } else {
    uint4 x = __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const unsigned short*>(p) + idx));
    uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if constexpr (DT == kBF16) {
        v[2 * t] = __uint_as_float(w[t] << 16);
        v[2 * t + 1] = __uint_as_float(w[t] & 0xFFFF0000u);
      } else {
        __half2 h = *reinterpret_cast<__half2*>(&w[t]);
        float2 f = __half22float2(h);
        v[2 * t] = f.x;
        v[2 * t + 1] = f.y;
      }
    }
  }
}

__device__ __forceinline__ uint32_t pack2(float a, float b, int mode) {
  if (mode == kModeF16) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Byte offset of 16-byte chunk `kc` (8 elements along K) of tile row `row`
// in the 128-byte-swizzle K-major layout.
__device__ __forceinline__ uint32_t sw128_off(int row, int kc) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((kc ^ (row & 7)) << 4));
}

// Round the 8 FP32 sums to the leaf format and store (hi, and lo for the
// three-product split) at (row, kc).
template <int MODE>
__device__ __forceinline__ void store_chunk(uint8_t* hi, uint8_t* lo, int row, int kc, const float (&s)[8]) {
  const uint32_t off = sw128_off(row, kc);
  uint4 h;
  h.x = pack2(s[0], s[1], MODE);
  h.y = pack2(s[2], s[3], MODE);
  h.z = pack2(s[4], s[5], MODE);
  h.w = pack2(s[6], s[7], MODE);
  *reinterpret_cast<uint4*>(hi + off) = h;
  if constexpr (MODE == kModeBF16x3) {
    float r[8];
    const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      r[2 * t] = s[2 * t] - __uint_as_float(hw[t] << 16);
      r[2 * t + 1] = s[2 * t + 1] - __uint_as_float(hw[t] & 0xFFFF0000u);
    }
    uint4 l;
    l.x = pack2(r[0], r[1], MODE);
    l.y = pack2(r[2], r[3], MODE);
    l.z = pack2(r[4], r[5], MODE);
    l.w = pack2(r[6], r[7], MODE);
    *reinterpret_cast<uint4*>(lo + off) = l;
  }
}

// Accumulate one term's 8 values (k = kl .. kl+7 of tile row tl) into s.
template <int DT>
__device__ __forceinline__ void add_term(const TileOperand& op, int32_t blk, float coef, int64_t tl, int64_t kl,
                                         float (&s)[8]) {
  const int64_t tb = (blk >> op.blk_t_shift) & 0xFFFF;
  const int64_t kb = (blk >> op.blk_k_shift) & 0xFFFF;
  if (tl >= op.bt) return;
  const int64_t gt = tb * op.bt + tl;
  if (gt >= op.T) return;
  const int64_t gk = kb * op.bk + kl;
  float v[8];
  const bool full = (kl + 8 <= op.bk) && (gk + 8 <= op.K);
  if (op.kcontig) {
    if (full && op.vec_ok) {
      load8<DT>(op.ptr, gt * op.ld + gk, v);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        v[j] = (kl + j < op.bk && gk + j < op.K) ? load1<DT>(op.ptr, gt * op.ld + gk + j) : 0.f;
    }
  } else {
    if (full) {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = load1<DT>(op.ptr, (gk + j) * op.ld + gt);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        v[j] = (kl + j < op.bk && gk + j < op.K) ? load1<DT>(op.ptr, (gk + j) * op.ld + gt) : 0.f;
    }
  }
  if (op.k_exp) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (gk + j < op.K) v[j] *= exp2i(op.k_sign * __ldg(op.k_exp + gk + j));
  }
  if (op.t_exp) {
    const float ts = exp2i(op.t_sign * __ldg(op.t_exp + gt));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] *= ts;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) s[j] = fmaf(coef, v[j], s[j]);
}

// Produce one ROWS x 64 operand tile (the sum over the leaf's terms) into
// hi (and lo).  ptid in [0, 256).
template <int ROWS, int MODE, int DT>
__device__ __forceinline__ void fill_tile(const TileOperand& op, const int32_t* blk, const float* coef, int nterms,
                                          int64_t t0, int64_t k0, uint8_t* hi, uint8_t* lo, int ptid) {
  constexpr int kIters = ROWS * 8 / kProdThreads;
#pragma unroll 1
  for (int it = 0; it < kIters; ++it) {
    const int c = ptid + kProdThreads * it;
    // k-contiguous operands: 8 lanes cover one 64-wide row (vector loads);
    // t-contiguous operands: consecutive lanes take consecutive rows.
    const int row = op.kcontig ? (c >> 3) : (c % ROWS);
    const int kc = op.kcontig ? (c & 7) : (c / ROWS);
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int t = 0; t < nterms; ++t) add_term<DT>(op, __ldg(blk + t), __ldg(coef + t), t0 + row, k0 + kc * 8, s);
    store_chunk<MODE>(hi, lo, row, kc, s);
  }
}

template <int ROWS, int MODE>
__device__ __forceinline__ void fill_tile_dt(const TileOperand& op, const int32_t* blk, const float* coef,
                                             int nterms, int64_t t0, int64_t k0, uint8_t* hi, uint8_t* lo,
                                             int ptid) {
  switch (op.dtype) {
    case kF32: fill_tile<ROWS, MODE, kF32>(op, blk, coef, nterms, t0, k0, hi, lo, ptid); break;
    case kBF16: fill_tile<ROWS, MODE, kBF16>(op, blk, coef, nterms, t0, k0, hi, lo, ptid); break;
    default: fill_tile<ROWS, MODE, kF16>(op, blk, coef, nterms, t0, k0, hi, lo, ptid); break;
  }
}

// ------------------------------------------------------------ epilogue side

__device__ __forceinline__ void epi_chunk(const EpilogueArgs& c, const LeafDesc* L, int64_t ml, int64_t nl0,
                                          const uint32_t (&r)[32]) {
  const int nc = __ldg(&L->nc);
  for (int t = 0; t < nc; ++t) {
    const int32_t blk = __ldg(&L->c_blk[t]);
    const int64_t bi = (blk >> 16) & 0xFFFF, bj = blk & 0xFFFF;
    const int64_t gi = bi * c.bm + ml;
    if (gi >= c.M) continue;
    const float coef = __ldg(&L->c_coef[t]);
    const bool first = __ldg(&L->c_first[t]) != 0;
    const float s = c.eA ? coef * exp2i(__ldg(c.eA + gi)) : coef;
    const int64_t gj0 = bj * c.bn + nl0;
    float* crow = c.C + gi * c.ldc;
    if (c.vec_ok && nl0 + 32 <= c.bn && gj0 + 32 <= c.N) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float4 v;
        float* vp = reinterpret_cast<float*>(&v);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = 4 * q + u;
          float x = s * __uint_as_float(r[j]);
          if (c.eB) x *= exp2i(__ldg(c.eB + gj0 + j));
          vp[u] = x;
        }
        float4* dst = reinterpret_cast<float4*>(crow + gj0 + 4 * q);
        if (!first) {
          const float4 o = *dst;
          v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
        }
        *dst = v;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int64_t nl = nl0 + j, gj = gj0 + j;
        if (nl < c.bn && gj < c.N) {
          float x = s * __uint_as_float(r[j]);
          if (c.eB) x *= exp2i(__ldg(c.eB + gj));
          crow[gj] = first ? x : crow[gj] + x;
        }
      }
    }
  }
}

// ------------------------------------------------------------ the kernel

template <int BN, int MODE>
__global__ void __launch_bounds__(kThreads, 1) fused_fmm_kernel(const __grid_constant__ GemmArgs args) {
  using C = Cfg<BN, MODE>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kStages * C::kStage);
  uint64_t* empty = full + C::kStages;
  uint64_t* tfull = empty + C::kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], kProdThreads);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps * 32);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == kMmaWarp) tmem_alloc(tmem_slot, C::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int64_t ntm = (args.c.bm + BM - 1) / BM;
  const int64_t ntn = (args.c.bn + BN - 1) / BN;
  const int64_t ntiles = ntm * ntn;
  const int64_t KT = (args.kl + BK - 1) / BK;
  const int64_t NL = args.num_leaves;

  if (warp >= kProdWarp0) {
    // ---------------------------------------------------------- producers
    const int ptid = threadIdx.x - kProdWarp0 * 32;
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int64_t tm = tile / ntn, tn = tile % ntn;
      for (int64_t leaf = 0; leaf < NL && ok; ++leaf) {
        const LeafDesc* L = args.leaves + leaf;
        const int na = __ldg(&L->na), nb = __ldg(&L->nb);
        for (int64_t kt = 0; kt < KT; ++kt) {
          if (!mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, args.timeout_ns)) { ok = false; break; }
          uint8_t* st = smem + stage * C::kStage;
          uint8_t* a_hi = st;
          uint8_t* a_lo = st + C::kATile;
          uint8_t* b_hi = st + C::kSplit * C::kATile;
          uint8_t* b_lo = b_hi + C::kBTile;
          fill_tile_dt<BM, MODE>(args.a, L->a_blk, L->a_coef, na, tm * BM, kt * BK, a_hi, a_lo, ptid);
          fill_tile_dt<BN, MODE>(args.b, L->b_blk, L->b_coef, nb, tn * BN, kt * BK, b_hi, b_lo, ptid);
          fence_proxy_async_smem();
          mbar_arrive(&full[stage]);
          if (++stage == C::kStages) { stage = 0; phase ^= 1u; }
        }
      }
    }
    if (!ok) *abort_flag = 1;
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(MODE == kModeF16 ? 0u : 1u, BM, BN);
      int stage = 0;
      uint32_t phase = 0, acc_iter = 0;
      bool ok = true;
      const uint32_t sbase = smem_u32(smem);
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int64_t leaf = 0; leaf < NL && ok; ++leaf) {
          const uint32_t buf = acc_iter & 1u, aph = (acc_iter >> 1) & 1u;
          if (!mbar_wait_bounded(&tempty[buf], aph ^ 1u, abort_flag, args.timeout_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + buf * BN;
          for (int64_t kt = 0; kt < KT; ++kt) {
            if (!mbar_wait_bounded(&full[stage], phase, abort_flag, args.timeout_ns)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a_hi = sbase + stage * C::kStage;
            const uint32_t a_lo = a_hi + C::kATile;
            const uint32_t b_hi = a_hi + C::kSplit * C::kATile;
            const uint32_t b_lo = b_hi + C::kBTile;
#pragma unroll
            for (int k16 = 0; k16 < BK / 16; ++k16) {
              const uint32_t acc = (kt > 0 || k16 > 0) ? 1u : 0u;
              const uint64_t ah = smem_desc_sw128(a_hi + k16 * 32);
              const uint64_t bh = smem_desc_sw128(b_hi + k16 * 32);
              mma_f16(d_tmem, ah, bh, idesc, acc);
              if constexpr (MODE == kModeBF16x3) {
                mma_f16(d_tmem, ah, smem_desc_sw128(b_lo + k16 * 32), idesc, 1u);
                mma_f16(d_tmem, smem_desc_sw128(a_lo + k16 * 32), bh, idesc, 1u);
              }
            }
            mma_commit(&empty[stage]);
            if (++stage == C::kStages) { stage = 0; phase ^= 1u; }
          }
          if (!ok) break;
          mma_commit(&tfull[buf]);
          ++acc_iter;
        }
      }
      if (!ok) *abort_flag = 1;
      // All issued MMAs complete before TMEM is released.  MMAs never wait on
      // anything, so this wait ends within microseconds; it has its own 1 s
      // cap, independent of the configured wait limit and of the abort flag.
      mma_commit(drain);
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(drain, 0) && globaltimer_ns() - t0 < 1000000000ull) {
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- epilogue
    uint32_t acc_iter = 0;
    bool ok = true;
    const int row = warp * 32 + lane;  // TMEM lane = tile row
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int64_t tm = tile / ntn, tn = tile % ntn;
      const int64_t ml = tm * BM + row;
      for (int64_t leaf = 0; leaf < NL; ++leaf) {
        const uint32_t buf = acc_iter & 1u, aph = (acc_iter >> 1) & 1u;
        // warp-uniform outcome: the TMEM loads below are .sync.aligned
        ok = __all_sync(0xffffffffu, mbar_wait_bounded(&tfull[buf], aph, abort_flag, args.timeout_ns));
        if (!ok) break;
        tc_fence_after();
        const LeafDesc* L = args.leaves + leaf;
#pragma unroll 1
        for (int cc = 0; cc < BN / 32; ++cc) {
          uint32_t r[32];
          tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(warp * 32) << 16) + buf * BN + cc * 32, r);
          if (ml < args.c.bm) epi_chunk(args.c, L, ml, tn * BN + cc * 32, r);
        }
        tc_fence_before();
        mbar_arrive(&tempty[buf]);
        ++acc_iter;
      }
    }
    if (!ok) *abort_flag = 1;
  }

  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(args.status, kStatusTimeout);
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem_base, C::kTmemCols);
  }
}

template <int BN, int MODE>
cudaError_t launch_cfg(const GemmArgs& a, cudaStream_t st) {
  using C = Cfg<BN, MODE>;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(fused_fmm_kernel<BN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::kSmem);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const int64_t ntiles = ((a.c.bm + BM - 1) / BM) * ((a.c.bn + BN - 1) / BN);
  const int64_t grid = std::min<int64_t>(ntiles, device_sm_count());
  fused_fmm_kernel<BN, MODE><<<(unsigned)grid, kThreads, C::kSmem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

int device_sm_count() {
  static int n[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (n[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n[dev] = v > 0 ? v : 1;
  }
  return n[dev];
}

cudaError_t launch_fused_gemm(const GemmArgs& a, int leaf_format, cudaStream_t st) {
  // N tile: 256 unless the smaller tile gives fewer idle SMs.
  const int sms = device_sm_count();
  auto util = [&](int bn) {
    const double t = (double)((a.c.bm + BM - 1) / BM) * (double)((a.c.bn + bn - 1) / bn);
    const double waves = std::ceil(t / sms);
    const double eff_n = (double)a.c.bn / (double)(((a.c.bn + bn - 1) / bn) * bn);
    return t / (waves * sms) * eff_n;
  };
  const bool small = util(128) > util(256) * 1.05;
  switch (leaf_format) {
    case FMM_LEAF_BF16: return small ? launch_cfg<128, kModeBF16>(a, st) : launch_cfg<256, kModeBF16>(a, st);
    case FMM_LEAF_F16: return small ? launch_cfg<128, kModeF16>(a, st) : launch_cfg<256, kModeF16>(a, st);
    default: return small ? launch_cfg<128, kModeBF16x3>(a, st) : launch_cfg<256, kModeBF16x3>(a, st);
  }
}

}  // namespace fmm
