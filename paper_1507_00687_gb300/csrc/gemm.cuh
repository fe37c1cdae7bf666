#pragma once
// Fused recursive fast matrix multiplication kernel (sm_103a, tcgen05).
//
// One launch runs every leaf of a flattened plan (Eq. 4.4):
//   S_r = sum_t a_coef[t] A'(a_blk[t]),  T_r = sum_t b_coef[t] B'(b_blk[t]),
//   M_r = S_r T_r,                       C(c_blk[t]) += c_coef[t] M_r,
// on operands A', B' (when scaling, the power-of-two scaled copies that the
// apply pass of scale.cu wrote) and the unscale C = 2^eA C' 2^eB of
// Algs. 1-3 folded into the last step.
//
// CTA roles (384 threads, one CTA per SM, persistent over output tiles):
//   warps 0-3   epilogue: TMEM -> registers, C(blk) = / += coef 2^(eA+eB) M_r
//   warp  4     TMEM allocator and single-thread tcgen05.mma issuer
//   warps 5-11  producers: load the terms of S_r / T_r from global memory,
//               sum them in FP32 in index order,
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

// Kernel templates of the fused multiply; instantiated per leaf format by
// gemm_bf16.cu, gemm_f16.cu and gemm_bf16x3.cu.

namespace fmm {
namespace gemm {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kProdWarp0 = 5;
constexpr int kProdWarps = 7;  // 12 warps in all: registers are granted per 4 warps
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kThreads = (kEpiWarps + 1 + kProdWarps) * 32;

constexpr int kModeBF16 = 0, kModeF16 = 1, kModeBF16x3 = 2;


// Per-iteration facts about one term of one operand side, computed once per
// term so that a load unit costs one shared-memory lookup and one add:
//   base      element offset of the term's tile origin (t0, k0) in its operand
//   interior  the whole ROWS x 64 tile lies inside the term's block and the
//             operand, and vector loads are allowed
struct TermInfo {
  int64_t base;
  float coef;
  int32_t interior;
  int32_t tb, kb;
};

// What the producers of one pipeline iteration read from shared memory.
// Two copies alternate; the copy for iteration i+1 is written during
// iteration i, and the producers' named barrier at the top of each
// iteration orders the writes before the reads.
struct StageCtx {
  TermInfo a[kMaxTerms];
  TermInfo b[kMaxTerms];
  int32_t na, nb;
  int32_t a_interior, b_interior;  // every term of the side is interior
};

template <int BN, int MODE>
struct Cfg {
  static constexpr int kSplit = MODE == kModeBF16x3 ? 2 : 1;
  static constexpr int kATile = BM * BK * 2;
  static constexpr int kBTile = BN * BK * 2;
  static constexpr int kStage = kSplit * (kATile + kBTile);
  static constexpr int kCtx = 2 * (int)sizeof(StageCtx);  // two iteration contexts
  static constexpr int kStages =
      (220 * 1024 - kCtx) / kStage > 8 ? 8 : (220 * 1024 - kCtx) / kStage;
  static constexpr int kTmemCols = 2 * BN;  // double-buffered fp32 accumulator
  static constexpr int kBarBytes = 256;
  static constexpr int kSmem = kStages * kStage + kCtx + kBarBytes + 1024;  // + alignment slack
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

// 16-byte read-only load that does not allocate in L1 (operand data is
// streamed once per CTA; L1 is left to the small, reused lookups).
__device__ __forceinline__ uint4 ldg_stream(const void* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

template <int DT>
__device__ __forceinline__ void load8(const void* p, int64_t idx, float (&v)[8]) {
  if constexpr (DT == kF32) {
    const uint4* q = reinterpret_cast<const uint4*>(reinterpret_cast<const float*>(p) + idx);
    const uint4 x = ldg_stream(q), y = ldg_stream(q + 1);
    v[0] = __uint_as_float(x.x); v[1] = __uint_as_float(x.y); v[2] = __uint_as_float(x.z); v[3] = __uint_as_float(x.w);
    v[4] = __uint_as_float(y.x); v[5] = __uint_as_float(y.y); v[6] = __uint_as_float(y.z); v[7] = __uint_as_float(y.w);
  } else {
    uint4 x = ldg_stream(reinterpret_cast<const unsigned short*>(p) + idx);
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

// Byte offset of the 16-byte unit holding elements (t, 8kc .. 8kc+7) of a
// K-major tile: one 128-byte row of 64 k per t, 8-row groups 1024 bytes
// apart, units XOR-swizzled by (t mod 8) (the 128-byte swizzle pattern).
__device__ __forceinline__ uint32_t kmajor_off(int t, int kc) {
  return (uint32_t)((t >> 3) * 1024 + (t & 7) * 128 + ((kc ^ (t & 7)) << 4));
}

// Byte offset of the 16-byte unit holding elements (8tu .. 8tu+7, k) of an
// MN-major tile: one 128-byte row of 64 t per k, 8-k groups 1024 bytes
// apart, 64-wide t chunks 8192 bytes apart, units XOR-swizzled by (k mod 8).
__device__ __forceinline__ uint32_t mnmajor_off(int k, int tu) {
  return (uint32_t)((tu >> 3) * 8192 + (k >> 3) * 1024 + (k & 7) * 128 + (((tu & 7) ^ (k & 7)) << 4));
}

// Round 8 FP32 sums to the leaf format and store them (hi, and lo for the
// three-product split) at byte offset `off` of the tile.
template <int MODE>
__device__ __forceinline__ void store_unit(uint8_t* hi, uint8_t* lo, uint32_t off, const float (&s)[8]) {
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

// One load unit in flight: 8 operand values of one term (its coefficient is
// looked up when it is consumed).
struct Slot {
  float v[8];
};

// 32-byte / 16-byte read-only loads that do not allocate in L1 (operand data
// is streamed; L1 is left to small reused lookups).
__device__ __forceinline__ void ldg_v8f(const void* p, float (&v)[8]) {
  asm volatile("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}

template <int DT>
__device__ __forceinline__ void load8_vec(const void* p, int64_t idx, float (&v)[8]) {
  if constexpr (DT == kF32) {
    ldg_v8f(reinterpret_cast<const float*>(p) + idx, v);
  } else {
    const uint4 x = ldg_stream(reinterpret_cast<const unsigned short*>(p) + idx);
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if constexpr (DT == kBF16) {
        v[2 * t] = __uint_as_float(w[t] << 16);
        v[2 * t + 1] = __uint_as_float(w[t] & 0xFFFF0000u);
      } else {
        const __half2 h = *reinterpret_cast<const __half2*>(&w[t]);
        const float2 f = __half22float2(h);
        v[2 * t] = f.x;
        v[2 * t + 1] = f.y;
      }
    }
  }
}

// Position of chunk c of this thread inside the ROWS x 64 tile.
// KC (k contiguous): (t = c / 8, k = 8 (c % 8) .. +7), K-major smem layout.
// MN (t contiguous): (k = c / (ROWS/8), t = 8 (c % (ROWS/8)) .. +7),
//                    MN-major smem layout.
template <int ROWS, bool KC>
__device__ __forceinline__ int64_t chunk_off(int64_t ld, int c) {
  if constexpr (KC) {
    return (int64_t)(c >> 3) * ld + (c & 7) * 8;
  } else {
    constexpr int TU = ROWS / 8;
    return (int64_t)(c / TU) * ld + (c % TU) * 8;
  }
}
template <int ROWS, bool KC>
__device__ __forceinline__ uint32_t chunk_smem(int c) {
  if constexpr (KC) {
    return kmajor_off(c >> 3, c & 7);
  } else {
    constexpr int TU = ROWS / 8;
    return mnmajor_off(c / TU, c % TU);
  }
}

// Interior tiles: every term's ROWS x 64 tile lies inside its block and the
// operand, so every unit is one unconditional vector load.  Loads run
// kDepth units ahead of the arithmetic in a register ring, so each thread
// keeps kDepth x 32 bytes in flight; the loop body has no data-dependent
// branches between a load and its use.
constexpr int kDepth = 8;

template <int ROWS, int MODE, int DT, bool KC>
__device__ __forceinline__ void fill_interior(const TileOperand& op, const TermInfo* terms, int nterms, uint8_t* hi,
                                              uint8_t* lo, int ptid) {
  const int nch = (ROWS * 8 - ptid + kProdThreads - 1) / kProdThreads;  // chunks of this thread
  Slot ring[kDepth];
  int ic = 0, it = 0;  // next unit to issue: chunk (of this thread), term
  int cc = 0, ct = 0;  // next unit to consume
  int64_t ioff = chunk_off<ROWS, KC>(op.ld, ptid);
#pragma unroll
  for (int s = 0; s < kDepth; ++s) {
    if (ic < nch) {
      load8_vec<DT>(op.ptr, terms[it].base + ioff, ring[s].v);
      if (++it == nterms) {
        it = 0;
        if (++ic < nch) ioff = chunk_off<ROWS, KC>(op.ld, ptid + kProdThreads * ic);
      }
    }
  }
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int units = nch * nterms;
#pragma unroll 1
  for (int base = 0; base < units; base += kDepth) {
#pragma unroll
    for (int s = 0; s < kDepth; ++s) {
      if (cc < nch) {
        const float coef = terms[ct].coef;
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = fmaf(coef, ring[s].v[j], acc[j]);
        if (++ct == nterms) {
          store_unit<MODE>(hi, lo, chunk_smem<ROWS, KC>(ptid + kProdThreads * cc), acc);
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[j] = 0.f;
          ct = 0;
          ++cc;
        }
      }
      if (ic < nch) {
        load8_vec<DT>(op.ptr, terms[it].base + ioff, ring[s].v);
        if (++it == nterms) {
          it = 0;
          if (++ic < nch) ioff = chunk_off<ROWS, KC>(op.ld, ptid + kProdThreads * ic);
        }
      }
    }
  }
}

// Tiles touching a block or operand edge: element-wise loads with the
// block and operand limits (zero outside), one chunk at a time.
template <int ROWS, int MODE>
__device__ __noinline__ void fill_boundary(const TileOperand& op, const TermInfo* terms, int nterms, int64_t t0,
                                           int64_t k0, uint8_t* hi, uint8_t* lo, int ptid) {
  for (int c = ptid; c < ROWS * 8; c += kProdThreads) {
    int tl, kl;
    uint32_t soff;
    if (op.kcontig) {
      tl = c >> 3; kl = (c & 7) * 8; soff = kmajor_off(c >> 3, c & 7);
    } else {
      constexpr int TU = ROWS / 8;
      kl = c / TU; tl = (c % TU) * 8; soff = mnmajor_off(c / TU, c % TU);
    }
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int t = 0; t < nterms; ++t) {
      const TermInfo& ti = terms[t];
      const int64_t tg = t0 + tl, kg = k0 + kl;
      const int64_t gt = (int64_t)ti.tb * op.bt + tg, gk = (int64_t)ti.kb * op.bk + kg;
      const int64_t off = op.kcontig ? (int64_t)tl * op.ld + kl : (int64_t)kl * op.ld + tl;
      for (int j = 0; j < 8; ++j) {
        const bool ok = op.kcontig ? (tg < op.bt && gt < op.T && kg + j < op.bk && gk + j < op.K)
                                   : (kg < op.bk && gk < op.K && tg + j < op.bt && gt + j < op.T);
        if (ok) {
          const int64_t idx = ti.base + off + j;
          const float v = op.dtype == kF32 ? load1<kF32>(op.ptr, idx)
                                           : (op.dtype == kBF16 ? load1<kBF16>(op.ptr, idx) : load1<kF16>(op.ptr, idx));
          acc[j] = fmaf(ti.coef, v, acc[j]);
        }
      }
    }
    store_unit<MODE>(hi, lo, soff, acc);
  }
}

// Produce one ROWS x 64 operand tile: for each chunk, the sum over the
// leaf's terms in term (index) order, rounded to the leaf format.
template <int ROWS, int MODE, int DT, bool KC>
__device__ __forceinline__ void fill_tile(const TileOperand& op, const TermInfo* terms, int nterms, bool interior,
                                          int64_t t0, int64_t k0, uint8_t* hi, uint8_t* lo, int ptid) {
  if (nterms <= 0) return;
  if (interior) {
    fill_interior<ROWS, MODE, DT, KC>(op, terms, nterms, hi, lo, ptid);
  } else {
    fill_boundary<ROWS, MODE>(op, terms, nterms, t0, k0, hi, lo, ptid);
  }
}

// ------------------------------------------------------------ iteration context

struct IterPos {
  int64_t tm, tn, leaf, kt;
};

// Phase 1 (global loads into registers) and phase 2 (compute and store) of
// writing the context of one iteration.  Threads 0-15 own A's terms, 16-31
// B's terms, 32-33 the term counts.
struct CtxLoad {
  int32_t blk, n;
  float coef;
};

__device__ __forceinline__ void ctx_load(const GemmArgs& a, const IterPos& p, int ptid, CtxLoad& cl) {
  const LeafDesc* L = a.leaves + p.leaf;
  if (ptid < 2 * kMaxTerms) {
    const int q = ptid % kMaxTerms;
    const bool side_a = ptid < kMaxTerms;
    cl.n = __ldg(side_a ? &L->na : &L->nb);
    cl.blk = __ldg(side_a ? &L->a_blk[q] : &L->b_blk[q]);
    cl.coef = __ldg(side_a ? &L->a_coef[q] : &L->b_coef[q]);
  } else if (ptid < 2 * kMaxTerms + 2) {
    cl.n = __ldg(ptid == 2 * kMaxTerms ? &L->na : &L->nb);
  }
}

template <int ROWS>
__device__ __forceinline__ TermInfo term_info(const TileOperand& op, int32_t blk, float coef, int64_t t0,
                                              int64_t k0) {
  TermInfo ti;
  const int64_t tb = (blk >> op.blk_t_shift) & 0xFFFF, kb = (blk >> op.blk_k_shift) & 0xFFFF;
  const int64_t gt0 = tb * op.bt + t0, gk0 = kb * op.bk + k0;
  ti.base = op.kcontig ? gt0 * op.ld + gk0 : gk0 * op.ld + gt0;
  ti.coef = coef;
  ti.tb = (int32_t)tb;
  ti.kb = (int32_t)kb;
  ti.interior = (op.vec_ok && t0 + ROWS <= op.bt && k0 + BK <= op.bk && gt0 + ROWS <= op.T && gk0 + BK <= op.K) ? 1 : 0;
  return ti;
}

template <int BN>
__device__ __forceinline__ void ctx_store(const GemmArgs& a, const IterPos& p, int ptid, const CtxLoad& cl,
                                          StageCtx* c) {
  if (ptid < 2 * kMaxTerms) {
    // threads 0-31 are warp 0 of the producers: lanes 0-15 A's terms, 16-31 B's
    const int q = ptid % kMaxTerms;
    bool interior = true;
    if (q < cl.n) {
      const TermInfo ti = ptid < kMaxTerms ? term_info<BM>(a.a, cl.blk, cl.coef, p.tm * BM, p.kt * BK)
                                           : term_info<BN>(a.b, cl.blk, cl.coef, p.tn * BN, p.kt * BK);
      interior = ti.interior != 0;
      if (ptid < kMaxTerms) c->a[q] = ti;
      else c->b[q] = ti;
    }
    const unsigned all = __ballot_sync(0xffffffffu, interior);
    if (ptid == 0) {
      c->a_interior = (all & 0x0000FFFFu) == 0x0000FFFFu;
      c->b_interior = (all & 0xFFFF0000u) == 0xFFFF0000u;
    }
  } else if (ptid == 2 * kMaxTerms) {
    c->na = cl.n;
  } else if (ptid == 2 * kMaxTerms + 1) {
    c->nb = cl.n;
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

template <int BN, int MODE, int DTA, bool KCA, int DTB, bool KCB>
__global__ void __launch_bounds__(kThreads, 1) fused_fmm_kernel(const __grid_constant__ GemmArgs args) {
  using C = Cfg<BN, MODE>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  StageCtx* ctx = reinterpret_cast<StageCtx*>(smem + C::kStages * C::kStage);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kStages * C::kStage + C::kCtx);
  uint64_t* empty = full + C::kStages;
  uint64_t* tfull = empty + C::kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* prod_abort = abort_flag + 1;  // written by producers only

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
    *prod_abort = 0;
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
    // The terms of each iteration are staged in shared memory one iteration
    // ahead; all producers pass a named barrier per iteration, so they also
    // share the decision to stop (prod_abort is read after it).
    const int64_t my_tiles = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const int64_t per_tile = NL * KT;
    const int64_t iters = my_tiles * per_tile;
    auto pos = [&](int64_t i) {
      const int64_t tile = blockIdx.x + (i / per_tile) * gridDim.x, r = i % per_tile;
      return IterPos{tile / ntn, tile % ntn, r / KT, r % KT};
    };
    if (iters > 0) {
      CtxLoad cl;
      const IterPos p0 = pos(0);
      ctx_load(args, p0, ptid, cl);
      ctx_store<BN>(args, p0, ptid, cl, ctx);
    }
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t i = 0; i < iters; ++i) {
      ok = mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, args.timeout_ns);
      if (!ok) *prod_abort = 1;
      asm volatile("bar.sync 1, %0;" ::"n"(kProdThreads) : "memory");
      ok = *prod_abort == 0;
      if (!ok) break;
      const IterPos p = pos(i);
      const StageCtx* cur = ctx + (i & 1);
      CtxLoad cl;
      const bool more = i + 1 < iters;
      IterPos pn{};
      if (more) {
        pn = pos(i + 1);
        ctx_load(args, pn, ptid, cl);
      }
      uint8_t* st = smem + stage * C::kStage;
      uint8_t* a_hi = st;
      uint8_t* a_lo = st + C::kATile;
      uint8_t* b_hi = st + C::kSplit * C::kATile;
      uint8_t* b_lo = b_hi + C::kBTile;
      fill_tile<BM, MODE, DTA, KCA>(args.a, cur->a, cur->na, cur->a_interior, p.tm * BM, p.kt * BK, a_hi, a_lo,
                                    ptid);
      if (more) ctx_store<BN>(args, pn, ptid, cl, ctx + ((i + 1) & 1));
      fill_tile<BN, MODE, DTB, KCB>(args.b, cur->b, cur->nb, cur->b_interior, p.tn * BN, p.kt * BK, b_hi, b_lo,
                                    ptid);
      fence_proxy_async_smem();
      mbar_arrive(&full[stage]);
      if (++stage == C::kStages) { stage = 0; phase ^= 1u; }
    }
    if (!ok) *abort_flag = 1;
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      // K-major operands advance 32 bytes per 16-wide K step inside the
      // swizzled row; MN-major operands advance two 8-k groups (2048 bytes).
      constexpr bool a_mn = !KCA, b_mn = !KCB;
      constexpr uint32_t idesc = idesc_f16(MODE == kModeF16 ? 0u : 1u, BM, BN, a_mn, b_mn);
      auto a_desc = [&](uint32_t base, int k16) {
        return a_mn ? smem_desc_mn_sw128(base + k16 * 2048) : smem_desc_sw128(base + k16 * 32);
      };
      auto b_desc = [&](uint32_t base, int k16) {
        return b_mn ? smem_desc_mn_sw128(base + k16 * 2048) : smem_desc_sw128(base + k16 * 32);
      };
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
              const uint64_t ah = a_desc(a_hi, k16), bh = b_desc(b_hi, k16);
              mma_f16(d_tmem, ah, bh, idesc, acc);
              if constexpr (MODE == kModeBF16x3) {
                mma_f16(d_tmem, ah, b_desc(b_lo, k16), idesc, 1u);
                mma_f16(d_tmem, a_desc(a_lo, k16), bh, idesc, 1u);
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

// Launch one instantiation: grid = min(tiles, SMs), one CTA per SM.
template <int BN, int MODE, int DTA, bool KCA, int DTB, bool KCB>
cudaError_t launch_cfg(const GemmArgs& a, cudaStream_t st) {
  using C = Cfg<BN, MODE>;
  auto kern = fused_fmm_kernel<BN, MODE, DTA, KCA, DTB, KCB>;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const int64_t ntiles = ((a.c.bm + BM - 1) / BM) * ((a.c.bn + BN - 1) / BN);
  const int64_t grid = std::min<int64_t>(ntiles, device_sm_count());
  kern<<<(unsigned)grid, kThreads, C::kSmem, st>>>(a);
  return cudaGetLastError();
}

// The operand (dtype, layout) pairs the forward and backward passes use:
// forward A (in, k-contiguous) x B (in, n-contiguous); dA = dC B^T with
// dC (fp32, k-contiguous) x B^T (in, k-contiguous); dB = A^T dC with
// A^T (in, m-contiguous) x dC (fp32, n-contiguous); in = fp32 or bf16.
template <int MODE>
cudaError_t launch_mode(const GemmArgs& a, cudaStream_t st) {
  constexpr int BN = 256;
  const int da = a.a.dtype, db = a.b.dtype;
  const bool ka = a.a.kcontig != 0, kb = a.b.kcontig != 0;
  if (ka && !kb && da == kF32 && db == kF32) return launch_cfg<BN, MODE, kF32, true, kF32, false>(a, st);
  if (ka && !kb && da == kBF16 && db == kBF16) return launch_cfg<BN, MODE, kBF16, true, kBF16, false>(a, st);
  if (ka && kb && da == kF32 && db == kF32) return launch_cfg<BN, MODE, kF32, true, kF32, true>(a, st);
  if (ka && kb && da == kF32 && db == kBF16) return launch_cfg<BN, MODE, kF32, true, kBF16, true>(a, st);
  if (!ka && !kb && da == kF32 && db == kF32) return launch_cfg<BN, MODE, kF32, false, kF32, false>(a, st);
  if (!ka && !kb && da == kBF16 && db == kF32) return launch_cfg<BN, MODE, kBF16, false, kF32, false>(a, st);
  return cudaErrorNotSupported;
}

}  // namespace gemm
}  // namespace fmm
