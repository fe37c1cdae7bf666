#pragma once
// Pieces shared by the multiply kernels: bulk tensor copies and the
// epilogue that adds one leaf product into its C blocks (Eq. 4.4, third
// line) with the unscale 2^(eA_i + eB_j) of Algs. 1-3 folded in.
#include <cuda.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace fmm {
namespace gemm {

// ------------------------------------------------------------ TMA / bulk copies

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 2-D tiled bulk tensor copy global -> shared, completion counted on *bar.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// The same copy for a CTA pair: the destination is this CTA's shared
// memory, the completion is counted on the barrier at `bar_cluster` (a
// cluster address, the leader's barrier for both CTAs).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, int32_t x, int32_t y,
                                                 uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cluster)
      : "memory");
}

// 2-D tiled bulk tensor copy shared -> global (one box of the map from
// `src`, 1024-byte aligned for the 128-byte swizzle), in this thread's
// current bulk async-group.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int32_t x, int32_t y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Until at most N of this thread's bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// Until at most N of this thread's bulk groups are incomplete.
template <int N>
__device__ __forceinline__ void bulk_wait() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}
// This thread's shared-memory writes become visible to bulk copies.
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
      const int* eb = c.eB ? c.eB + gj0 : nullptr;
      const bool eb_vec = ((uintptr_t)eb & 15) == 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float4 v;
        float* vp = reinterpret_cast<float*>(&v);
        int4 e4 = make_int4(0, 0, 0, 0);
        if (eb) {
          if (eb_vec) e4 = __ldg(reinterpret_cast<const int4*>(eb + 4 * q));
          else e4 = make_int4(__ldg(eb + 4 * q), __ldg(eb + 4 * q + 1), __ldg(eb + 4 * q + 2), __ldg(eb + 4 * q + 3));
        }
        const int ev[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float x = s * __uint_as_float(r[4 * q + u]);
          if (eb) x *= exp2i(ev[u]);
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

// The same terms added into C by atomic FP32 additions (the accumulating
// epilogue: C starts at zero and every leaf's units may run on any CTA, in
// any order).
__device__ __forceinline__ void red_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

__device__ __forceinline__ void epi_chunk_red(const EpilogueArgs& c, const LeafDesc* L, int64_t ml, int64_t nl0,
                                              const uint32_t (&r)[32]) {
  const int nc = __ldg(&L->nc);
  for (int t = 0; t < nc; ++t) {
    const int32_t blk = __ldg(&L->c_blk[t]);
    const int64_t bi = (blk >> 16) & 0xFFFF, bj = blk & 0xFFFF;
    const int64_t gi = bi * c.bm + ml;
    if (gi >= c.M) continue;
    const float coef = __ldg(&L->c_coef[t]);
    const float s = c.eA ? coef * exp2i(__ldg(c.eA + gi)) : coef;
    const int64_t gj0 = bj * c.bn + nl0;
    float* crow = c.C + gi * c.ldc;
    if (c.vec_ok && nl0 + 32 <= c.bn && gj0 + 32 <= c.N) {
      const int* eb = c.eB ? c.eB + gj0 : nullptr;
      const bool eb_vec = ((uintptr_t)eb & 15) == 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        int4 e4 = make_int4(0, 0, 0, 0);
        if (eb) {
          if (eb_vec) e4 = __ldg(reinterpret_cast<const int4*>(eb + 4 * q));
          else e4 = make_int4(__ldg(eb + 4 * q), __ldg(eb + 4 * q + 1), __ldg(eb + 4 * q + 2), __ldg(eb + 4 * q + 3));
        }
        float x0 = s * __uint_as_float(r[4 * q]), x1 = s * __uint_as_float(r[4 * q + 1]);
        float x2 = s * __uint_as_float(r[4 * q + 2]), x3 = s * __uint_as_float(r[4 * q + 3]);
        if (eb) {
          x0 *= exp2i(e4.x);
          x1 *= exp2i(e4.y);
          x2 *= exp2i(e4.z);
          x3 *= exp2i(e4.w);
        }
        red_v4(crow + gj0 + 4 * q, x0, x1, x2, x3);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int64_t nl = nl0 + j, gj = gj0 + j;
        if (nl < c.bn && gj < c.N) {
          float x = s * __uint_as_float(r[j]);
          if (c.eB) x *= exp2i(__ldg(c.eB + gj));
          atomicAdd(crow + gj, x);
        }
      }
    }
  }
}

}  // namespace gemm
}  // namespace fmm
