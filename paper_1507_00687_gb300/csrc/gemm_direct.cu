// Leaf products over combined operands (Eq. 4.4, second and third lines):
// M_r = S_r T_r on the tensor cores, C(c_blk) += w 2^(eA+eB) M_r in the
// epilogue, for operands the combination pass already formed in the leaf
// format.  There is no arithmetic between memory and the tensor cores, so
// the kernel is the plain warp-specialised tcgen05 pipeline:
//
//   warps 0..E-1  epilogue (E = 4 or 8): TMEM -> registers, C(blk) = / +=
//              coef 2^(eA+eB) M_r; warp w reads the tile rows of TMEM lanes
//              32 (w mod 4) .. + 31 (the lanes a warp may access) and, with
//              E = 8, column half w / 4.  Eight warps where the epilogue
//              unscales and adds into C (fused epilogue, batches: measured
//              1.6 ms faster on a 512-product batch); four where it only
//              stores M_r (measured 3% faster there)
//   warp E     lane 0: TMEM allocator and single-thread tcgen05.mma issuer
//   warp E+1   lane 0: TMA issuer: bulk tensor copies of each operand plane
//              and stage straight into the 128-byte-swizzled layout the MMA
//              descriptors read (K-major: one 64 k x rows box; MN-major: one
//              64 t x 64 k box per 64 rows)
//
// One CTA per SM, persistent over work units, each one BM x BN tile of one
// leaf product.  Two orders:
//   fused epilogue (args.mbuf null): a CTA owns a tile position and visits
//     every leaf for it in leaf order, adding w 2^(eA+eB) M_r into C in its
//     epilogue, so each C element is updated by one thread in a fixed order
//     (deterministic);
//   stored products (args.mbuf set): units (leaf, tile) are spread over all
//     CTAs and the epilogue stores the fp32 tile of M_r; the output
//     combination pass then forms C.  For plans with few tiles per leaf
//     (deep recursion, small products) this keeps every SM busy.
// The fp32 accumulator is double-buffered in TMEM so the epilogue of one
// unit overlaps the products of the next.  Every mbarrier wait is bounded
// (globaltimer); on expiry the kernel sets the timeout bit of the status
// word, stops all roles, waits for its own copies and MMAs, frees its TMEM
// and returns.
#include <algorithm>
#include <cstring>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/fmm.h"
#include "device.cuh"
#include "gemm_common.cuh"
#include "kernels.h"

namespace fmm {
namespace direct {

using gemm::epi_chunk;
using gemm::mbar_arrive_expect_tx;
using gemm::tma_load_2d;

constexpr int BM = 128;

// K per stage: 64 (128-byte rows); the kernel also supports 32 (64-byte
// rows, a deeper ring of smaller stages), which measured slower.
template <int FMT, int BN>
struct Cfg {
  static constexpr int BK = 64;
  static constexpr int kSplit = FMT == FMM_LEAF_BF16X3 ? 2 : 1;
  static constexpr int kATile = BM * BK * 2;
  static constexpr int kBTile = BN * BK * 2;
  static constexpr int kStage = kSplit * (kATile + kBTile);
  static constexpr int kStages = (220 * 1024) / kStage > 8 ? 8 : (220 * 1024) / kStage;
  static constexpr int kTmemCols = 2 * BN;
  static constexpr int kBarBytes = 256;
  static constexpr int kSmem = kStages * kStage + kBarBytes + 1024;  // + alignment slack
};

// Operand tile of `rows` t x BK k from plane row block `blk` (= plane R +
// leaf) at t offset t0, k offset k0, into dst.  MN-major: one 64 t x BK k
// box (BK rows of 128 bytes) per 64 t.
template <bool MN, int BK>
__device__ __forceinline__ void load_tile(uint8_t* dst, const CUtensorMap* map, int rows, int64_t blk, int64_t tp,
                                          int64_t kp, int64_t t0, int64_t k0, uint64_t* bar) {
  if constexpr (MN) {
    for (int c = 0; c < rows / 64; ++c)
      tma_load_2d(dst + c * (BK * 128), map, (int32_t)(t0 + 64 * c), (int32_t)(blk * kp + k0), bar);
  } else {
    tma_load_2d(dst, map, (int32_t)k0, (int32_t)(blk * tp + t0), bar);
  }
}

// Descriptor of the 16-wide k step k16 of an operand tile at saddr:
// MN-major advances two 8-k groups (2048 bytes); K-major advances 32 bytes
// inside the swizzled row (128-byte rows for BK 64, 64-byte rows for 32).
template <bool MN, int BK>
__device__ __forceinline__ uint64_t tile_desc(uint32_t saddr, int k16) {
  if constexpr (MN) return smem_desc_mn_sw128(saddr + k16 * 2048, BK * 128);
  else if constexpr (BK == 64) return smem_desc_sw128(saddr + k16 * 32);
  else return smem_desc_sw64(saddr + k16 * 32);
}

// What one launch covers: one problem (`one`), or, when `tab` is set, the
// `count` problems of a batch whose (leaf, tile) units are numbered
// consecutively: units of problem p are [unit_start[p], unit_start[p + 1]).
// Batched problems always store their leaf products.
struct DirectLaunch {
  DirectArgs one;
  const DirectArgs* tab;
  const int64_t* unit_start;
  int count;
  int64_t total_units;
};

__device__ __forceinline__ int find_unit_problem(const int64_t* start, int count, int64_t u) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int FMT, int BN, bool A_MN, bool B_MN, int EPI>
__global__ void __launch_bounds__((EPI + 2) * 32, 1) direct_fmm_kernel(const __grid_constant__ DirectLaunch launch) {
  constexpr int kEpiWarps = EPI, kMmaWarp = EPI, kTmaWarp = EPI + 1;
  const DirectArgs& args = launch.one;  // the single problem (status, timeout for both forms)
  using C = Cfg<FMT, BN>;
  constexpr int BK = C::BK;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kStages * C::kStage);
  uint64_t* empty = full + C::kStages;
  uint64_t* tfull = empty + C::kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint64_t* never = drain + 1;  // no thread ever arrives here (timeout-path test)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps * 32);
    }
    mbar_init(drain, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == kMmaWarp) tmem_alloc(tmem_slot, C::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // the set-up above overlaps the previous kernel's tail; its outputs (the
  // combined operands) are read from here on
  pdl_wait();
  pdl_trigger();

  // Work units of this CTA: global units u = blockIdx.x, + gridDim.x, ...;
  // a unit is one tile of one leaf product (problems with stored products)
  // or one tile with all its leaves in leaf order (fused epilogue).
  const bool batched = launch.tab != nullptr;
  const int64_t total_units = batched ? launch.total_units
                                      : (args.tp_a / BM) * (args.tp_b / BN) * (args.mbuf ? args.num_leaves : 1);
  struct Cursor {
    int64_t u, leaf, leaf_end, tm, tn, kt;
    const DirectArgs* a;
  };
  auto decode = [&](Cursor& c) {
    if (c.u >= total_units) return;
    int64_t local;
    if (batched) {
      const int p = find_unit_problem(launch.unit_start, launch.count, c.u);
      c.a = launch.tab + p;
      local = c.u - __ldg(launch.unit_start + p);
    } else {
      c.a = &args;
      local = c.u;
    }
    const int64_t ntn = c.a->tp_b / BN, ntiles = (c.a->tp_a / BM) * ntn;
    int64_t tile;
    if (c.a->mbuf) {
      c.leaf = local / ntiles;
      c.leaf_end = c.leaf + 1;
      tile = local % ntiles;
    } else {
      c.leaf = 0;
      c.leaf_end = c.a->num_leaves;
      tile = local;
    }
    c.tm = tile / ntn;
    c.tn = tile % ntn;
    c.kt = c.a->kp / BK;
  };
  auto first = [&]() {
    Cursor c;
    c.u = blockIdx.x;
    decode(c);
    return c;
  };
  auto advance = [&](Cursor& c) {
    if (++c.leaf >= c.leaf_end) {
      c.u += gridDim.x;
      decode(c);
    }
  };

  if (warp == kTmaWarp) {
    if (lane == 0) {
      // ------------------------------------------------------ TMA issuer
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      uint32_t armed = 0, armed_parity = 0;  // per stage: copy issued, parity it completes
      for (Cursor w = first(); w.u < total_units && ok; advance(w)) {
        const DirectArgs& a = *w.a;
        const int64_t NL = a.num_leaves;
        for (int64_t kt = 0; kt < w.kt && ok; ++kt) {
          if (!mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, args.timeout_ns)) { ok = false; break; }
          uint8_t* st = smem + stage * C::kStage;
          mbar_arrive_expect_tx(&full[stage], (uint32_t)C::kStage);
          const int64_t k0 = kt * BK, ta = w.tm * BM, tb = w.tn * BN;
          load_tile<A_MN, BK>(st, &a.map_a, BM, w.leaf, a.tp_a, a.kp, ta, k0, &full[stage]);
          load_tile<B_MN, BK>(st + C::kSplit * C::kATile, &a.map_b, BN, w.leaf, a.tp_b, a.kp, tb, k0, &full[stage]);
          if constexpr (C::kSplit == 2) {
            load_tile<A_MN, BK>(st + C::kATile, &a.map_a, BM, NL + w.leaf, a.tp_a, a.kp, ta, k0, &full[stage]);
            load_tile<B_MN, BK>(st + 2 * C::kATile + C::kBTile, &a.map_b, BN, NL + w.leaf, a.tp_b, a.kp, tb, k0,
                                &full[stage]);
          }
          armed |= 1u << stage;
          armed_parity = (armed_parity & ~(1u << stage)) | (phase << stage);
          if (++stage == C::kStages) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) *abort_flag = 1;
      // No copy may still be writing shared memory when the CTA exits: wait
      // (1 s cap each) for every issued copy.
      for (int s = 0; s < C::kStages; ++s) {
        if (armed & (1u << s)) {
          const uint64_t t0 = globaltimer_ns();
          while (!mbar_try_wait(&full[s], (armed_parity >> s) & 1u) && globaltimer_ns() - t0 < 1000000000ull) {
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // ------------------------------------------------------ MMA issuer
      constexpr uint32_t idesc = idesc_f16(FMT == FMM_LEAF_F16 ? 0u : 1u, BM, BN, A_MN, B_MN);
      int stage = 0;
      uint32_t phase = 0, acc_iter = 0;
      bool ok = true;
      const uint32_t sbase = smem_u32(smem);
      for (Cursor w = first(); w.u < total_units && ok; advance(w)) {
        {
          const int64_t KT = w.kt;
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
              const uint64_t ah = tile_desc<A_MN, BK>(a_hi, k16), bh = tile_desc<B_MN, BK>(b_hi, k16);
              mma_f16(d_tmem, ah, bh, idesc, acc);
              if constexpr (C::kSplit == 2) {
                mma_f16(d_tmem, ah, tile_desc<B_MN, BK>(b_lo, k16), idesc, 1u);
                mma_f16(d_tmem, tile_desc<A_MN, BK>(a_lo, k16), bh, idesc, 1u);
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
      // All issued MMAs complete before TMEM is released (own 1 s cap: MMAs
      // never wait on anything).
      mma_commit(drain);
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(drain, 0) && globaltimer_ns() - t0 < 1000000000ull) {
      }
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------- epilogue
    uint32_t acc_iter = 0;
    bool ok = true;
    if (args.stall_test) ok = __all_sync(0xffffffffu, mbar_wait_bounded(never, 0, abort_flag, args.timeout_ns));
    const int quarter = warp & 3, half = EPI == 8 ? warp >> 2 : 0;
    constexpr int kChunks = BN / 32 / (EPI / 4);  // 32-column chunks per warp
    const int row = quarter * 32 + lane;  // TMEM lane = tile row
    for (Cursor w = first(); w.u < total_units && ok; advance(w)) {
      const DirectArgs& a = *w.a;
      const bool store_m = a.mbuf != nullptr;
      const int64_t leaf = w.leaf, tn = w.tn;
      const int64_t ml = w.tm * BM + row;
      const uint32_t buf = acc_iter & 1u, aph = (acc_iter >> 1) & 1u;
      // warp-uniform outcome: the TMEM loads below are .sync.aligned
      ok = __all_sync(0xffffffffu, mbar_wait_bounded(&tfull[buf], aph, abort_flag, args.timeout_ns));
      if (!ok) break;
      tc_fence_after();
      const LeafDesc* L = a.leaves + leaf;
      // stored products: M_r (padded tp_a x tp_b, fp32) row ml, from column tn BN
      float* mrow = store_m ? a.mbuf + (leaf * a.tp_a + ml) * a.tp_b + tn * BN : nullptr;
#pragma unroll 1
      for (int cc = half * kChunks; cc < (half + 1) * kChunks; ++cc) {
        uint32_t r[32];
        tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) + buf * BN + cc * 32, r);
        if (store_m) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            *reinterpret_cast<uint4*>(mrow + cc * 32 + 4 * q) =
                make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
        } else if (ml < a.c.bm) {
          epi_chunk(a.c, L, ml, tn * BN + cc * 32, r);
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[buf]);
      ++acc_iter;
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
template <int FMT, int BN, bool A_MN, bool B_MN, int EPI>
cudaError_t launch_cfg(const DirectArgs& a, const DirectArgs* tab, const int64_t* unit_start, int count,
                       int64_t total_units, cudaStream_t st) {
  using C = Cfg<FMT, BN>;
  auto kern = direct_fmm_kernel<FMT, BN, A_MN, B_MN, EPI>;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  DirectLaunch L;
  std::memset(&L, 0, sizeof(L));
  int64_t units;
  if (tab) {
    L.one = a;  // status and timeout
    L.tab = tab;
    L.unit_start = unit_start;
    L.count = count;
    L.total_units = total_units;
    units = total_units;
  } else {
    if (a.tp_a % BM != 0 || a.tp_b % BN != 0 || a.kp % C::BK != 0) return cudaErrorInvalidValue;
    const int64_t ntiles = (a.tp_a / BM) * (a.tp_b / BN);
    if (ntiles == 0 || a.num_leaves == 0) return cudaSuccess;
    L.one = a;
    units = a.mbuf ? ntiles * a.num_leaves : ntiles;
  }
  if (units == 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>(units, device_sm_count());
  KernelTimer timer("multiply", st);
  return launch_pdl(kern, dim3((unsigned)grid), dim3((EPI + 2) * 32), C::kSmem, st, L);
}

// Operand layouts used: forward (A K-major, B MN-major), dA = dC B^T (both
// K-major), dB = A^T dC (both MN-major).
template <int FMT, int BN>
cudaError_t launch_layout(const DirectArgs& a, const DirectArgs* tab, const int64_t* us, int count, int64_t total,
                          cudaStream_t st) {
  if (!a.a_mn && a.b_mn) {
    // forward products: eight epilogue warps where the epilogue adds into C
    if (tab || !a.mbuf) return launch_cfg<FMT, BN, false, true, 8>(a, tab, us, count, total, st);
    return launch_cfg<FMT, BN, false, true, 4>(a, tab, us, count, total, st);
  }
  if (!a.a_mn && !a.b_mn) return launch_cfg<FMT, BN, false, false, 4>(a, tab, us, count, total, st);
  if (a.a_mn && a.b_mn) return launch_cfg<FMT, BN, true, true, 4>(a, tab, us, count, total, st);
  return cudaErrorNotSupported;
}

template <int BN>
cudaError_t launch_bn(const DirectArgs& a, int fmt, const DirectArgs* tab, const int64_t* us, int count,
                      int64_t total, cudaStream_t st) {
  switch (fmt) {
    case FMM_LEAF_BF16: return launch_layout<FMM_LEAF_BF16, BN>(a, tab, us, count, total, st);
    case FMM_LEAF_F16: return launch_layout<FMM_LEAF_F16, BN>(a, tab, us, count, total, st);
    default: return launch_layout<FMM_LEAF_BF16X3, BN>(a, tab, us, count, total, st);
  }
}

}  // namespace direct

int direct_gemm_bk(int leaf_format) {
  return leaf_format == FMM_LEAF_BF16X3 ? direct::Cfg<FMM_LEAF_BF16X3, 256>::BK : direct::Cfg<FMM_LEAF_BF16, 256>::BK;
}

cudaError_t launch_direct_gemm(const DirectArgs& a, int leaf_format, int bn, cudaStream_t st) {
  return bn == 256 ? direct::launch_bn<256>(a, leaf_format, nullptr, nullptr, 0, 0, st)
                   : direct::launch_bn<128>(a, leaf_format, nullptr, nullptr, 0, 0, st);
}

cudaError_t launch_direct_gemm_batched(const DirectArgs& layout, const DirectArgs* tab, const int64_t* unit_start,
                                       int count, int64_t total_units, int leaf_format, int bn, cudaStream_t st) {
  if (count == 0 || total_units == 0) return cudaSuccess;
  return bn == 256 ? direct::launch_bn<256>(layout, leaf_format, tab, unit_start, count, total_units, st)
                   : direct::launch_bn<128>(layout, leaf_format, tab, unit_start, count, total_units, st);
}

}  // namespace fmm
