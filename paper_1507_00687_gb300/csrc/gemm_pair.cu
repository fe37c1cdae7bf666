// Leaf products on CTA pairs (Eq. 4.4, second and third lines): the same
// work units as the one-CTA multiply kernel (gemm_direct.cu) with 256 x 256
// tiles shared by two CTAs on neighbouring SMs (a cluster of two):
// tcgen05.mma.cta_group::2 with M = 256 takes A rows 0..127 from the
// leader's shared memory and 128..255 from the peer's, B columns 0..127
// from the leader's and 128..255 from the peer's, and writes each CTA's
// 128 x 256 FP32 accumulator into its own TMEM.  Per CTA a 64-wide K stage
// is 16 KB of A and 16 KB of B (32 KB, one plane) for a 128 x 256 x 64
// share of the products, where the one-CTA 128 x 256 tile needs 48 KB: a
// third less operand traffic from L2 and through shared memory per flop.
//
//   warps 0..E-1  epilogue of this CTA's 128 tile rows (TMEM lane quarters,
//                 and with E = 8 column halves), as in the one-CTA kernel
//   warp E        lane 0: TMEM allocation (both CTAs, together); in the
//                 leader, the single-thread MMA issuer
//   warp E+1      lane 0: TMA issuer for this CTA's halves of A and B; each
//                 copy counts its bytes on the leader's stage barrier
//
// Protocol (barriers at the same offsets in both CTAs):
//   full[s]   leader only: the leader's producer expects both CTAs' bytes,
//             both producers' copies complete on it;
//   empty[s]  each CTA: the leader's MMA commit arrives on both (multicast);
//   tfull[b]  each CTA: the leader's commit after a unit's last MMA;
//   tempty[b] leader only: one arrival per epilogue warp of both CTAs.
// Every wait is bounded (globaltimer, the status word's timeout bit on
// expiry); a CTA that stops sets its own and its peer's abort flag.  Both
// CTAs leave through one path: after their roles end they wait (bounded)
// for their own outstanding work, meet at a cluster barrier -- reached by
// every thread of both CTAs, since every loop before it is bounded -- and
// only then free TMEM and exit, so neither exits while the other may still
// touch its shared memory or TMEM.
#include <algorithm>
#include <cstring>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/fmm.h"
#include "device.cuh"
#include "gemm_common.cuh"
#include "kernels.h"

namespace fmm {
namespace pair {

using gemm::epi_chunk;
using gemm::epi_chunk_red;
using gemm::mbar_arrive_expect_tx;
using gemm::tma_load_2d_pair;
using gemm::bulk_commit;
using gemm::bulk_wait;
using gemm::bulk_wait_read;
using gemm::fence_proxy_async_shared;
using gemm::tma_store_2d;

constexpr int BM = 256, BN = 256;  // tile of the pair
constexpr int HM = 128, HN = 128;  // this CTA's rows of A, columns of B

// Pipeline depth: the most 64-wide K stages that fit in 212 KB, less
// FMM_PAIR_SINGLE_STAGE_CUT for one product and FMM_PAIR_BATCH_STAGE_CUT for
// batches (never below three), which leaves the rest of the SM's 256 KB of
// shared memory and L1 to L1.  Measured on the 512-product batch (bf16):
// six stages and a 2048-entry unit cache 706 TFLOP/s, five 737, four with a
// 1024-entry cache 745; without the cache 696-703.
#ifndef FMM_PAIR_SINGLE_STAGE_CUT
#define FMM_PAIR_SINGLE_STAGE_CUT 0
#endif
#ifndef FMM_PAIR_BATCH_STAGE_CUT
#define FMM_PAIR_BATCH_STAGE_CUT 2
#endif
#ifndef FMM_PAIR_UNIT_CACHE
#define FMM_PAIR_UNIT_CACHE 1024
#endif

template <int FMT, bool BATCH = false, bool TSTORE = false>
struct Cfg {
  static constexpr int BK = 64;
  static constexpr int kSplit = FMT == FMM_LEAF_BF16X3 ? 2 : 1;
  static constexpr int kATile = HM * BK * 2;
  static constexpr int kBTile = HN * BK * 2;
  static constexpr int kStage = kSplit * (kATile + kBTile);
  static constexpr int kStagesMax = (212 * 1024) / kStage > 8 ? 8 : (212 * 1024) / kStage;
  static constexpr int kCut = BATCH ? FMM_PAIR_BATCH_STAGE_CUT : FMM_PAIR_SINGLE_STAGE_CUT;
  static constexpr int kStages = kStagesMax - kCut >= 3 ? kStagesMax - kCut : (kStagesMax < 3 ? kStagesMax : 3);
  static constexpr int kTmemCols = 2 * BN;
  static constexpr int kBarBytes = 256;
  static constexpr int kUnitCache = BATCH ? FMM_PAIR_UNIT_CACHE : 0;  // batch unit table entries in shared memory
  // TSTORE: two 32 x 32 fp32 staging buffers (4 KB, 128-byte swizzle) per
  // epilogue warp (four for one product, eight for batches) for bulk
  // tensor stores of M_r or C
  static constexpr int kEpiBuf = TSTORE ? (BATCH ? 8 : 4) * 2 * 4096 : 0;
  // + alignment slack
  static constexpr int kSmem = kStages * kStage + kEpiBuf + kBarBytes + kUnitCache * 8 + 1024;
  static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
};

// The configuration of one kernel instantiation: single products with four
// epilogue warps store M_r, and batches (eight epilogue warps, 16-bit
// leaves: bf16x3 stages leave no room) store the C of their direct entries,
// by bulk tensor stores.  The kernel and its launcher both take it from
// here, so the shared memory the launch gives is the layout the kernel uses.
template <int FMT, bool BATCH, int EPI>
using CfgFor = Cfg<FMT, BATCH, BATCH ? (EPI == 8 && FMT != FMM_LEAF_BF16X3) : EPI == 4>;

__device__ __forceinline__ uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}

// This CTA's half of an operand tile: `rows` t x BK k from plane row block
// `blk` at t offset t0, k offset k0 (MN-major: one 64 t x BK k box per 64 t).
template <bool MN, int BK>
__device__ __forceinline__ void load_half(uint8_t* dst, const CUtensorMap* map, int rows, int64_t blk, int64_t tp,
                                          int64_t kp, int64_t t0, int64_t k0, uint32_t bar) {
  if constexpr (MN) {
    for (int c = 0; c < rows / 64; ++c)
      tma_load_2d_pair(dst + c * (BK * 128), map, (int32_t)(t0 + 64 * c), (int32_t)(blk * kp + k0), bar);
  } else {
    tma_load_2d_pair(dst, map, (int32_t)k0, (int32_t)(blk * tp + t0), bar);
  }
}

template <bool MN, int BK>
__device__ __forceinline__ uint64_t tile_desc(uint32_t saddr, int k16) {
  if constexpr (MN) return smem_desc_mn_sw128(saddr + k16 * 2048, BK * 128);
  else return smem_desc_sw128(saddr + k16 * 32);
}

// What one launch covers: one problem (`one`), or, when `tab` is set, the
// `count` problems of a batch (device table, one DirectArgs each, tensor
// maps included) whose units are numbered consecutively: units of problem
// p are [unit_start[p], unit_start[p + 1]).  `one` also gives the status
// word, the wait limit and the stall test for both forms.
struct PairLaunch {
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

// BATCH: the launch covers a batch's problems (`tab`); otherwise one
// problem, whose arguments every role reads from the launch itself.
template <int FMT, bool A_MN, bool B_MN, int EPI, bool BATCH>
__global__ void __launch_bounds__((EPI + 2) * 32, 1) pair_fmm_kernel(const __grid_constant__ PairLaunch launch) {
  const DirectArgs& args = launch.one;
  constexpr int kMmaWarp = EPI, kTmaWarp = EPI + 1;
  using C = CfgFor<FMT, BATCH, EPI>;
  constexpr bool kTStore = C::kEpiBuf > 0;
  constexpr int BK = C::BK;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* epibuf = smem + C::kStages * C::kStage;  // 1024-aligned
  uint64_t* full = reinterpret_cast<uint64_t*>(epibuf + C::kEpiBuf);
  uint64_t* empty = full + C::kStages;
  uint64_t* tfull = empty + C::kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint64_t* never = drain + 1;  // no thread ever arrives here (timeout-path test)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int64_t* ustart = reinterpret_cast<int64_t*>(epibuf + C::kEpiBuf + C::kBarBytes);

  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 2 * EPI);
    }
    mbar_init(drain, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == kMmaWarp) tmem_alloc_pair(tmem_slot, C::kTmemCols);
  tc_fence_before();
  __syncthreads();
  // both CTAs' barriers exist before either CTA signals the other's
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t peer_abort = mapa_shared(smem_u32((const void*)abort_flag), rank ^ 1u);
  auto stop = [&]() {
    *abort_flag = 1;
    st_cluster_u32(peer_abort, 1u);
  };
  // the combined operands of the previous kernel are read from here on
  pdl_wait();
  pdl_trigger();
  // a batch's unit numbering, in shared memory when it fits
  const bool ucached = BATCH && launch.count + 1 <= C::kUnitCache;
  if (ucached)
    for (int i = threadIdx.x; i <= launch.count; i += blockDim.x) ustart[i] = __ldg(launch.unit_start + i);
  __syncthreads();

  // Units of this pair: u = cluster id, + cluster count, ...; one 256 x 256
  // tile of one leaf (stored products) or one tile position with all its
  // leaves in leaf order (fused epilogue).
  auto units_of = [&](const DirectArgs& a) {
    const int64_t nt = (a.tm_count ? a.tm_count : a.tp_a / BM) * (a.tp_b / BN);
    return (a.mbuf || a.accumulate) ? nt * a.num_leaves : nt;
  };
  const int64_t total_units = BATCH ? launch.total_units : units_of(args);
  const int64_t u0 = cluster_id_x(), ustep = cluster_count_x();
  struct Cursor {
    int64_t u, leaf, leaf_end, tm, tn, kt;
    const DirectArgs* a;
    int p;  // batch: problem of unit u (each role walks its units in increasing order)
  };
  // the problem a cursor's unit belongs to
  auto prob = [&](const Cursor& c) -> const DirectArgs& {
    if constexpr (BATCH) return *c.a;
    else return args;
  };
  auto decode = [&](Cursor& c) {
    if (c.u >= total_units) return;
    int64_t local;
    if constexpr (BATCH) {
      if (ucached) {
        while (c.p + 1 < launch.count && ustart[c.p + 1] <= c.u) ++c.p;
        local = c.u - ustart[c.p];
      } else {
        c.p = find_unit_problem(launch.unit_start, launch.count, c.u);
        local = c.u - __ldg(launch.unit_start + c.p);
      }
      c.a = launch.tab + c.p;
    } else {
      c.a = &args;
      local = c.u;
    }
    const DirectArgs& a = prob(c);
    const int64_t ntn = a.tp_b / BN, ntiles = (a.tm_count ? a.tm_count : a.tp_a / BM) * ntn;
    int64_t tile;
    if (a.mbuf || a.accumulate) {  // units are (leaf, tile)
      c.leaf = local / ntiles;
      c.leaf_end = c.leaf + 1;
      tile = local % ntiles;
    } else {
      c.leaf = 0;
      c.leaf_end = a.num_leaves;
      tile = local;
    }
    c.tm = a.tm_begin + tile / ntn;
    c.tn = tile % ntn;
    c.kt = a.kp / BK;
  };
  auto first = [&]() {
    Cursor c;
    c.u = u0;
    c.p = 0;
    decode(c);
    return c;
  };
  auto advance = [&](Cursor& c) {
    if (++c.leaf >= c.leaf_end) {
      c.u += ustep;
      decode(c);
    }
  };

  if (warp == kTmaWarp) {
    if (lane == 0) {
      // ------------------------------------------------------ TMA issuer
      const uint32_t full0 = mapa_shared(smem_u32(&full[0]), 0u);  // the leader's stage barriers
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      uint32_t armed = 0, armed_parity = 0;  // leader: per stage, expecting bytes, parity it completes
      for (Cursor w = first(); w.u < total_units && ok; advance(w)) {
        const DirectArgs& a = prob(w);
        const int64_t NL = a.num_leaves;
        for (int64_t kt = 0; kt < w.kt && ok; ++kt) {
          if (!mbar_wait_bounded_cluster(&empty[stage], phase ^ 1u, abort_flag, args.timeout_ns)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + stage * C::kStage;
          const uint32_t fb = full0 + 8u * (uint32_t)stage;
          if (leader) mbar_arrive_expect_tx(&full[stage], 2u * (uint32_t)C::kStage);
          const int64_t k0 = kt * BK, ta = w.tm * BM + rank * HM, tb = w.tn * BN + rank * HN;
          load_half<A_MN, BK>(st, &a.map_a, HM, w.leaf, a.tp_a, a.kp, ta, k0, fb);
          load_half<B_MN, BK>(st + C::kSplit * C::kATile, &a.map_b, HN, w.leaf, a.tp_b, a.kp, tb, k0, fb);
          if constexpr (C::kSplit == 2) {
            load_half<A_MN, BK>(st + C::kATile, &a.map_a, HM, NL + w.leaf, a.tp_a, a.kp, ta, k0, fb);
            load_half<B_MN, BK>(st + 2 * C::kATile + C::kBTile, &a.map_b, HN, NL + w.leaf, a.tp_b, a.kp, tb, k0,
                                fb);
          }
          if (leader) {
            armed |= 1u << stage;
            armed_parity = (armed_parity & ~(1u << stage)) | (phase << stage);
          }
          if (++stage == C::kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) stop();
      // The leader's stage barriers complete only when both CTAs' copies
      // have landed: wait (1 s cap each) for every stage it armed.
      for (int s = 0; s < C::kStages; ++s) {
        if (armed & (1u << s)) {
          const uint64_t t0 = globaltimer_ns();
          while (!mbar_try_wait_cluster(&full[s], (armed_parity >> s) & 1u) &&
                 globaltimer_ns() - t0 < 1000000000ull) {
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    if (lane == 0 && leader) {
      // ------------------------------------------------------ MMA issuer
      constexpr uint32_t idesc = idesc_f16(FMT == FMM_LEAF_F16 ? 0u : 1u, BM, BN, A_MN, B_MN);
      int stage = 0;
      uint32_t phase = 0, acc_iter = 0;
      bool ok = true;
      const uint32_t sbase = smem_u32(smem);
      for (Cursor w = first(); w.u < total_units && ok; advance(w)) {
        const uint32_t buf = acc_iter & 1u, aph = (acc_iter >> 1) & 1u;
        if (!mbar_wait_bounded_cluster(&tempty[buf], aph ^ 1u, abort_flag, args.timeout_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + buf * BN;
        for (int64_t kt = 0; kt < w.kt; ++kt) {
          if (!mbar_wait_bounded_cluster(&full[stage], phase, abort_flag, args.timeout_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_hi = sbase + stage * C::kStage;
          const uint32_t a_lo = a_hi + C::kATile;
          const uint32_t b_hi = a_hi + C::kSplit * C::kATile;
          const uint32_t b_lo = b_hi + C::kBTile;
#pragma unroll
          for (int k16 = 0; k16 < BK / 16; ++k16) {
            const uint32_t acc = (kt > 0 || k16 > 0) ? 1u : 0u;
            const uint64_t ah = tile_desc<A_MN, BK>(a_hi, k16), bh = tile_desc<B_MN, BK>(b_hi, k16);
            mma_f16_pair(d_tmem, ah, bh, idesc, acc);
            if constexpr (C::kSplit == 2) {
              mma_f16_pair(d_tmem, ah, tile_desc<B_MN, BK>(b_lo, k16), idesc, 1u);
              mma_f16_pair(d_tmem, tile_desc<A_MN, BK>(a_lo, k16), bh, idesc, 1u);
            }
          }
          mma_commit_pair(&empty[stage]);
          if (++stage == C::kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit_pair(&tfull[buf]);
        ++acc_iter;
      }
      if (!ok) stop();
      // every issued MMA completes before either CTA frees its TMEM (own
      // 1 s cap: MMAs wait on nothing)
      mma_commit_pair(drain);
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
    const int row = (int)rank * HM + quarter * 32 + lane;  // tile row of this thread (TMEM lane = row mod 128)
    const uint32_t tempty0 = mapa_shared(smem_u32(&tempty[0]), 0u);
    // bulk tensor stores of M_r (stored products) or of C (batch entries
    // whose C is the product itself): this warp's two staging buffers,
    // chunks stored so far (buffer = count mod 2)
    const uint32_t sbuf0 = smem_u32(epibuf) + (uint32_t)(kTStore ? warp * 8192 : 0);
    uint32_t nstored = 0;
    for (Cursor w = first(); w.u < total_units && ok; advance(w)) {
      const DirectArgs& a = prob(w);
      const int64_t leaf = w.leaf, tn = w.tn;
      const int64_t ml = w.tm * BM + row;
      const uint32_t buf = acc_iter & 1u, aph = (acc_iter >> 1) & 1u;
      ok = __all_sync(0xffffffffu, mbar_wait_bounded_cluster(&tfull[buf], aph, abort_flag, args.timeout_ns));
      if (!ok) break;
      tc_fence_after();
      const LeafDesc* L = a.leaves + leaf;
      float* mrow = a.mbuf ? a.mbuf + (leaf * a.tp_a + ml) * a.tp_b + tn * BN : nullptr;
      const bool tstore = kTStore && a.tma_store;
      // C stores: the leaf's single C term's coefficient, rows of this warp
      const float ccoef = (tstore && !a.mbuf) ? __ldg(&L->c_coef[0]) : 1.f;
      const int64_t wrow = w.tm * BM + (int64_t)rank * HM + quarter * 32;
#pragma unroll 1
      for (int cc = half * kChunks; cc < (half + 1) * kChunks; ++cc) {
        uint32_t r[32];
        tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) + buf * BN + cc * 32, r);
        if (kTStore && tstore) {
          const int64_t bx = tn * BN + cc * 32, by = a.mbuf ? leaf * a.tp_a + wrow : wrow;
          // a C box wholly outside C (tile padding) is not stored
          if (a.mbuf || (by < a.c.M && bx < a.c.N)) {
            if (!a.mbuf) {
#pragma unroll
              for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(ccoef * __uint_as_float(r[j]));
            }
            // the store that last used this buffer (two chunks ago) has read it
            if (lane == 0 && nstored >= 2) bulk_wait_read<1>();
            __syncwarp();
            // row `lane` of the 32 x 32 chunk, 16-byte piece q at q xor (row mod 8)
            const uint32_t sb = sbuf0 + (nstored & 1u) * 4096u + (uint32_t)lane * 128u;
#pragma unroll
            for (int q = 0; q < 8; ++q)
              asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sb + (uint32_t)((q ^ (lane & 7)) * 16)),
                           "r"(r[4 * q]), "r"(r[4 * q + 1]), "r"(r[4 * q + 2]), "r"(r[4 * q + 3])
                           : "memory");
            fence_proxy_async_shared();
            __syncwarp();
            if (lane == 0) {
              // the map of M_r (one product) or of this entry's C (batches)
              tma_store_2d(&a.map_m, sbuf0 + (nstored & 1u) * 4096u, (int32_t)bx, (int32_t)by);
              bulk_commit();
            }
            ++nstored;
          }
        } else if (mrow) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            *reinterpret_cast<uint4*>(mrow + cc * 32 + 4 * q) =
                make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
        } else if (ml < a.c.bm) {
          if (a.accumulate) epi_chunk_red(a.c, L, ml, tn * BN + cc * 32, r);
          else epi_chunk(a.c, L, ml, tn * BN + cc * 32, r);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(tempty0 + 8u * buf);
      ++acc_iter;
    }
    if (!ok && lane == 0) stop();
    // every bulk store of this warp complete before the CTA leaves (its
    // shared memory stays valid, its writes visible to the next kernel)
    if (kTStore && lane == 0 && nstored > 0) bulk_wait<0>();
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    // copies or arrivals this CTA issued before stopping land within
    // microseconds; let them before the pair meets for the last time
    const uint64_t t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 200000ull) {
    }
  }
  cluster_sync_all();
  if (*abort_flag && threadIdx.x == 0) atomicOr(args.status, kStatusTimeout);
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, C::kTmemCols);
  }
}

template <int FMT, bool A_MN, bool B_MN, int EPI, bool BATCH>
cudaError_t launch_cfg(const DirectArgs& a, const DirectArgs* tab, const int64_t* unit_start, int count,
                       int64_t total_units, cudaStream_t st) {
  using C = CfgFor<FMT, BATCH, EPI>;
  auto kern = pair_fmm_kernel<FMT, A_MN, B_MN, EPI, BATCH>;
  constexpr int kSmem = C::kSmem;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  PairLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.one = a;
  int64_t units;
  if (BATCH) {
    if (!tab) return cudaErrorInvalidValue;
    L.tab = tab;
    L.unit_start = unit_start;
    L.count = count;
    L.total_units = total_units;
    units = total_units;
  } else {
    if (a.tp_a % BM != 0 || a.tp_b % BN != 0 || a.kp % C::BK != 0) return cudaErrorInvalidValue;
    if (a.tm_count && a.tm_begin + a.tm_count > a.tp_a / BM) return cudaErrorInvalidValue;
    const int64_t ntiles = (a.tm_count ? a.tm_count : a.tp_a / BM) * (a.tp_b / BN);
    if (ntiles == 0 || a.num_leaves == 0) return cudaSuccess;
    units = (a.mbuf || a.accumulate) ? ntiles * a.num_leaves : ntiles;
  }
  if (units == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3((EPI + 2) * 32);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  // as many pairs as can be resident at once (pairs need two SMs of one GPC)
  static int resident[64] = {0};
  if (!resident[dev]) {
    int n = 0;
    cfg.gridDim = dim3((unsigned)(device_sm_count() & ~1));
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = device_sm_count() / 2;
    }
    resident[dev] = n;
  }
  const int64_t pairs = std::min<int64_t>(units, resident[dev]);
  cfg.gridDim = dim3((unsigned)(2 * pairs));
  KernelTimer timer("multiply", st);
  return cudaLaunchKernelEx(&cfg, kern, L);
}

// Operand layouts: forward (A K-major, B MN-major), dA = dC B^T (both
// K-major), dB = A^T dC (both MN-major); eight epilogue warps where the
// epilogue adds into C (fused epilogue, accumulate), four where it stores.
template <int FMT>
cudaError_t launch_fmt(const DirectArgs& a, const DirectArgs* tab, const int64_t* us, int count, int64_t total,
                       cudaStream_t st) {
  if (tab) {  // batches: forward products, unscaling epilogue
    if (!a.a_mn && a.b_mn) return launch_cfg<FMT, false, true, 8, true>(a, tab, us, count, total, st);
    return cudaErrorNotSupported;
  }
  if (!a.a_mn && a.b_mn) {
    if (!a.mbuf) return launch_cfg<FMT, false, true, 8, false>(a, nullptr, nullptr, 0, 0, st);
    return launch_cfg<FMT, false, true, 4, false>(a, nullptr, nullptr, 0, 0, st);
  }
  if (!a.a_mn && !a.b_mn) return launch_cfg<FMT, false, false, 4, false>(a, nullptr, nullptr, 0, 0, st);
  if (a.a_mn && a.b_mn) return launch_cfg<FMT, true, true, 4, false>(a, nullptr, nullptr, 0, 0, st);
  return cudaErrorNotSupported;
}

}  // namespace pair

cudaError_t launch_pair_gemm(const DirectArgs& a, int leaf_format, cudaStream_t st) {
  switch (leaf_format) {
    case FMM_LEAF_BF16: return pair::launch_fmt<FMM_LEAF_BF16>(a, nullptr, nullptr, 0, 0, st);
    case FMM_LEAF_F16: return pair::launch_fmt<FMM_LEAF_F16>(a, nullptr, nullptr, 0, 0, st);
    default: return pair::launch_fmt<FMM_LEAF_BF16X3>(a, nullptr, nullptr, 0, 0, st);
  }
}

cudaError_t launch_pair_gemm_batched(const DirectArgs& layout, const DirectArgs* tab, const int64_t* unit_start,
                                     int count, int64_t total_units, int leaf_format, cudaStream_t st) {
  if (count == 0 || total_units == 0) return cudaSuccess;
  switch (leaf_format) {
    case FMM_LEAF_BF16: return pair::launch_fmt<FMM_LEAF_BF16>(layout, tab, unit_start, count, total_units, st);
    case FMM_LEAF_F16: return pair::launch_fmt<FMM_LEAF_F16>(layout, tab, unit_start, count, total_units, st);
    default: return pair::launch_fmt<FMM_LEAF_BF16X3>(layout, tab, unit_start, count, total_units, st);
  }
}

}  // namespace fmm
