#pragma once
// Fused recursive fast matrix multiplication kernel (sm_103a, tcgen05 + TMA).
//
// One launch runs every leaf of a flattened plan (Eq. 4.4):
//   S_r = sum_t a_coef[t] A(a_blk[t]),  T_r = sum_t b_coef[t] B(b_blk[t]),
//   M_r = S_r T_r,                      C(c_blk[t]) += c_coef[t] M_r,
// and folds the unscale C = 2^eA C' 2^eB of Algs. 1-3 into the last step.
// The operands it reads are "prepared": every leaf block is a whole number of
// 128 x 64 tiles (the host either uses the caller's matrices directly or lets
// the apply pass write scaled, zero-padded copies), so no tile ever crosses a
// block or matrix edge.
//
// CTA roles (384 threads, one CTA per SM, persistent over 128 x 128 output
// tiles of the leaf block grid; a CTA visits every leaf for its tile, in leaf
// order, so each C element is updated by one thread in a fixed order):
//   warps 0-3   epilogue: TMEM -> registers, C(blk) = / += coef 2^(eA+eB) M_r
//   warp 4      lane 0: TMEM allocator and single-thread tcgen05.mma issuer;
//               lane 1: TMA issuer -- one bulk tensor copy per term tile into a
//               ring of shared-memory staging slots
//   warps 5-11  producers: add the staged term tiles in FP32 in index order,
//               round to the leaf format (bf16 / fp16 / bf16 hi+lo) and store
//               the tensor-core operand tiles (A K-major or MN-major, B
//               likewise, 128-byte swizzle).
//
// Every mbarrier wait is bounded (globaltimer); on expiry the kernel sets the
// timeout bit of the status word, stops all roles, waits for its own copies
// and MMAs, frees its TMEM and returns.
#include <cmath>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "gemm_common.cuh"
#include "kernels.h"

namespace fmm {
namespace gemm {

constexpr int BM = 128;  // tile rows (M side) = TMEM lanes
constexpr int BN = 128;  // tile columns (N side)
constexpr int BK = 64;   // K per stage
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kProdWarp0 = 5;
constexpr int kProdWarps = 7;  // 12 warps in all: registers are granted per 4 warps
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kThreads = (kEpiWarps + 1 + kProdWarps) * 32;
constexpr int kChunks = BM * BK / 8;  // 16-byte output units per operand tile (both sides)
constexpr int kChunksPerThread = (kChunks + kProdThreads - 1) / kProdThreads;
constexpr int kSlotBytes = 128 * 64 * 4;  // one staged fp32 term tile

constexpr int kModeBF16 = 0, kModeF16 = 1, kModeBF16x3 = 2;

template <int MODE>
struct Cfg {
  static constexpr int kSplit = MODE == kModeBF16x3 ? 2 : 1;
  static constexpr int kATile = BM * BK * 2;
  static constexpr int kBTile = BN * BK * 2;
  static constexpr int kStage = kSplit * (kATile + kBTile);
  static constexpr int kSlots = MODE == kModeBF16x3 ? 2 : 3;
  static constexpr int kStaging = kSlots * kSlotBytes;
  static constexpr int kStages = (220 * 1024 - kStaging) / kStage > 4 ? 4 : (220 * 1024 - kStaging) / kStage;
  static constexpr int kTmemCols = 2 * BN;  // double-buffered fp32 accumulator
  static constexpr int kBarBytes = 512;
  static constexpr int kSmem = kStages * kStage + kStaging + kBarBytes + 1024;  // + alignment slack
};

// What the TMA issuer tells the producers about each staged tile.
struct SlotInfo {
  float coef;
  int32_t flags;  // kLastA: last A term of its iteration; kLastB: last B term
};
constexpr int kLastA = 1, kLastB = 2;

// ------------------------------------------------------------ smem layouts

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

__device__ __forceinline__ uint32_t pack2(float a, float b, int mode) {
  if (mode == kModeF16) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
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

// Chunk c of a staged term tile: its 8 values.  The staged tile is the TMA
// box in row-major order: KC sides [128 t][64 k], MN sides [64 k][128 t].
// Chunk c covers (t = c / 8, k = 8 (c % 8) ..) for KC and (k = c / 16,
// t = 8 (c % 16) ..) for MN; either way its 8 values are contiguous at
// element offset 8 c.
template <int DT>
__device__ __forceinline__ void read_chunk(const uint8_t* slot, int c, float (&v)[8]) {
  if constexpr (DT == kF32) {
    const float4 a = *reinterpret_cast<const float4*>(slot + c * 32);
    const float4 b = *reinterpret_cast<const float4*>(slot + c * 32 + 16);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
    const uint4 x = *reinterpret_cast<const uint4*>(slot + c * 16);
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      v[2 * t] = __uint_as_float(w[t] << 16);
      v[2 * t + 1] = __uint_as_float(w[t] & 0xFFFF0000u);
    }
  }
}

template <bool KC>
__device__ __forceinline__ uint32_t chunk_smem(int c) {
  if constexpr (KC) {
    return kmajor_off(c >> 3, c & 7);
  } else {
    return mnmajor_off(c >> 4, c & 15);
  }
}

// ------------------------------------------------------------ the kernel

template <int MODE, int DTA, bool KCA, int DTB, bool KCB>
__global__ void __launch_bounds__(kThreads, 1) fused_fmm_kernel(const __grid_constant__ GemmArgs args) {
  using C = Cfg<MODE>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* staging = smem + C::kStages * C::kStage;
  uint64_t* full = reinterpret_cast<uint64_t*>(staging + C::kStaging);
  uint64_t* empty = full + C::kStages;
  uint64_t* sfull = empty + C::kStages;
  uint64_t* sempty = sfull + C::kSlots;
  uint64_t* tfull = sempty + C::kSlots;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  SlotInfo* sinfo = reinterpret_cast<SlotInfo*>(drain + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sinfo + C::kSlots);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], kProdThreads);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < C::kSlots; ++s) {
      mbar_init(&sfull[s], 1);
      mbar_init(&sempty[s], kProdThreads);
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

  const int64_t ntm = args.a.bt / BM;  // prepared block extents are tile multiples
  const int64_t ntn = args.b.bt / BN;
  const int64_t ntiles = ntm * ntn;
  const int64_t KT = args.a.bk / BK;
  const int64_t NL = args.num_leaves;
  const int64_t my_tiles = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
  const int64_t iters = my_tiles * NL * KT;

  if (warp >= kProdWarp0) {
    // ---------------------------------------------------------- producers
    const int ptid = threadIdx.x - kProdWarp0 * 32;
    int stage = 0, slot = 0;
    uint32_t phase = 0, sphase = 0;
    bool ok = true;
    for (int64_t i = 0; i < iters && ok; ++i) {
#pragma unroll 1
      for (int side = 0; side < 2 && ok; ++side) {
        float acc[kChunksPerThread][8];
#pragma unroll
        for (int q = 0; q < kChunksPerThread; ++q)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[q][j] = 0.f;
        // add the side's staged term tiles, in term order
        for (;;) {
          if (!mbar_wait_bounded(&sfull[slot], sphase, abort_flag, args.timeout_ns)) { ok = false; break; }
          const SlotInfo info = sinfo[slot];
          const uint8_t* st = staging + slot * kSlotBytes;
#pragma unroll
          for (int q = 0; q < kChunksPerThread; ++q) {
            const int c = ptid + kProdThreads * q;
            if (c < kChunks) {
              float v[8];
              if (side == 0) read_chunk<DTA>(st, c, v);
              else read_chunk<DTB>(st, c, v);
#pragma unroll
              for (int j = 0; j < 8; ++j) acc[q][j] = fmaf(info.coef, v[j], acc[q][j]);
            }
          }
          mbar_arrive(&sempty[slot]);
          if (++slot == C::kSlots) { slot = 0; sphase ^= 1u; }
          if (info.flags & (side == 0 ? kLastA : kLastB)) break;
        }
        if (!ok) break;
        if (side == 0 && !mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, args.timeout_ns)) {
          ok = false;
          break;
        }
        uint8_t* st = smem + stage * C::kStage;
        uint8_t* hi = side == 0 ? st : st + C::kSplit * C::kATile;
        uint8_t* lo = hi + (side == 0 ? C::kATile : C::kBTile);
#pragma unroll
        for (int q = 0; q < kChunksPerThread; ++q) {
          const int c = ptid + kProdThreads * q;
          if (c < kChunks) {
            const uint32_t off = side == 0 ? chunk_smem<KCA>(c) : chunk_smem<KCB>(c);
            store_unit<MODE>(hi, lo, off, acc[q]);
          }
        }
      }
      if (!ok) break;
      fence_proxy_async_smem();
      mbar_arrive(&full[stage]);
      if (++stage == C::kStages) { stage = 0; phase ^= 1u; }
    }
    if (!ok) *abort_flag = 1;
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // -------------------------------------------------------- MMA issuer
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
      for (int64_t tile = 0; tile < my_tiles && ok; ++tile) {
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
      // All issued MMAs complete before TMEM is released (own 1 s cap: MMAs
      // never wait on anything).
      mma_commit(drain);
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(drain, 0) && globaltimer_ns() - t0 < 1000000000ull) {
      }
    } else if (lane == 1) {
      // -------------------------------------------------------- TMA issuer
      int slot = 0;
      uint32_t sphase = 0;
      bool ok = true;
      uint32_t armed = 0, armed_parity = 0;  // per slot: copy issued, parity it completes
      const int64_t tb_a = args.a.bt, tb_b = args.b.bt, kbx = args.a.bk;
      for (int64_t i = 0; i < iters && ok; ++i) {
        const int64_t tile = blockIdx.x + (i / (NL * KT)) * gridDim.x, r = i % (NL * KT);
        const int64_t leaf = r / KT, kt = r % KT;
        const int64_t tm = tile / ntn, tn = tile % ntn;
        const LeafDesc* L = args.leaves + leaf;
        for (int side = 0; side < 2 && ok; ++side) {
          const int n = side == 0 ? __ldg(&L->na) : __ldg(&L->nb);
          const TileOperand& op = side == 0 ? args.a : args.b;
          const CUtensorMap* map = side == 0 ? &args.map_a : &args.map_b;
          const uint32_t bytes = (uint32_t)(128 * 64 * (op.dtype == kF32 ? 4 : 2));
          for (int t = 0; t < n && ok; ++t) {
            if (!mbar_wait_bounded(&sempty[slot], sphase ^ 1u, abort_flag, args.timeout_ns)) { ok = false; break; }
            const int32_t blk = side == 0 ? __ldg(&L->a_blk[t]) : __ldg(&L->b_blk[t]);
            const int64_t tb = (blk >> op.blk_t_shift) & 0xFFFF, kb = (blk >> op.blk_k_shift) & 0xFFFF;
            const int64_t tpos = tb * (side == 0 ? tb_a : tb_b) + (side == 0 ? tm : tn) * 128;
            const int64_t kpos = kb * kbx + kt * BK;
            SlotInfo info;
            info.coef = side == 0 ? __ldg(&L->a_coef[t]) : __ldg(&L->b_coef[t]);
            info.flags = (t == n - 1) ? (side == 0 ? kLastA : kLastB) : 0;
            sinfo[slot] = info;
            mbar_arrive_expect_tx(&sfull[slot], bytes);
            // KC operands: x = k, y = t;  MN operands: x = t, y = k
            if (op.kcontig) tma_load_2d(staging + slot * kSlotBytes, map, (int32_t)kpos, (int32_t)tpos, &sfull[slot]);
            else tma_load_2d(staging + slot * kSlotBytes, map, (int32_t)tpos, (int32_t)kpos, &sfull[slot]);
            armed |= 1u << slot;
            armed_parity = (armed_parity & ~(1u << slot)) | (sphase << slot);
            if (++slot == C::kSlots) { slot = 0; sphase ^= 1u; }
          }
        }
      }
      if (!ok) *abort_flag = 1;
      // No copy may still be writing shared memory when the CTA exits: wait
      // (1 s cap each) for every issued copy whose slot was not seen free.
      for (int s = 0; s < C::kSlots; ++s) {
        if (armed & (1u << s)) {
          const uint64_t t0 = globaltimer_ns();
          while (!mbar_try_wait(&sfull[s], (armed_parity >> s) & 1u) && globaltimer_ns() - t0 < 1000000000ull) {
          }
        }
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
template <int MODE, int DTA, bool KCA, int DTB, bool KCB>
cudaError_t launch_cfg(const GemmArgs& a, cudaStream_t st) {
  using C = Cfg<MODE>;
  auto kern = fused_fmm_kernel<MODE, DTA, KCA, DTB, KCB>;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const int64_t ntiles = (a.a.bt / BM) * (a.b.bt / BN);
  const int64_t grid = std::min<int64_t>(ntiles, device_sm_count());
  KernelTimer timer("multiply", st);
  kern<<<(unsigned)grid, kThreads, C::kSmem, st>>>(a);
  return cudaGetLastError();
}

// The operand (dtype, layout) pairs the forward and backward passes use:
// forward A (k-contiguous) x B (n-contiguous); dA = dC B^T with both
// operands k-contiguous; dB = A^T dC with both operands t-contiguous.
// Element types fp32 or bf16 (each side independently).
template <int MODE>
cudaError_t launch_mode(const GemmArgs& a, cudaStream_t st) {
  const int da = a.a.dtype, db = a.b.dtype;
  const bool ka = a.a.kcontig != 0, kb = a.b.kcontig != 0;
#define FMM_LAUNCH(KA, KB)                                                                            \
  if (ka == KA && kb == KB) {                                                                         \
    if (da == kF32 && db == kF32) return launch_cfg<MODE, kF32, KA, kF32, KB>(a, st);                 \
    if (da == kBF16 && db == kBF16) return launch_cfg<MODE, kBF16, KA, kBF16, KB>(a, st);             \
    if (da == kF32 && db == kBF16) return launch_cfg<MODE, kF32, KA, kBF16, KB>(a, st);               \
    if (da == kBF16 && db == kF32) return launch_cfg<MODE, kBF16, KA, kF32, KB>(a, st);               \
  }
  FMM_LAUNCH(true, false)
  FMM_LAUNCH(true, true)
  FMM_LAUNCH(false, false)
#undef FMM_LAUNCH
  return cudaErrorNotSupported;
}

}  // namespace gemm
}  // namespace fmm
