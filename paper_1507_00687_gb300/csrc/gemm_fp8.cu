// Leaf products in E4M3 with power-of-two scales per 128-block along K (the
// leaf format FMM_LEAF_E4M3B128):
//   M_r[i, j] = sum over k blocks kb of 2^(sa[i, kb] + sb[kb, j]) (S8 T8)_kb[i, j]
// with S8, T8 the E4M3 operands the combination pass wrote.  A block's
// scales differ per row and column, so each 128-wide K block is one pipeline
// stage multiplied into its own TMEM block accumulator; the epilogue warps
// fold it into FP32 running sums (running = fma(block, 2^sa 2^sb, running),
// blocks in order) and store the finished tile of M_r for the output pass.
//
//   warps 0-15 epilogue: warps w, w + 4, w + 8, w + 12 share TMEM lanes
//              32 (w mod 4) .. + 31 (one tile row per thread) and take 32
//              columns each
//   warp 16    lane 0: TMEM allocator and tcgen05.mma issuer (kind::f8f6f4,
//              four K = 32 steps per block)
//   warp 17    lane 0: TMA issuer: per stage the A and B tiles (128 x 128
//              bytes, K-major, 128-byte swizzle) and the block's 128 column
//              factors 2^sb (one bulk copy)
//
// One CTA per SM, persistent over (leaf, tile) units.  A stage is released
// when both the MMAs that read its tiles and the epilogue warps that read
// its column factors are done.  Every wait is bounded; on expiry the kernel
// sets the timeout bit of the status word, stops, waits for its own copies
// and MMAs, frees its TMEM and returns.
#include <algorithm>
#include <cstring>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/fmm.h"
#include "device.cuh"
#include "gemm_common.cuh"
#include "kernels.h"

namespace fmm {
namespace fp8 {

using gemm::mbar_arrive_expect_tx;
using gemm::tma_load_2d;

constexpr int BM = 128, BN = 256, BK = 128;  // BK in bytes = elements
constexpr int kEpiWarps = 16, kMmaWarp = 16, kTmaWarp = 17, kThreads = 18 * 32;
constexpr int kEpiCols = BN / (kEpiWarps / 4);  // tile columns per epilogue thread
constexpr int kTile = BM * BK;                 // A tile
constexpr int kTileB = BN * BK;                // B tile (two 128-row boxes)
constexpr int kScaleBytes = BN * 4;
constexpr int kStage = kTile + kTileB + kScaleBytes;  // tiles + column factors, 1024-aligned
constexpr int kStages = 4;
constexpr int kTmemCols = 2 * BN;
constexpr int kSmem = kStages * kStage + 256 + 1024;

// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                      uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Instruction descriptor, kind::f8f6f4: fp32 accumulator, A and B E4M3
// (format code 0), both K-major, M x N.
constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__global__ void __launch_bounds__(kThreads, 1) fp8_fmm_kernel(const __grid_constant__ Fp8Args args) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStage);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1 + kEpiWarps * 32);  // the MMA commit and every epilogue thread
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps * 32);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == kMmaWarp) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int64_t ntn = args.tp_b / BN, ntiles = (args.tp_a / BM) * ntn;
  const int64_t total = ntiles * args.num_leaves;
  const int64_t KB = args.kp / BK;

  if (warp == kTmaWarp) {
    if (lane == 0) {
      // ------------------------------------------------------ TMA issuer
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      uint32_t armed = 0, armed_parity = 0;
      for (int64_t u = blockIdx.x; u < total && ok; u += gridDim.x) {
        const int64_t leaf = u / ntiles, tile = u % ntiles, tm = tile / ntn, tn = tile % ntn;
        for (int64_t kb = 0; kb < KB && ok; ++kb) {
          if (!mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, args.timeout_ns)) { ok = false; break; }
          uint8_t* st = smem + stage * kStage;
          mbar_arrive_expect_tx(&full[stage], (uint32_t)(kTile + kTileB + kScaleBytes));
          tma_load_2d(st, &args.map_a, (int32_t)(kb * BK), (int32_t)(leaf * args.tp_a + tm * BM), &full[stage]);
          for (int h = 0; h < BN / 128; ++h)
            tma_load_2d(st + kTile + h * 128 * BK, &args.map_b, (int32_t)(kb * BK),
                        (int32_t)(leaf * args.tp_b + tn * BN + h * 128), &full[stage]);
          bulk_load(st + kTile + kTileB, args.fb + (leaf * KB + kb) * args.tp_b + tn * BN, kScaleBytes, &full[stage]);
          armed |= 1u << stage;
          armed_parity = (armed_parity & ~(1u << stage)) | (phase << stage);
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) *abort_flag = 1;
      for (int s = 0; s < kStages; ++s) {
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
      constexpr uint32_t idesc = idesc_e4m3(BM, BN);
      int stage = 0;
      uint32_t phase = 0, acc_iter = 0;
      bool ok = true;
      const uint32_t sbase = smem_u32(smem);
      for (int64_t u = blockIdx.x; u < total && ok; u += gridDim.x) {
        for (int64_t kb = 0; kb < KB && ok; ++kb) {
          const uint32_t buf = acc_iter & 1u, aph = (acc_iter >> 1) & 1u;
          if (!mbar_wait_bounded(&tempty[buf], aph ^ 1u, abort_flag, args.timeout_ns)) { ok = false; break; }
          if (!mbar_wait_bounded(&full[stage], phase, abort_flag, args.timeout_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = sbase + stage * kStage, b0 = a0 + kTile;
#pragma unroll
          for (int k32 = 0; k32 < BK / 32; ++k32)
            mma_f8(tmem_base + buf * BN, smem_desc_sw128(a0 + k32 * 32), smem_desc_sw128(b0 + k32 * 32), idesc,
                   k32 > 0 ? 1u : 0u);
          mma_commit(&empty[stage]);
          mma_commit(&tfull[buf]);
          ++acc_iter;
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) *abort_flag = 1;
      mma_commit(drain);
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(drain, 0) && globaltimer_ns() - t0 < 1000000000ull) {
      }
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------- epilogue
    const int quarter = warp & 3, group = warp >> 2;
    const int row = quarter * 32 + lane;
    int stage = 0;
    uint32_t phase = 0, acc_iter = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; u < total && ok; u += gridDim.x) {
      const int64_t leaf = u / ntiles, tile = u % ntiles, tm = tile / ntn, tn = tile % ntn;
      const int64_t ml = tm * BM + row;
      float run[kEpiCols];
#pragma unroll
      for (int j = 0; j < kEpiCols; ++j) run[j] = 0.f;
      for (int64_t kb = 0; kb < KB; ++kb) {
        const uint32_t buf = acc_iter & 1u, aph = (acc_iter >> 1) & 1u;
        const float fa = __ldg(args.fa + (leaf * KB + kb) * args.tp_a + ml);
        // warp-uniform outcome: the TMEM loads below are .sync.aligned
        ok = __all_sync(0xffffffffu, mbar_wait_bounded(&tfull[buf], aph, abort_flag, args.timeout_ns));
        if (!ok) break;
        tc_fence_after();
        const float* fb = reinterpret_cast<const float*>(smem + stage * kStage + kTile + kTileB) + group * kEpiCols;
#pragma unroll
        for (int c = 0; c < kEpiCols / 16; ++c) {
          uint32_t r[16];
          tmem_ld_32x32b_x16(tmem_base + ((uint32_t)(quarter * 32) << 16) + buf * BN + group * kEpiCols + c * 16, r);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 f = *reinterpret_cast<const float4*>(fb + c * 16 + 4 * q);
            const int j = c * 16 + 4 * q;
            run[j] = fmaf(__uint_as_float(r[4 * q]), fa * f.x, run[j]);
            run[j + 1] = fmaf(__uint_as_float(r[4 * q + 1]), fa * f.y, run[j + 1]);
            run[j + 2] = fmaf(__uint_as_float(r[4 * q + 2]), fa * f.z, run[j + 2]);
            run[j + 3] = fmaf(__uint_as_float(r[4 * q + 3]), fa * f.w, run[j + 3]);
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[buf]);
        mbar_arrive(&empty[stage]);  // this block's column factors are consumed
        ++acc_iter;
        if (++stage == kStages) { stage = 0; phase ^= 1u; }
      }
      if (!ok) break;
      float* dst = args.mbuf + (leaf * args.tp_a + ml) * args.tp_b + tn * BN + group * kEpiCols;
#pragma unroll
      for (int q = 0; q < kEpiCols / 4; ++q)
        *reinterpret_cast<float4*>(dst + 4 * q) = make_float4(run[4 * q], run[4 * q + 1], run[4 * q + 2], run[4 * q + 3]);
    }
    if (!ok) *abort_flag = 1;
  }

  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(args.status, kStatusTimeout);
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
}

// ---------------------------------------------------------------- block-scaled form
//
// The same products with the scales applied by the tensor core itself
// (tcgen05.mma kind::mxf8f6f4.block_scale, one UE8M0 scale per row of A and
// per column of B for every 32-wide K sub-block): each unit is one chain of
// MMAs into a single TMEM accumulator, with no per-block fold.  A stage
// carries the A and B tiles and the block's scale atoms (512 bytes per 128
// rows, the layout the combination pass writes); the MMA thread copies the
// atoms into TMEM (tcgen05.cp 32x128b.warpx4: 32 lanes x 128 bits, repeated
// in each lane quarter) ahead of the block's four MMAs, which the tensor
// pipe executes in issue order.  TMEM: the 128 x 256 FP32 accumulator in
// columns 0-255 and one scale slot per stage (A: 4 columns, B: 8) from
// column 256.  The accumulator is single-buffered: the sixteen epilogue
// warps copy it into registers (64 columns per thread), release it, and
// store from registers while the next unit's MMAs run.
//
//   warps 0-15 epilogue (as above: lane quarter w mod 4, 64-column group w / 4)
//   warp 16    lane 0: TMEM allocator, scale copies and MMA issuer
//   warp 17    lane 0: TMA issuer (A tile, two B boxes, the two scale atoms)
constexpr int kSfA = 512, kSfB = 1024;  // scale atoms per stage
constexpr int kStageBs = ((kTile + kTileB + kSfA + kSfB) + 1023) / 1024 * 1024;
constexpr int kStagesBs = 4;
constexpr int kSmemBs = kStagesBs * kStageBs + 256 + 1024;
constexpr uint32_t kSfCol0 = 256, kSfSlot = 32;  // TMEM: scale slot s at column 256 + 32 s (A), + 16 (B)

// Shared-memory descriptor of a scale atom for tcgen05.cp: 32 rows of 16
// bytes, no swizzle, 8-row core matrices 128 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_atom(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)(128 >> 4) << 16;           // leading byte offset (one 16-byte column: unused)
  d |= (uint64_t)(128 >> 4) << 32;           // stride byte offset: next 8 rows
  d |= (uint64_t)1 << 46;                    // descriptor version
  return d;                                  // layout type 0: no swizzle
}

__device__ __forceinline__ void tmem_cp_atom(uint32_t taddr, uint64_t sdesc) {
  asm volatile("tcgen05.cp.cta_group::1.32x128b.warpx4 [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
}

__device__ __forceinline__ void mma_mxf8(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        uint32_t sfa_tmem, uint32_t sfb_tmem, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::mxf8f6f4.block_scale.scale_vec::1X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(
          d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(sfa_tmem), "r"(sfb_tmem), "r"(accumulate)
      : "memory");
}

// Instruction descriptor, kind::mxf8f6f4 with block scaling: A and B E4M3
// (format code 0), both K-major, UE8M0 scales, M x N, scale sub-block 0 of
// each TMEM word for A and B (the four sub-blocks of a 128-block share one
// scale); the accumulator is FP32.
constexpr uint32_t idesc_mx_e4m3(int M, int N) {
  return ((uint32_t)(N >> 3) << 17) | (1u << 23) | ((uint32_t)(M >> 4) << 24);
}

__global__ void __launch_bounds__(kThreads, 1) fp8_bs_kernel(const __grid_constant__ Fp8Args args) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStagesBs * kStageBs);
  uint64_t* empty = full + kStagesBs;
  uint64_t* tfull = empty + kStagesBs;
  uint64_t* tempty = tfull + 1;
  uint64_t* drain = tempty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesBs; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, kEpiWarps);
    mbar_init(drain, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == kMmaWarp) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int64_t ntn = args.tp_b / BN, ntiles = (args.tp_a / BM) * ntn;
  const int64_t total = ntiles * args.num_leaves;
  const int64_t KB = args.kp / BK;
  const int64_t ga = args.tp_a / 128, gb = args.tp_b / 128;  // scale atoms per (leaf, kb)
  const uint8_t* sfa = reinterpret_cast<const uint8_t*>(args.fa);
  const uint8_t* sfb = reinterpret_cast<const uint8_t*>(args.fb);

  if (warp == kTmaWarp) {
    if (lane == 0) {
      // ------------------------------------------------------ TMA issuer
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      uint32_t armed = 0, armed_parity = 0;
      for (int64_t u = blockIdx.x; u < total && ok; u += gridDim.x) {
        const int64_t leaf = u / ntiles, tile = u % ntiles, tm = tile / ntn, tn = tile % ntn;
        for (int64_t kb = 0; kb < KB && ok; ++kb) {
          if (!mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, args.timeout_ns)) { ok = false; break; }
          uint8_t* st = smem + stage * kStageBs;
          mbar_arrive_expect_tx(&full[stage], (uint32_t)(kTile + kTileB + kSfA + kSfB));
          tma_load_2d(st, &args.map_a, (int32_t)(kb * BK), (int32_t)(leaf * args.tp_a + tm * BM), &full[stage]);
          for (int h = 0; h < BN / 128; ++h)
            tma_load_2d(st + kTile + h * 128 * BK, &args.map_b, (int32_t)(kb * BK),
                        (int32_t)(leaf * args.tp_b + tn * BN + h * 128), &full[stage]);
          bulk_load(st + kTile + kTileB, sfa + ((leaf * KB + kb) * ga + tm) * kSfA, kSfA, &full[stage]);
          bulk_load(st + kTile + kTileB + kSfA, sfb + ((leaf * KB + kb) * gb + 2 * tn) * kSfA, kSfB, &full[stage]);
          armed |= 1u << stage;
          armed_parity = (armed_parity & ~(1u << stage)) | (phase << stage);
          if (++stage == kStagesBs) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) *abort_flag = 1;
      for (int s = 0; s < kStagesBs; ++s) {
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
      constexpr uint32_t idesc = idesc_mx_e4m3(BM, BN);
      int stage = 0;
      uint32_t phase = 0, acc_iter = 0;
      bool ok = true;
      const uint32_t sbase = smem_u32(smem);
      for (int64_t u = blockIdx.x; u < total && ok; u += gridDim.x) {
        if (!mbar_wait_bounded(tempty, (acc_iter & 1u) ^ 1u, abort_flag, args.timeout_ns)) { ok = false; break; }
        tc_fence_after();
        for (int64_t kb = 0; kb < KB && ok; ++kb) {
          if (!mbar_wait_bounded(&full[stage], phase, abort_flag, args.timeout_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = sbase + stage * kStageBs, b0 = a0 + kTile, s0 = b0 + kTileB;
          const uint32_t ts_a = tmem_base + kSfCol0 + kSfSlot * (uint32_t)stage, ts_b = ts_a + 16;
          tmem_cp_atom(ts_a, smem_desc_atom(s0));
          tmem_cp_atom(ts_b, smem_desc_atom(s0 + kSfA));
          tmem_cp_atom(ts_b + 4, smem_desc_atom(s0 + 2 * kSfA));
#pragma unroll
          for (int k32 = 0; k32 < BK / 32; ++k32)
            mma_mxf8(tmem_base, smem_desc_sw128(a0 + k32 * 32), smem_desc_sw128(b0 + k32 * 32), idesc, ts_a, ts_b,
                     (kb > 0 || k32 > 0) ? 1u : 0u);
          mma_commit(&empty[stage]);
          if (++stage == kStagesBs) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(tfull);
        ++acc_iter;
      }
      if (!ok) *abort_flag = 1;
      mma_commit(drain);
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(drain, 0) && globaltimer_ns() - t0 < 1000000000ull) {
      }
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------- epilogue
    const int quarter = warp & 3, group = warp >> 2;
    const int row = quarter * 32 + lane;
    uint32_t acc_iter = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; u < total && ok; u += gridDim.x) {
      const int64_t leaf = u / ntiles, tile = u % ntiles, tm = tile / ntn, tn = tile % ntn;
      const int64_t ml = tm * BM + row;
      // warp-uniform outcome: the TMEM loads below are .sync.aligned
      ok = __all_sync(0xffffffffu, mbar_wait_bounded(tfull, acc_iter & 1u, abort_flag, args.timeout_ns));
      if (!ok) break;
      tc_fence_after();
      uint32_t r0[32], r1[32];
      const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + group * kEpiCols;
      tmem_ld_32x32b_x32(taddr, r0);
      tmem_ld_32x32b_x32(taddr + 32, r1);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty);  // the accumulator may be overwritten
      ++acc_iter;
      float* dst = args.mbuf + (leaf * args.tp_a + ml) * args.tp_b + tn * BN + group * kEpiCols;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<uint4*>(dst + 4 * q) = make_uint4(r0[4 * q], r0[4 * q + 1], r0[4 * q + 2], r0[4 * q + 3]);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<uint4*>(dst + 32 + 4 * q) =
            make_uint4(r1[4 * q], r1[4 * q + 1], r1[4 * q + 2], r1[4 * q + 3]);
    }
    if (!ok) *abort_flag = 1;
  }

  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(args.status, kStatusTimeout);
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}

}  // namespace fp8

cudaError_t launch_fp8_gemm(const Fp8Args& a, cudaStream_t st) {
  if (a.tp_a % fp8::BM != 0 || a.tp_b % fp8::BN != 0 || a.kp % fp8::BK != 0) return cudaErrorInvalidValue;
  const int64_t units = (a.tp_a / fp8::BM) * (a.tp_b / fp8::BN) * a.num_leaves;
  if (units == 0 || a.kp == 0) return cudaSuccess;
  static bool attr_set[64][2] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  const int bs = a.block_scaled ? 1 : 0;
  if (bs && (a.tp_a % 128 != 0 || a.tp_b % 256 != 0)) return cudaErrorInvalidValue;
  if (!attr_set[dev][bs]) {
    cudaError_t e = bs ? cudaFuncSetAttribute(fp8::fp8_bs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              fp8::kSmemBs)
                       : cudaFuncSetAttribute(fp8::fp8_fmm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              fp8::kSmem);
    if (e != cudaSuccess) return e;
    attr_set[dev][bs] = true;
  }
  const int64_t grid = std::min<int64_t>(units, device_sm_count());
  KernelTimer timer("multiply", st);
  if (bs) fp8::fp8_bs_kernel<<<(unsigned)grid, fp8::kThreads, fp8::kSmemBs, st>>>(a);
  else fp8::fp8_fmm_kernel<<<(unsigned)grid, fp8::kThreads, fp8::kSmem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace fmm
