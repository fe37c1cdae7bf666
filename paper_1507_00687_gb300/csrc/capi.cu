// C ABI (include/fmm.h): argument validation, plan lifetime, and the
// launch sequences of the scaling steps, the forward and the backward
// multiply.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/fmm.h"
#include "device.cuh"
#include "kernels.h"
#include "plan.h"
#include "rules.h"

namespace fmm {

static thread_local std::string t_last_error;

// Record a failed CUDA call's error text for fmm_last_error().
static bool cuda_ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return false;
}

// Device status word: bits kStatusTimeout / kStatusNonfinite, OR-ed by the
// kernels, read and cleared by fmm_sync_status.
__device__ int g_status;

static int* status_ptr() {
  static int* cache[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
    cache[dev] = static_cast<int*>(p);
  }
  return cache[dev];
}

// FMM_TEST_STALL (environment, read once): the multiply kernel's epilogue
// waits on a barrier that nothing arrives at, so its bounded wait runs out
// and the timeout path (status word, clean stop) can be tested.
static int stall_test() {
  static int v = [] {
    const char* s = std::getenv("FMM_TEST_STALL");
    return s && std::atoi(s) != 0 ? 1 : 0;
  }();
  return v;
}

static uint64_t timeout_ns() {
  static uint64_t v = [] {
    const char* s = std::getenv("FMM_WAIT_TIMEOUT_NS");
    uint64_t t = s ? std::strtoull(s, nullptr, 10) : 0;
    return t ? t : (uint64_t)2000000000ull;  // 2 s per wait
  }();
  return v;
}


static bool valid_dtype(int dt) { return dt == FMM_DT_F32 || dt == FMM_DT_BF16 || dt == FMM_DT_F16; }

static cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// Copy the leaf descriptors to the current device on first use, so that
// plan construction and inspection are host-only.
static fmm_status ensure_uploaded(const Plan* cp) {
  static std::mutex mu;
  Plan* p = const_cast<Plan*>(cp);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FMM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (p->dev) return dev == p->device ? FMM_OK : FMM_ERR_CUDA;
  const size_t bytes = p->host.size() * sizeof(LeafDesc);
  LeafDesc* d = nullptr;
  if (cudaMalloc(&d, bytes + p->lists.size() * 4) != cudaSuccess) return FMM_ERR_CUDA;
  if (cudaMemcpy(d, p->host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(reinterpret_cast<char*>(d) + bytes, p->lists.data(), p->lists.size() * 4, cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    cudaFree(d);
    return FMM_ERR_CUDA;
  }
  p->dev = d;
  p->device = dev;
  return FMM_OK;
}

static fmm_status make_plan(const std::vector<CanonRule>& rules, int leaf, Plan** out,
                            const std::vector<int>* node_rule = nullptr, int levels = 0) {
  Plan* p = nullptr;
  fmm_status s = node_rule ? build_tree_plan(rules, levels, *node_rule, leaf, &p) : build_plan(rules, leaf, &p);
  if (s != FMM_OK) return s;
  if (p->max_terms > kMaxTerms) {
    destroy_plan(p);
    return FMM_ERR_UNSUPPORTED;
  }
  *out = p;
  return FMM_OK;
}

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
static int64_t ceil_div(int64_t x, int64_t m) { return (x + m - 1) / m; }

// ---------------------------------------------------------------- tensor maps

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// A 2-D tensor map over a row-major (rows x cols, ld) matrix with a box of
// box_cols x box_rows elements, no swizzle, zero fill outside.
static bool make_map(CUtensorMap* m, const void* ptr, int dt, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                     int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    t_last_error = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * (dt == kF32 ? 4 : 2))};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, dt == kF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    t_last_error = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

// A 2-D tensor map over a row-major 16-bit matrix (rows x cols, ld) with a
// box of box_cols (32 or 64: 64 or 128 bytes) x box_rows, landing in shared
// memory in the 64- or 128-byte-swizzle layout the MMA descriptors read.
static bool make_map_sw(CUtensorMap* m, const void* ptr, bool f16, int64_t rows, int64_t cols, int64_t ld,
                        int box_cols, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    t_last_error = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  box_cols == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    t_last_error = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

// A 2-D tensor map over a row-major fp32 matrix (rows x cols, ld) with
// 32 x 32 boxes in the 128-byte-swizzle layout (bulk tensor stores of the
// multiply epilogue's chunks).
static bool make_map_f32_sw128(CUtensorMap* m, const void* ptr, int64_t rows, int64_t cols, int64_t ld) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    t_last_error = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  const cuuint32_t box[2] = {32u, 32u};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    t_last_error = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

// Rows of X start on 16-byte boundaries (the reductions' vector path).
static int vec_aligned_host(const void* X, int64_t ld, int dt) {
  const int es = dt == FMM_DT_F32 ? 4 : 2;
  return ((uintptr_t)X % 16 == 0) && ((ld * es) % 16 == 0) ? 1 : 0;
}

// ---------------------------------------------------------------- operands

// One operand of a fast product as stored by the caller: a row-major memory
// matrix (rows x cols, ld).  kcontig: the product's k index runs along the
// memory columns (t along rows); else t runs along the columns.  T, Kd: the
// logical extents; pt, pk: the plan's block counts along t and k; re / ce:
// optional exponents scaling memory rows / columns (signs rs, cs).
struct Source {
  const void* ptr;
  int64_t ld;
  int dtype;
  bool kcontig;
  int64_t T, Kd, pt, pk;
  const int* re;
  int rs;
  const int* ce;
  int cs;
};

// Bytes of the prepared copy of a source (fp32 upper bound).
static int64_t prepared_bytes(int64_t T, int64_t Kd, int64_t pt, int64_t pk) {
  return round_up(pt * round_up(ceil_div(T, pt), 128) * pk * round_up(ceil_div(Kd, pk), 64) * 4, 256);
}

// Build the kernel's view of a source: use the caller's matrix when every
// block is already whole tiles, aligned and unscaled; else write the
// blocked, padded (and scaled) copy into *ws and use that.
static fmm_status prepare(const Source& s, int blk_t_shift, int blk_k_shift, char** ws, char* ws_end, TileOperand* op,
                          CUtensorMap* map, cudaStream_t st) {
  const int64_t bt = ceil_div(s.T, s.pt), bk = ceil_div(s.Kd, s.pk);
  const int64_t btp = round_up(bt, 128), bkp = round_up(bk, 64);
  const int es = s.dtype == kF32 ? 4 : 2;
  const bool direct = !s.re && !s.ce && s.dtype != kF16 && (uintptr_t)s.ptr % 16 == 0 && (s.ld * es) % 16 == 0 &&
                      bt == btp && bk == bkp && bt * s.pt == s.T && bk * s.pk == s.Kd;
  op->kcontig = s.kcontig ? 1 : 0;
  op->bt = btp;
  op->bk = bkp;
  op->blk_t_shift = blk_t_shift;
  op->blk_k_shift = blk_k_shift;
  if (direct) {
    op->ptr = s.ptr;
    op->ld = s.ld;
    op->dtype = s.dtype;
  } else {
    const int odt = s.dtype == kBF16 ? kBF16 : kF32;
    const int oes = odt == kF32 ? 4 : 2;
    // memory rows follow t (kcontig) or k; columns the other index
    const int64_t rblk = s.kcontig ? bt : bk, rpad = s.kcontig ? btp : bkp;
    const int64_t cblk = s.kcontig ? bk : bt, cpad = s.kcontig ? bkp : btp;
    const int64_t R = s.kcontig ? s.T : s.Kd, Cc = s.kcontig ? s.Kd : s.T;
    const int64_t Rp = (s.kcontig ? s.pt : s.pk) * rpad, Cp = (s.kcontig ? s.pk : s.pt) * cpad;
    const int64_t bytes = round_up(Rp * Cp * oes, 256);
    if (*ws + bytes > ws_end) return FMM_ERR_WORKSPACE;
    if (!cuda_ok(launch_prepare(s.ptr, s.dtype, R, Cc, s.ld, rblk, rpad, cblk, cpad, s.re, s.rs, s.ce, s.cs, *ws, Rp,
                                Cp, Cp, st),
                 "operand preparation"))
      return FMM_ERR_CUDA;
    op->ptr = *ws;
    op->ld = Cp;
    op->dtype = odt;
    *ws += bytes;
  }
  // memory rows x cols of the prepared operand
  const int64_t rows = s.kcontig ? s.pt * btp : s.pk * bkp, cols = s.kcontig ? s.pk * bkp : s.pt * btp;
  if (!make_map(map, op->ptr, op->dtype, rows, cols, op->ld, s.kcontig ? 64 : 128, s.kcontig ? 128 : 64))
    return FMM_ERR_CUDA;
  return FMM_OK;
}

// ---------------------------------------------------------------- pass schedule

// Tile width along N of the pass-schedule multiply for a leaf block of bt_b
// columns: 256 (fewer operand bytes per flop) unless the block is narrower.
// FMM_TILE_N=128 or 256 overrides it (tuning).
static int pass_tile_n(int64_t bt_b) {
  static int forced = [] {
    const char* s = std::getenv("FMM_TILE_N");
    const int v = s ? std::atoi(s) : 0;
    return (v == 128 || v == 256) ? v : 0;
  }();
  if (forced) return forced;
  return bt_b >= 256 ? 256 : 128;
}

// Bytes of one side's combined operands: planes x R leaf blocks of
// round_up(bt, tile) x round_up(bk, 64) 16-bit elements.
static int64_t combined_bytes(int64_t T, int64_t Kd, int64_t pt, int64_t pk, int64_t leaves, int planes,
                              int64_t tile) {
  return round_up(planes * leaves * round_up(ceil_div(T, pt), tile) * round_up(ceil_div(Kd, pk), 64) * 2, 256);
}

// Bytes of the stored leaf products (fp32, R padded leaf blocks).
static int64_t products_bytes(int64_t Tx, int64_t Ty, int64_t ptx, int64_t pty, int64_t leaves, int64_t tile_n) {
  return round_up(leaves * round_up(ceil_div(Tx, ptx), 256) * round_up(ceil_div(Ty, pty), tile_n) * 4, 256);
}

// Leaf products on CTA pairs (256 x 256 tiles shared by two SMs) for the
// pass schedule's 16-bit leaves when the leaf blocks are at least 256 x 256;
// FMM_TILE_PAIRS=0 in the environment (read once) keeps the one-CTA kernel.
// The streamed combination pass (bulk tensor copies through a ring of
// stages) for FP32 sources of at most 2 x 2 blocks; FMM_COMBINE_STREAM=0 in
// the environment (read once) keeps the unrolled one.
static bool combine_stream_enabled() {
  static bool on = [] {
    const char* s = std::getenv("FMM_COMBINE_STREAM");
    return !(s && std::atoi(s) == 0);
  }();
  return on;
}

// Output pass of a first half overlapped with the second half's multiply
// (CTA-pair products of at least two tile rows); FMM_OVERLAP=0 in the
// environment (read once) keeps one multiply launch and one output pass.
// Measured at 8192^3 Winograd bf16 with the bulk-store epilogue: calls run
// back to back (the precision sweep) 959 vs 925 TFLOP/s, 886 vs 827 at
// 8192 x 16384 x 4096; single calls timed apart, equal within 1%.
static bool overlap_enabled() {
  static bool on = [] {
    const char* s = std::getenv("FMM_OVERLAP");
    return !(s && std::atoi(s) == 0);
  }();
  return on;
}

// A non-blocking stream per device for work that overlaps the caller's
// stream, with the fork and join events (created on first use; the mutex
// keeps each fork / join sequence of one call together).
struct SideStream {
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  std::mutex mu;
};

static SideStream* side_stream() {
  static SideStream side[64];
  static std::mutex init_mu;
  int dev = 0;
  if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice") || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(init_mu);
  SideStream& s = side[dev];
  if (!s.stream) {
    if (!cuda_ok(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking), "side stream") ||
        !cuda_ok(cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming), "side-stream event") ||
        !cuda_ok(cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming), "side-stream event"))
      return nullptr;
  }
  return &s;
}

// The CTA-pair multiply writes stored products with bulk tensor stores
// from shared memory (whole 128-byte rows); FMM_TMA_STORE=0 in the
// environment (read once) keeps per-thread stores.
static bool tma_store_enabled() {
  static bool on = [] {
    const char* s = std::getenv("FMM_TMA_STORE");
    return !(s && std::atoi(s) == 0);
  }();
  return on;
}

static bool pair_tiles_enabled() {
  static bool on = [] {
    const char* s = std::getenv("FMM_TILE_PAIRS");
    return !(s && std::atoi(s) == 0);
  }();
  return on;
}

// Workspace of the pass schedule for the product X (T_x x Kd) Y (Kd x T_y)
// (upper bound over the tile width; with room for stored leaf products
// when the plan has more than one leaf).
static int64_t pass_bytes(const Plan* p, int64_t Tx, int64_t Kd, int64_t Ty, int64_t ptx, int64_t pk,
                          int64_t pty) {
  if (p->leaf_format == FMM_LEAF_E4M3B128) {
    // bytes of S_r and T_r, their per-block factors, the stored products
    const int64_t R = p->leaves;
    const int64_t ta = round_up(ceil_div(Tx, ptx), 128), tb = round_up(ceil_div(Ty, pty), 256);
    const int64_t kp = round_up(ceil_div(Kd, pk), 128);
    return round_up(R * ta * kp, 256) + round_up(R * (kp / 128) * ta * 4, 256) + round_up(R * tb * kp, 256) +
           round_up(R * (kp / 128) * tb * 4, 256) + round_up(R * ta * tb * 4, 256);
  }
  const int planes = p->leaf_format == FMM_LEAF_BF16X3 ? 2 : 1;
  int64_t between = 0;
  if (p->between && p->levels >= 2) {
    const int64_t k1 = ceil_div(Kd, pk) * (pk / p->rules[0].k0);
    between = 3 * round_up(p->rules[0].r * k1 * 4, 256);
  }
  // A blocks padded to 256 rows when the CTA-pair kernel takes the product
  const int64_t ta = pair_tiles_enabled() && ceil_div(Tx, ptx) >= 256 ? 256 : 128;
  return combined_bytes(Tx, Kd, ptx, pk, p->leaves, planes, ta) +
         combined_bytes(Ty, Kd, pty, pk, p->leaves, planes, 256) +
         (p->leaves > 1 ? products_bytes(Tx, Ty, ptx, pty, p->leaves, 256) : 0) + between;
}

// Geometry of the pass schedule for one product: leaf block extents, their
// padded extents in the combined operands (t: 128 for A, bn for B; k: 64)
// and the workspace bytes of the combined A, B and the stored products.
struct PassGeom {
  int planes, bn;
  bool pair;  // the CTA-pair multiply kernel (256 x 256 tiles)
  int64_t R, bt_a, bt_b, bk, tp_a, tp_b, kp, bytes_a, bytes_b, bytes_m;
};

static PassGeom pass_geom(const Plan* p, const Source& x, const Source& y, int bn, bool force_pair = false) {
  PassGeom g;
  g.planes = p->leaf_format == FMM_LEAF_BF16X3 ? 2 : 1;
  g.R = p->leaves;
  g.bt_a = ceil_div(x.T, x.pt);
  g.bt_b = ceil_div(y.T, y.pt);
  g.bk = ceil_div(x.Kd, x.pk);
  g.bn = bn > 0 ? bn : pass_tile_n(g.bt_b);
  g.pair = bn <= 0 && g.bn == 256 && g.bt_a >= 256 && p->leaf_format != FMM_LEAF_E4M3B128 && pair_tiles_enabled();
  if (force_pair) {  // batches on CTA pairs: 256 x 256 tiles whatever the block size
    g.bn = 256;
    g.pair = true;
  }
  g.tp_a = round_up(g.bt_a, g.pair ? 256 : 128);
  g.tp_b = round_up(g.bt_b, g.bn);
  g.kp = round_up(g.bk, 64);
  g.bytes_a = round_up(g.planes * g.R * g.tp_a * g.kp * 2, 256);
  g.bytes_b = round_up(g.planes * g.R * g.tp_b * g.kp * 2, 256);
  g.bytes_m = round_up(g.R * g.tp_a * g.tp_b * 4, 256);
  return g;
}

// Combination-pass arguments for one side (0: A terms from x, 1: B terms
// from y); the source's memory rows follow t (k-contiguous) or k.
static CombineArgs combine_args(const Plan* p, const PassGeom& g, const Source& s, int side, const LeafDesc* leaves,
                                char* out) {
  const int64_t bt = side == 0 ? g.bt_a : g.bt_b, tp = side == 0 ? g.tp_a : g.tp_b;
  CombineArgs ca;
  std::memset(&ca, 0, sizeof(ca));
  ca.src = s.ptr;
  ca.ld = s.ld;
  ca.dtype = s.dtype;
  ca.rows = s.kcontig ? s.T : s.Kd;
  ca.cols = s.kcontig ? s.Kd : s.T;
  ca.b_rows = s.kcontig ? bt : g.bk;
  ca.b_cols = s.kcontig ? g.bk : bt;
  ca.n_rb = s.kcontig ? s.pt : s.pk;
  ca.n_cb = s.kcontig ? s.pk : s.pt;
  ca.p_rows = s.kcontig ? tp : g.kp;
  ca.p_cols = s.kcontig ? g.kp : tp;
  ca.t_rows = s.kcontig ? 1 : 0;
  ca.re = s.re;
  ca.rs = s.rs;
  ca.ce = s.ce;
  ca.cs = s.cs;
  ca.leaves = leaves;
  ca.num_leaves = g.R;
  ca.side = side;
  const int32_t* lists = reinterpret_cast<const int32_t*>(leaves + g.R);
  ca.t_start = lists + p->list_off[side];
  ca.t_blk = ca.t_start + g.R + 1;
  ca.t_coef = reinterpret_cast<const float*>(ca.t_blk + p->list_nnz[side]);
  ca.t_nnz = p->list_nnz[side];
  ca.blk_t_shift = side == 0 ? 16 : 0;
  ca.blk_k_shift = side == 0 ? 0 : 16;
  ca.out = out;
  ca.fmt = p->leaf_format;
  ca.bk = g.bk;
  return ca;
}

// Multiply-kernel arguments (tensor maps over the combined operands wa, wb).
static bool direct_args(const Plan* p, const PassGeom& g, const Source& x, const Source& y, const EpilogueArgs& c,
                        const LeafDesc* leaves, char* wa, char* wb, float* mbuf, int* status, DirectArgs* d) {
  std::memset(d, 0, sizeof(*d));
  const bool f16 = p->leaf_format == FMM_LEAF_F16;
  // K-major planes: rows (plane, leaf, t), k contiguous, box BK k x tile t;
  // MN-major planes: rows (plane, leaf, k), t contiguous, box 64 t x BK k.
  const int bk_step = direct_gemm_bk(p->leaf_format);
  auto map = [&](CUtensorMap* m, const Source& s, char* buf, int64_t tp, int tile) {
    return s.kcontig ? make_map_sw(m, buf, f16, g.planes * g.R * tp, g.kp, g.kp, bk_step, tile)
                     : make_map_sw(m, buf, f16, g.planes * g.R * g.kp, tp, tp, 64, bk_step);
  };
  // K-major B boxes: the tile's width, or half of it per CTA of a pair
  if (!map(&d->map_a, x, wa, g.tp_a, 128) || !map(&d->map_b, y, wb, g.tp_b, g.pair ? 128 : g.bn)) return false;
  d->a_mn = x.kcontig ? 0 : 1;
  d->b_mn = y.kcontig ? 0 : 1;
  d->c = c;
  d->leaves = leaves;
  d->num_leaves = g.R;
  d->tp_a = g.tp_a;
  d->tp_b = g.tp_b;
  d->kp = g.kp;
  d->mbuf = mbuf;
  // CTA pairs store M_r by bulk tensor copies (FMM_TMA_STORE=0: plain stores)
  if (mbuf && g.pair && tma_store_enabled()) {
    if (!make_map_f32_sw128(&d->map_m, mbuf, g.R * g.tp_a, g.tp_b, g.tp_b)) return false;
    d->tma_store = 1;
  }
  d->status = status;
  d->timeout_ns = timeout_ns();
  d->stall_test = stall_test();
  return true;
}

// Output-pass arguments over the stored products mbuf.
static OutArgs out_args(const Plan* p, const PassGeom& g, const EpilogueArgs& c, const LeafDesc* leaves,
                        float* mbuf) {
  OutArgs o;
  std::memset(&o, 0, sizeof(o));
  o.mbuf = mbuf;
  o.tp_a = g.tp_a;
  o.tp_b = g.tp_b;
  o.c = c;
  o.leaves = leaves;
  o.num_leaves = g.R;
  o.c_blocks = p->pm * p->pn;
  o.pn = p->pn;
  const int32_t* lists = reinterpret_cast<const int32_t*>(leaves + g.R);
  o.c_start = lists + p->list_off[2];
  o.c_blk = o.c_start + g.R + 1;
  o.c_coef = reinterpret_cast<const float*>(o.c_blk + p->list_nnz[2]);
  o.c_nnz = p->list_nnz[2];
  if (p->gather_off >= 0) {
    o.g_start = lists + p->gather_off;
    o.g_leaf = o.g_start + o.c_blocks + 1;
    o.g_coef = reinterpret_cast<const float*>(o.g_leaf + p->list_nnz[2]);
  }
  return o;
}

// The pass schedule: the combination pass writes S_r (from x) and T_r (from
// y) for every leaf into the workspace; the multiply kernel then streams
// them and either adds W-weighted products into C in its epilogue or stores
// them for the output pass.  FMM_ERR_WORKSPACE when the workspace is too
// small.
// A 2-D byte tensor map (rows x cols, ld), 128 x 128 boxes, 128-byte swizzle.
static bool make_map_u8(CUtensorMap* m, const void* ptr, int64_t rows, int64_t cols, int64_t ld) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    t_last_error = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld};
  const cuuint32_t box[2] = {128u, 128u};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    t_last_error = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

// E4M3 leaf products with the tensor core's block scaling (UE8M0 scale
// atoms); FMM_FP8_FOLD=1 in the environment (read once) keeps the kernel
// that folds each 128-wide K block's product into FP32 sums itself.
static bool fp8_block_scaled() {
  static bool on = [] {
    const char* s = std::getenv("FMM_FP8_FOLD");
    return !(s && std::atoi(s) != 0);
  }();
  return on;
}

// The pass schedule with E4M3 leaves: the E4M3 combination pass writes
// S_r, T_r (K-major bytes) and their per-128-block scales; the FP8
// multiply kernel stores M_r; the output pass forms C.
static fmm_status run_pass_fp8(const Plan* p, const Source& x, const Source& y, const EpilogueArgs& c,
                               const LeafDesc* leaves, int* status, void* ws, size_t ws_bytes, cudaStream_t st) {
  PassGeom g = pass_geom(p, x, y, 128);
  g.planes = 1;
  g.tp_a = round_up(g.bt_a, 128);
  g.tp_b = round_up(g.bt_b, 256);  // the E4M3 multiply kernel's 256-wide tiles
  g.kp = round_up(g.bk, 128);
  const int64_t R = g.R, KB = g.kp / 128;
  const int64_t ba = round_up(R * g.tp_a * g.kp, 256), fa = round_up(R * KB * g.tp_a * 4, 256);
  const int64_t bb = round_up(R * g.tp_b * g.kp, 256), fbb = round_up(R * KB * g.tp_b * 4, 256);
  const int64_t bm = round_up(R * g.tp_a * g.tp_b * 4, 256);
  if (!ws || (uintptr_t)ws % 256 != 0 || (int64_t)ws_bytes < ba + fa + bb + fbb + bm) return FMM_ERR_WORKSPACE;
  char* w = static_cast<char*>(ws);
  char* wa = w;
  float* sa = reinterpret_cast<float*>(w + ba);
  char* wb = w + ba + fa;
  float* sb = reinterpret_cast<float*>(w + ba + fa + bb);
  float* mbuf = reinterpret_cast<float*>(w + ba + fa + bb + fbb);
  CombineArgs ca = combine_args(p, g, x, 0, leaves, wa), cb = combine_args(p, g, y, 1, leaves, wb);
  // both sides K-major: [leaf][t][k]
  ca.p_rows = g.tp_a;
  ca.p_cols = g.kp;
  const int bs = fp8_block_scaled() ? 1 : 0;
  ca.scale_out = sa;
  ca.sf_atoms = bs;
  cb.p_rows = g.tp_b;
  cb.p_cols = g.kp;
  cb.scale_out = sb;
  cb.sf_atoms = bs;
  if (!cuda_ok(launch_combine_e4m3(cb, st), "E4M3 combination pass (B)") ||
      !cuda_ok(launch_combine_e4m3(ca, st), "E4M3 combination pass (A)"))
    return FMM_ERR_CUDA;
  Fp8Args f;
  std::memset(&f, 0, sizeof(f));
  if (!make_map_u8(&f.map_a, wa, R * g.tp_a, g.kp, g.kp) || !make_map_u8(&f.map_b, wb, R * g.tp_b, g.kp, g.kp))
    return FMM_ERR_CUDA;
  f.fa = sa;
  f.fb = sb;
  f.mbuf = mbuf;
  f.tp_a = g.tp_a;
  f.tp_b = g.tp_b;
  f.kp = g.kp;
  f.num_leaves = R;
  f.status = status;
  f.timeout_ns = timeout_ns();
  f.block_scaled = bs;
  if (!cuda_ok(launch_fp8_gemm(f, st), "E4M3 multiply launch")) return FMM_ERR_CUDA;
  const OutArgs o = out_args(p, g, c, leaves, mbuf);
  const bool gather = p->pm * p->pn > kMaxOutBlocks;
  if (gather && p->gather_off < 0) return FMM_ERR_UNSUPPORTED;
  return cuda_ok(gather ? launch_out_gather(o, st) : launch_out_combine(o, st), "output combination pass")
             ? FMM_OK
             : FMM_ERR_CUDA;
}

static fmm_status run_pass(const Plan* p, const Source& x, const Source& y, const EpilogueArgs& c,
                           const LeafDesc* leaves, int* status, void* ws, size_t ws_bytes, cudaStream_t st,
                           bool between) {
  if (p->leaf_format == FMM_LEAF_E4M3B128) {
    if (between) return FMM_ERR_UNSUPPORTED;
    return run_pass_fp8(p, x, y, c, leaves, status, ws, ws_bytes, st);
  }
  const PassGeom g = pass_geom(p, x, y, 0);
  const int64_t R = g.R;
  if (!ws || (uintptr_t)ws % 256 != 0 || (int64_t)ws_bytes < g.bytes_a + g.bytes_b) return FMM_ERR_WORKSPACE;
  char* wa = static_cast<char*>(ws);
  char* wb = wa + g.bytes_a;
  // Stored leaf products unless the epilogue form is asked for: measured
  // faster at every size (every SM gets (leaf, tile) units; the fused
  // epilogue leaves SMs idle when tiles per leaf are few, and its C
  // read-modify-writes cost more than one more bandwidth pass).
  // Accumulating epilogue (CTA pairs only): every (leaf, tile) unit adds
  // its terms into a zeroed C by atomic FP32 additions, so neither stored
  // products nor the output pass are needed.
  const bool accumulate = p->schedule == FMM_SCHEDULE_PASS_ACCUMULATE && g.pair && g.R > 1;
  const bool want_m = p->schedule != FMM_SCHEDULE_PASS_EPILOGUE && !accumulate;
  // more C blocks than the stored-products pass keeps on chip: the output
  // pass gathers per C block instead
  const bool gather = p->pm * p->pn > kMaxOutBlocks;
  const bool store_m = want_m && g.R > 1 && (!gather || p->gather_off >= 0) &&
                       (int64_t)ws_bytes >= g.bytes_a + g.bytes_b + g.bytes_m;
  float* mbuf = store_m ? reinterpret_cast<float*>(wb + g.bytes_b) : nullptr;

  CombineArgs ca = combine_args(p, g, x, 0, leaves, wa), cb = combine_args(p, g, y, 1, leaves, wb);
  if (between) {
    // Scaling between recursive steps: the first level's pairs (S_r, T_r)
    // get inside-scaling exponents d^(r) from their FP32 sums; the
    // combination pass then scales each term element by 2^(+-d).
    const Plan* p1 = p->level1;
    if (ensure_uploaded(p1) != FMM_OK) return FMM_ERR_CUDA;
    const int64_t R1 = p1->leaves;
    const int64_t k1 = g.bk * (p->pk / p1->pk);
    const int64_t dbytes = round_up(R1 * k1 * 4, 256);
    char* wz = wb + g.bytes_b + (store_m ? g.bytes_m : 0);
    if ((int64_t)ws_bytes < (wz - wa) + 3 * dbytes) return FMM_ERR_WORKSPACE;
    int* cexp = reinterpret_cast<int*>(wz);
    int* rexp = reinterpret_cast<int*>(wz + dbytes);
    int* d1 = reinterpret_cast<int*>(wz + 2 * dbytes);
    Source x1 = x, y1 = y;
    x1.pt = p1->pm;
    x1.pk = p1->pk;
    y1.pt = p1->pn;
    y1.pk = p1->pk;
    const PassGeom g1 = pass_geom(p1, x1, y1, 128);
    CombineArgs na = combine_args(p1, g1, x1, 0, p1->dev, nullptr);
    CombineArgs nb = combine_args(p1, g1, y1, 1, p1->dev, nullptr);
    // level-1 blocks as the full plan partitions them (leaf blocks grouped)
    const int64_t bt1a = g.bt_a * (p->pm / p1->pm), bt1b = g.bt_b * (p->pn / p1->pn);
    na.b_rows = x.kcontig ? bt1a : k1;
    na.b_cols = x.kcontig ? k1 : bt1a;
    nb.b_rows = y.kcontig ? bt1b : k1;
    nb.b_cols = y.kcontig ? k1 : bt1b;
    if (!cuda_ok(launch_fill(cexp, 2 * dbytes / 4, kZeroExp, st), "between-steps fill") ||
        !cuda_ok(launch_node_exp(na, cexp, k1, st), "between-steps exponents (A)") ||
        !cuda_ok(launch_node_exp(nb, rexp, k1, st), "between-steps exponents (B)") ||
        !cuda_ok(launch_between_finalize(cexp, rexp, d1, R1 * k1, st), "between-steps exponents"))
      return FMM_ERR_CUDA;
    for (CombineArgs* c2 : {&ca, &cb}) {
      c2->between_d = d1;
      c2->between_k1 = k1;
      c2->leaves_per_node = R / R1;
      c2->kb_inner = p->pk / p1->pk;
    }
    ca.between_sign = +1;
    cb.between_sign = -1;
  }
  // B first: a scaling sequence that ends with a pass over B leaves it in L2
  cudaError_t ce = cudaErrorNotSupported;
  if (combine_stream_enabled() && x.dtype == kF32 && y.dtype == kF32) {
    CUtensorMap mx, my;
    if (make_map(&mx, x.ptr, kF32, ca.rows, ca.cols, x.ld, 256, 8) &&
        make_map(&my, y.ptr, kF32, cb.rows, cb.cols, y.ld, 256, 8))
      ce = launch_combine_pair_stream(cb, my, ca, mx, timeout_ns(), status, st);
  }
  if (ce == cudaErrorNotSupported) ce = launch_combine_pair(cb, ca, st);
  if (!cuda_ok(ce, "combination passes")) return FMM_ERR_CUDA;
  DirectArgs d;
  if (!direct_args(p, g, x, y, c, leaves, wa, wb, mbuf, status, &d)) return FMM_ERR_CUDA;
  if (accumulate) {
    d.accumulate = 1;
    if (!cuda_ok(cudaMemset2DAsync(c.C, (size_t)c.ldc * 4, 0, (size_t)c.N * 4, (size_t)c.M, st), "C zero fill"))
      return FMM_ERR_CUDA;
  }
  // Hiding half of the output pass pays only where the multiply is
  // compute-bound (leaf K of at least 2048), each half still fills the GPU
  // for several waves, and the output pass is light next to the multiply
  // (at most 16 leaves): at n = 4096 (three waves per half), for short leaf
  // K, and for the 49 leaves of two Strassen levels (the linear layer's
  // weight gradient: 177 vs 150 us) the single launch is faster.
  const int64_t ntm = g.tp_a / 256;
  const int64_t half_waves = ntm >= 2 ? (ntm / 2) * (g.tp_b / 256) * g.R / std::max(1, device_sm_count() / 2) : 0;
  if (store_m && g.pair && !gather && ntm >= 2 && p->pm * p->pn <= 16 && g.R <= 16 &&
      half_waves >= 5 && g.kp >= 2048 && overlap_enabled()) {
    // Two launches over the tile-row halves; the output pass of the first
    // half runs on a side stream, beside the second half's multiply (one
    // 256-thread CTA fits on each SM next to a pair CTA), then the second
    // half's output pass; the caller's stream waits for both.
    SideStream* side = side_stream();
    if (!side) return FMM_ERR_CUDA;
    const int64_t h = ntm / 2;
    DirectArgs d1 = d, d2 = d;
    d1.tm_begin = 0;
    d1.tm_count = h;
    d2.tm_begin = h;
    d2.tm_count = ntm - h;
    OutArgs o1 = out_args(p, g, c, leaves, mbuf), o2 = o1;
    o1.r_begin = 0;
    o1.r_end = h * 256;
    o2.r_begin = h * 256;
    std::lock_guard<std::mutex> lock(side->mu);
    if (!cuda_ok(launch_pair_gemm(d1, p->leaf_format, st), "multiply launch (first half)") ||
        !cuda_ok(cudaEventRecord(side->fork, st), "side-stream fork") ||
        !cuda_ok(cudaStreamWaitEvent(side->stream, side->fork, 0), "side-stream fork") ||
        !cuda_ok(launch_out_dense_slim(o1, side->stream), "output combination pass (first half)") ||
        !cuda_ok(cudaEventRecord(side->join, side->stream), "side-stream join") ||
        !cuda_ok(launch_pair_gemm(d2, p->leaf_format, st), "multiply launch (second half)") ||
        !cuda_ok(launch_out_combine(o2, st), "output combination pass (second half)") ||
        !cuda_ok(cudaStreamWaitEvent(st, side->join, 0), "side-stream join"))
      return FMM_ERR_CUDA;
    return FMM_OK;
  }
  if (!cuda_ok(g.pair ? launch_pair_gemm(d, p->leaf_format, st) : launch_direct_gemm(d, p->leaf_format, g.bn, st),
               "multiply launch"))
    return FMM_ERR_CUDA;
  if (!store_m) return FMM_OK;
  const OutArgs o = out_args(p, g, c, leaves, mbuf);
  return cuda_ok(gather ? launch_out_gather(o, st) : launch_out_combine(o, st), "output combination pass")
             ? FMM_OK
             : FMM_ERR_CUDA;
}

// Run the flattened plan p: C (M x N) = X (M x K) Y (K x N) with X, Y given
// as sources (X: t = M, k = K; Y: t = N, k = K).  leaves: a device copy of
// the plan's tables (the LeafDesc array followed by the term lists) to use
// instead of the plan's own upload (NULL: the plan's own, uploaded on first
// use).
static fmm_status run_plan(const Plan* p, const Source& x, const Source& y, float* C, int64_t ldc, int64_t M,
                           int64_t K, int64_t N, const int* eA, const int* eB, void* ws, size_t ws_bytes,
                           cudaStream_t st, const LeafDesc* leaves = nullptr, bool allow_between = true) {
  if (M == 0 || N == 0) return FMM_OK;
  if (K == 0) {
    return cuda_ok(cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)N * 4, (size_t)M, st), "memset")
               ? FMM_OK
               : FMM_ERR_CUDA;
  }
  int* status = status_ptr();
  if (!status) return FMM_ERR_CUDA;
  if (!leaves) {
    if (ensure_uploaded(p) != FMM_OK) return FMM_ERR_CUDA;
    leaves = p->dev;
  }
  EpilogueArgs c;
  c.C = C;
  c.ldc = ldc;
  c.M = M;
  c.N = N;
  c.bm = ceil_div(M, p->pm);
  c.bn = ceil_div(N, p->pn);
  c.eA = eA;
  c.eB = eB;
  c.vec_ok = ((uintptr_t)C % 16 == 0) && (ldc % 4 == 0) && (c.bn % 4 == 0) ? 1 : 0;
  const bool pass = p->schedule == FMM_SCHEDULE_PASS || p->schedule == FMM_SCHEDULE_PASS_EPILOGUE ||
                    p->schedule == FMM_SCHEDULE_PASS_PRODUCTS || p->schedule == FMM_SCHEDULE_PASS_ACCUMULATE ||
                    (p->schedule == FMM_SCHEDULE_AUTO && ws && (uintptr_t)ws % 256 == 0 &&
                     (int64_t)ws_bytes >= pass_bytes(p, M, K, N, p->pm, p->pk, p->pn));
  const bool between = allow_between && p->between && p->levels >= 2 && p->level1;
  const bool needs_pass = between || p->leaf_format == FMM_LEAF_E4M3B128;
  if (needs_pass && !pass) return p->schedule == FMM_SCHEDULE_LOAD_STAGE ? FMM_ERR_UNSUPPORTED : FMM_ERR_WORKSPACE;
  if (pass) return run_pass(p, x, y, c, leaves, status, ws, ws_bytes, st, between);
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  char* w = static_cast<char*>(ws);
  char* w_end = w ? w + ws_bytes : nullptr;
  if (w && (uintptr_t)w % 256 != 0) return FMM_ERR_WORKSPACE;
  fmm_status s = prepare(x, 16, 0, &w, w_end, &g.a, &g.map_a, st);
  if (s != FMM_OK) return s;
  s = prepare(y, 0, 16, &w, w_end, &g.b, &g.map_b, st);
  if (s != FMM_OK) return s;
  g.c = c;
  g.leaves = leaves;
  g.num_leaves = p->leaves;
  g.status = status;
  g.timeout_ns = timeout_ns();
  return cuda_ok(launch_fused_gemm(g, p->leaf_format, st), "fused multiply launch") ? FMM_OK : FMM_ERR_CUDA;
}

// Workspace of fmm_multiply and fmm_multiply_backward (fp32 upper bound):
// the prepared copies of the two operands of the largest of the forward,
// dA and dB products.
static size_t ws_bytes_for(const Plan* p, int64_t M, int64_t K, int64_t N) {
  int64_t fwd = prepared_bytes(M, K, p->pm, p->pk) + prepared_bytes(N, K, p->pn, p->pk);
  int64_t da = prepared_bytes(M, N, p->pm, p->pn) + prepared_bytes(K, N, p->pk, p->pn);
  int64_t db = prepared_bytes(K, M, p->pk, p->pm) + prepared_bytes(N, M, p->pn, p->pm);
  if (p->schedule != FMM_SCHEDULE_LOAD_STAGE) {
    // dA = dC B^T is an <m0, n0, k0> product, dB = A^T dC a <k0, m0, n0> one.
    fwd = std::max(fwd, pass_bytes(p, M, K, N, p->pm, p->pk, p->pn));
    da = std::max(da, pass_bytes(p, M, N, K, p->pm, p->pn, p->pk));
    db = std::max(db, pass_bytes(p, K, M, N, p->pk, p->pm, p->pn));
  }
  return (size_t)std::max(fwd, std::max(da, db));
}

// ---------------------------------------------------------------- no-alloc scratch

// Scratch of fmm_multiply_noalloc: the leaf table, then the prepared operand
// copies.  A file-scope device array, so that callers that may not allocate
// device memory still get a workspace; every device that loads the library
// holds it until exit.  In host code this name is only a stand-in for the
// array; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FMM_NOALLOC_SCRATCH_BYTES];

// The plan's tables reach the scratch inside kernel parameters, up to
// kTableChunkWords 32-bit words per launch: a launch copies its arguments
// when it is issued, so the host never waits for a copy out of its own
// (pageable) memory and no staging buffer is needed.
constexpr int kTableChunkWords = 8000;  // 32000 bytes, under the 32764-byte parameter limit
struct TableChunk {
  uint32_t w[kTableChunkWords];
};

__global__ void __launch_bounds__(256) table_chunk_kernel(const __grid_constant__ TableChunk c, uint32_t* dst,
                                                          int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = c.w[i];
}

// Copy `words` 32-bit words from host memory to dst (device) on st, one
// launch per kTableChunkWords words.
static bool upload_words(uint32_t* dst, const void* src, size_t words, cudaStream_t st) {
  static TableChunk chunk;  // staging for the launch arguments (copied by each launch)
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  const char* s = static_cast<const char*>(src);
  for (size_t off = 0; off < words; off += kTableChunkWords) {
    const int n = (int)std::min<size_t>(kTableChunkWords, words - off);
    std::memcpy(chunk.w, s + off * 4, (size_t)n * 4);
    table_chunk_kernel<<<(n + 255) / 256, 256, 0, st>>>(chunk, dst + off, n);
    if (!cuda_ok(cudaGetLastError(), "table copy into the no-alloc scratch")) return false;
  }
  return true;
}

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the first fmm_multiply_noalloc call there).
static char* noalloc_scratch() {
  static char* cache[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice") || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev]) {
    void* ptr = nullptr;
    if (!cuda_ok(cudaGetSymbolAddress(&ptr, g_noalloc_scratch), "cudaGetSymbolAddress(no-alloc scratch)"))
      return nullptr;
    cache[dev] = static_cast<char*>(ptr);
  }
  return cache[dev];
}

// ---------------------------------------------------------------- batches

constexpr int kBatchTileN = 128;

// Steps a batch supports (Alg. 3 from no scaling).
static int batch_steps(const char* steps) {
  if (!steps || !*steps) return 0;
  if (!std::strcmp(steps, "O")) return 1;
  if (!std::strcmp(steps, "I")) return 2;
  if (!std::strcmp(steps, "OI")) return 3;
  return -1;
}

// Where each part of a batch lives in the workspace, computed identically
// by fmm_batch_workspace_size and fmm_batch_create.
struct BatchLayout {
  size_t off_red[4], off_red_start[4];
  size_t off_comb, off_comb_start, off_copy_start, off_direct, off_unit_start, off_out, off_out_start;
  size_t off_exp;                  // eA (sum M) | d (sum K) | eB (sum N), int32
  int64_t sum_m, sum_k, sum_n;
  std::vector<size_t> off_a, off_b, off_m;  // per problem, combined A / B and stored products
  std::vector<PassGeom> geom;
  size_t total;
};

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static Source batch_source_a(const fmm_problem& q, const Plan* p, int dt, const int* eA, const int* d) {
  return Source{q.A, q.lda, dt, true, q.M, q.K, p->pm, p->pk, eA, -1, d, +1};
}
static Source batch_source_b(const fmm_problem& q, const Plan* p, int dt, const int* d, const int* eB) {
  return Source{q.B, q.ldb, dt, false, q.N, q.K, p->pn, p->pk, d, -1, eB, -1};
}

// A batch entry whose plan is the classical product (one leaf, one term per
// side) with bf16 inputs and bf16 leaves: the multiply reads the caller's A
// and B through tensor maps, with no scaling reductions and no conversion
// pass.  Power-of-two diagonal scaling cancels exactly for it: the inside
// factor 2^d_k cancels between A'_ik and B'_kj, and the outside factor
// 2^-(eA_i + eB_j) is common to every product of C_ij, so the rounded sums
// scaled and unscaled differ by that exact power of two and the unscaled C
// is the scaled path's bit for bit whenever no scaled operand or partial
// sum leaves the normal range.  bf16 has the exponent range of FP32, so
// that holds but at the extremes; fp16 (normal range down to 2^-14 only)
// loses or gains bits when small entries are shifted, so fp16 entries keep
// the scaled path.
static bool batch_direct(const fmm_problem& q, const Plan* p, int dt) {
  const bool same = dt == FMM_DT_BF16 && p->leaf_format == FMM_LEAF_BF16;
  return pair_tiles_enabled() && p->leaves == 1 && p->pm == 1 && p->pk == 1 && p->pn == 1 && same &&
         (uintptr_t)q.A % 16 == 0 && (uintptr_t)q.B % 16 == 0 && (q.lda * 2) % 16 == 0 && (q.ldb * 2) % 16 == 0;
}

static fmm_status batch_layout(const fmm_problem* probs, int count, int dt, BatchLayout* L) {
  size_t at = 0;
  const size_t cnt = (size_t)count;
  for (int k = 0; k < 4; ++k) {
    L->off_red[k] = at;
    at = align_up(at + cnt * sizeof(ReduceArgs), 256);
    L->off_red_start[k] = at;
    at = align_up(at + (cnt + 1) * 8, 256);
  }
  L->off_comb = at;
  at = align_up(at + 2 * cnt * sizeof(CombineArgs), 256);
  L->off_comb_start = at;
  at = align_up(at + (2 * cnt + 1) * 8, 256);
  L->off_copy_start = at;
  at = align_up(at + (2 * cnt + 1) * 8, 256);
  L->off_direct = at;
  at = align_up(at + cnt * sizeof(DirectArgs), 256);
  L->off_unit_start = at;
  at = align_up(at + (cnt + 1) * 8, 256);
  L->off_out = at;
  at = align_up(at + cnt * sizeof(OutArgs), 256);
  L->off_out_start = at;
  at = align_up(at + (cnt + 1) * 8, 256);
  L->sum_m = L->sum_k = L->sum_n = 0;
  for (int i = 0; i < count; ++i) {
    L->sum_m += probs[i].M;
    L->sum_k += probs[i].K;
    L->sum_n += probs[i].N;
  }
  L->off_exp = at;
  at = align_up(at + (size_t)(L->sum_m + L->sum_k + L->sum_n) * 4, 256);
  L->off_a.resize(cnt);
  L->off_b.resize(cnt);
  L->off_m.resize(cnt);
  L->geom.resize(cnt);
  for (int i = 0; i < count; ++i) {
    const Plan* p = reinterpret_cast<const Plan*>(probs[i].plan);
    const Source x = batch_source_a(probs[i], p, dt, nullptr, nullptr);
    const Source y = batch_source_b(probs[i], p, dt, nullptr, nullptr);
    const bool pairs = pair_tiles_enabled();
    PassGeom g = pass_geom(p, x, y, kBatchTileN, pairs);
    if (pairs && batch_direct(probs[i], p, dt)) g.bytes_a = g.bytes_b = g.bytes_m = 0;
    L->geom[(size_t)i] = g;
    L->off_a[(size_t)i] = at;
    at += (size_t)g.bytes_a;
    L->off_b[(size_t)i] = at;
    at += (size_t)g.bytes_b;
    L->off_m[(size_t)i] = at;
    at += (size_t)g.bytes_m;
  }
  L->total = at;
  return FMM_OK;
}

static fmm_status batch_check(const fmm_problem* probs, int count, int dt, const char* steps) {
  if (!probs || count <= 0 || count > 30000 || !valid_dtype(dt) || batch_steps(steps) < 0) return FMM_ERR_ARG;
  int fmt = -1;
  for (int i = 0; i < count; ++i) {
    const fmm_problem& q = probs[i];
    const Plan* p = reinterpret_cast<const Plan*>(q.plan);
    if (!p || !q.A || !q.B || !q.C) return FMM_ERR_ARG;
    if (q.M <= 0 || q.K <= 0 || q.N <= 0 || q.lda < q.K || q.ldb < q.N || q.ldc < q.N) return FMM_ERR_SHAPE;
    if (fmt >= 0 && p->leaf_format != fmt) return FMM_ERR_ARG;
    fmt = p->leaf_format;
    if (dt == FMM_DT_F16 && fmt == FMM_LEAF_BF16X3) return FMM_ERR_DTYPE;
    if ((p->between && p->levels >= 2) || p->leaf_format == FMM_LEAF_E4M3B128) return FMM_ERR_UNSUPPORTED;
    if (p->pm * p->pn > kMaxOutBlocks || p->pm * p->pk > 64 || p->pk * p->pn > 64) return FMM_ERR_UNSUPPORTED;
    if (ceil_div(q.M, p->pm) >= (1ll << 30) || ceil_div(q.N, p->pn) >= (1ll << 30) ||
        ceil_div(q.K, p->pk) >= (1ll << 30))
      return FMM_ERR_SHAPE;
  }
  return FMM_OK;
}

struct Batch {
  int count = 0, dt = 0, fmt = 0, steps = 0;
  char* ws = nullptr;
  int* status = nullptr;
  BatchLayout L;
  int64_t red_total[4] = {0, 0, 0, 0};
  int64_t comb_total = 0, copy_total = 0, unit_total = 0, out_total = 0;
  int comb_count = 0, copy_count = 0;  // staged entries first in the table, then plain conversions
  int out_count = 0;
  int comb_tr = 32, out_tr = 32;
  size_t comb_smem = 0, out_smem = 0;
  DirectArgs layout;  // status, wait limit, operand layouts
  bool pairs = false;   // the multiply runs on CTA pairs (256 x 256 tiles)
  bool any_scaled = true;  // some entry's scaling reductions run
};

static fmm_status batch_build(Batch* b, const fmm_problem* probs) {
  const int count = b->count, dt = b->dt;
  BatchLayout& L = b->L;
  char* ws = b->ws;
  int* eA_all = reinterpret_cast<int*>(ws + L.off_exp);
  int* d_all = eA_all + L.sum_m;
  int* eB_all = d_all + L.sum_k;
  const bool o_step = b->steps & 1, i_step = b->steps & 2;
  std::vector<ReduceArgs> red[4];
  std::vector<int64_t> red_start[4];
  for (int k = 0; k < 4; ++k) {
    red[k].resize((size_t)count);
    red_start[k].assign((size_t)count + 1, 0);
  }
  std::vector<CombineArgs> comb(2 * (size_t)count);
  std::vector<CombineArgs> staged, plain;  // the table is staged entries, then plain conversions
  std::vector<int64_t> comb_start(1, 0), copy_start(1, 0);
  std::vector<DirectArgs> dir((size_t)count);
  std::vector<int64_t> unit_start((size_t)count + 1, 0);
  std::vector<OutArgs> out;
  std::vector<int64_t> out_start(1, 0);
  std::vector<int64_t> unit_cost((size_t)count), units((size_t)count);
  b->pairs = pair_tiles_enabled();
  const int64_t tm_rows = b->pairs ? 256 : 128, tn_cols = b->pairs ? 256 : kBatchTileN;
  const int64_t workers = b->pairs ? device_sm_count() / 2 : device_sm_count();
  int64_t max_nb = 1, max_cb = 1, tiles_all = 0;
  for (int i = 0; i < count; ++i) {
    const Plan* p = reinterpret_cast<const Plan*>(probs[i].plan);
    if (p->leaves > 1) max_nb = std::max(max_nb, std::max(p->pm * p->pk, p->pk * p->pn));
    max_cb = std::max(max_cb, p->pm * p->pn);
    const PassGeom& g = L.geom[(size_t)i];
    tiles_all += (g.tp_a / tm_rows) * (g.tp_b / tn_cols);
  }
  // Output combination in the multiply epilogue (each tile of each product
  // a unit covering all its leaves) when the batch has tiles enough to
  // occupy the GPU; else stored leaf products for the many-leaf plans.
  const bool fused = tiles_all >= 2 * workers;
  b->any_scaled = false;
  b->comb_tr = combine_batched_rows(max_nb);
  b->out_tr = out_batched_rows(max_cb);
  int64_t om = 0, ok_ = 0, on = 0;
  for (int i = 0; i < count; ++i) {
    const fmm_problem& q = probs[i];
    const Plan* p = reinterpret_cast<const Plan*>(q.plan);
    if (ensure_uploaded(p) != FMM_OK) return FMM_ERR_CUDA;
    const LeafDesc* leaves = p->dev;
    int* eA = eA_all + om;
    int* d = d_all + ok_;
    int* eB = eB_all + on;
    om += q.M;
    ok_ += q.K;
    on += q.N;
    const size_t u = (size_t)i;
    const bool direct = b->pairs && batch_direct(q, p, dt);
    b->any_scaled = b->any_scaled || !direct;
    // scaling reductions: rows(A) -> eA, columns(A) -> d, columns(B) -> eB, rows(B) -> d
    const int vec_a = vec_aligned_host(q.A, q.lda, dt), vec_b = vec_aligned_host(q.B, q.ldb, dt);
    red[0][u] = ReduceArgs{q.A, q.M, q.K, q.lda, nullptr, +1, eA, vec_a, 0, 0};
    red[1][u] = ReduceArgs{q.A, q.M, q.K, q.lda, o_step ? eA : nullptr, -1, d, vec_a, kBatchColRows,
                           ceil_div(q.K, kBatchColSpan)};
    red[2][u] = ReduceArgs{q.B, q.K, q.N, q.ldb, nullptr, -1, eB, vec_b, kBatchColRows, ceil_div(q.N, kBatchColSpan)};
    red[3][u] = ReduceArgs{q.B, q.K, q.N, q.ldb, o_step ? eB : nullptr, -1, d, vec_b, 0, 0};
    // direct entries take no part in the reductions (empty ranges)
    red_start[0][u + 1] = red_start[0][u] + (direct ? 0 : q.M);
    red_start[1][u + 1] = red_start[1][u] + (direct ? 0 : red[1][u].gx * ceil_div(q.M, kBatchColRows));
    red_start[2][u + 1] = red_start[2][u] + (direct ? 0 : red[2][u].gx * ceil_div(q.K, kBatchColRows));
    red_start[3][u + 1] = red_start[3][u] + (direct ? 0 : q.K);
    // passes and multiply
    const Source x = batch_source_a(q, p, dt, o_step ? eA : nullptr, i_step ? d : nullptr);
    const Source y = batch_source_b(q, p, dt, i_step ? d : nullptr, o_step ? eB : nullptr);
    const PassGeom& g = L.geom[u];
    char* wa = ws + L.off_a[u];
    char* wb = ws + L.off_b[u];
    float* mbuf = (fused || g.R == 1) ? nullptr : reinterpret_cast<float*>(ws + L.off_m[u]);
    comb[2 * u] = combine_args(p, g, x, 0, leaves, wa);
    comb[2 * u + 1] = combine_args(p, g, y, 1, leaves, wb);
    for (int sd = 0; sd < 2 && !direct; ++sd) {
      const CombineArgs& ca = comb[2 * u + (size_t)sd];
      if (ca.n_rb == 1 && ca.n_cb == 1 && g.R == 1 && ca.t_nnz == 1) {
        // one term of one block: a plain scaled conversion
        plain.push_back(ca);
        copy_start.push_back(copy_start.back() + convert_batched_ctas(ca));
      } else {
        staged.push_back(ca);
        comb_start.push_back(comb_start.back() + (ca.p_rows / b->comb_tr) * (ca.p_cols / 64));
        b->comb_smem = std::max(b->comb_smem, combine_staged_smem(ca.n_rb * ca.n_cb, b->comb_tr, ca.t_nnz, g.R));
      }
    }
    EpilogueArgs c;
    c.C = q.C;
    c.ldc = q.ldc;
    c.M = q.M;
    c.N = q.N;
    c.bm = ceil_div(q.M, p->pm);
    c.bn = ceil_div(q.N, p->pn);
    c.eA = (o_step && !direct) ? eA : nullptr;
    c.eB = (o_step && !direct) ? eB : nullptr;
    c.vec_ok = ((uintptr_t)q.C % 16 == 0) && (q.ldc % 4 == 0) && (c.bn % 4 == 0) ? 1 : 0;
    if (!direct_args(p, g, x, y, c, leaves, wa, wb, mbuf, b->status, &dir[u])) return FMM_ERR_CUDA;
    if (direct) {
      // the caller's matrices themselves: A K-major (M x K), B MN-major (K x N)
      if (!make_map_sw(&dir[u].map_a, q.A, false, q.M, q.K, q.lda, 64, 128) ||
          !make_map_sw(&dir[u].map_b, q.B, false, q.K, q.N, q.ldb, 64, 64))
        return FMM_ERR_CUDA;
      // and C written by bulk tensor stores where its rows allow (the
      // stores clip the tiles' padding at C's edges)
      dir[u].tma_store = 0;
      if (tma_store_enabled() && (uintptr_t)q.C % 16 == 0 && (q.ldc * 4) % 16 == 0 && q.M >= 32 && q.N >= 32) {
        if (!make_map_f32_sw128(&dir[u].map_m, q.C, q.M, q.N, q.ldc)) return FMM_ERR_CUDA;
        dir[u].tma_store = 1;
      }
    }
    const int64_t tiles = (g.tp_a / tm_rows) * (g.tp_b / tn_cols);
    units[u] = mbuf ? g.R * tiles : tiles;
    unit_cost[u] = (mbuf ? 1 : g.R) * (g.kp / 64);
    if (mbuf) {
      out.push_back(out_args(p, g, c, leaves, mbuf));
      const OutArgs& o = out.back();
      out_start.push_back(out_start.back() + ceil_div(c.bm, b->out_tr) * ceil_div(c.bn, 64));
      b->out_smem = std::max(b->out_smem, (size_t)(p->pm * p->pn * b->out_tr * 256 + o.c_nnz * 8 +
                                                   (o.num_leaves + 1) * 4));
    }
  }
  // Multiply table ordered by decreasing work per unit, so the round-robin
  // assignment of units to CTAs hands out the long units first.
  std::vector<int> order((size_t)count);
  for (int i = 0; i < count; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return unit_cost[(size_t)x] > unit_cost[(size_t)y]; });
  {
    std::vector<DirectArgs> sorted((size_t)count);
    for (int i = 0; i < count; ++i) {
      sorted[(size_t)i] = dir[(size_t)order[(size_t)i]];
      unit_start[(size_t)i + 1] = unit_start[(size_t)i] + units[(size_t)order[(size_t)i]];
    }
    dir.swap(sorted);
  }
  b->out_count = (int)out.size();
  if (b->comb_smem > 200 * 1024 || b->out_smem > 200 * 1024) {
    t_last_error = "batch: a plan's term lists do not fit the passes' shared memory";
    return FMM_ERR_UNSUPPORTED;
  }
  for (int k = 0; k < 4; ++k) b->red_total[k] = red_start[k][(size_t)count];
  b->comb_total = comb_start.back();
  b->copy_total = copy_start.back();
  b->comb_count = (int)staged.size();
  b->copy_count = (int)plain.size();
  comb = staged;
  comb.insert(comb.end(), plain.begin(), plain.end());
  b->unit_total = unit_start[(size_t)count];
  b->out_total = out_start.back();
  b->layout = dir[0];
  // copy the tables into the workspace
  auto put = [&](size_t off, const void* src, size_t bytes) {
    return cuda_ok(cudaMemcpy(ws + off, src, bytes, cudaMemcpyHostToDevice), "batch table copy");
  };
  for (int k = 0; k < 4; ++k)
    if (!put(L.off_red[k], red[k].data(), red[k].size() * sizeof(ReduceArgs)) ||
        !put(L.off_red_start[k], red_start[k].data(), red_start[k].size() * 8))
      return FMM_ERR_CUDA;
  if (!put(L.off_comb, comb.data(), comb.size() * sizeof(CombineArgs)) ||
      !put(L.off_comb_start, comb_start.data(), comb_start.size() * 8) ||
      !put(L.off_copy_start, copy_start.data(), copy_start.size() * 8) ||
      !put(L.off_direct, dir.data(), dir.size() * sizeof(DirectArgs)) ||
      !put(L.off_unit_start, unit_start.data(), unit_start.size() * 8) ||
      (!out.empty() && !put(L.off_out, out.data(), out.size() * sizeof(OutArgs))) ||
      !put(L.off_out_start, out_start.data(), out_start.size() * 8))
    return FMM_ERR_CUDA;
  return FMM_OK;
}

static fmm_status batch_run(const Batch* b, cudaStream_t st) {
  const BatchLayout& L = b->L;
  char* ws = b->ws;
  int* eA_all = reinterpret_cast<int*>(ws + L.off_exp);
  int* d_all = eA_all + L.sum_m;
  int* eB_all = d_all + L.sum_k;
  auto red = [&](int k) { return reinterpret_cast<const ReduceArgs*>(ws + L.off_red[k]); };
  auto red_start = [&](int k) { return reinterpret_cast<const int64_t*>(ws + L.off_red_start[k]); };
  const bool o_step = (b->steps & 1) && b->any_scaled, i_step = (b->steps & 2) && b->any_scaled;
  const int n = b->count;
  if (o_step && i_step) {
    // rows(A) -> eA; columns(2^-eA A) -> d; columns(B) -> eB; rows(2^-eB B) with d -> d
    if (!cuda_ok(launch_fill(d_all, L.sum_k + L.sum_n, kZeroExp, st), "batch fill") ||
        !cuda_ok(launch_row_exp_batched(red(0), red_start(0), n, b->red_total[0], b->dt, false, kRowOStep, b->status, st),
                 "batch row reduction") ||
        !cuda_ok(launch_col_exp_batched(red(1), red_start(1), n, b->red_total[1], b->dt, true, b->status, st),
                 "batch column reduction") ||
        !cuda_ok(launch_col_exp_batched(red(2), red_start(2), n, b->red_total[2], b->dt, false, b->status, st),
                 "batch column reduction") ||
        !cuda_ok(launch_zero_sentinel(eB_all, L.sum_n, st), "batch fix-up") ||
        !cuda_ok(launch_row_exp_batched(red(3), red_start(3), n, b->red_total[3], b->dt, true, kRowIStep, b->status, st),
                 "batch row reduction"))
      return FMM_ERR_CUDA;
  } else if (o_step) {
    if (!cuda_ok(launch_fill(eB_all, L.sum_n, kZeroExp, st), "batch fill") ||
        !cuda_ok(launch_row_exp_batched(red(0), red_start(0), n, b->red_total[0], b->dt, false, kRowOStep, b->status, st),
                 "batch row reduction") ||
        !cuda_ok(launch_col_exp_batched(red(2), red_start(2), n, b->red_total[2], b->dt, false, b->status, st),
                 "batch column reduction") ||
        !cuda_ok(launch_zero_sentinel(eB_all, L.sum_n, st), "batch fix-up"))
      return FMM_ERR_CUDA;
  } else if (i_step) {
    if (!cuda_ok(launch_fill(d_all, L.sum_k, kZeroExp, st), "batch fill") ||
        !cuda_ok(launch_col_exp_batched(red(1), red_start(1), n, b->red_total[1], b->dt, false, b->status, st),
                 "batch column reduction") ||
        !cuda_ok(launch_row_exp_batched(red(3), red_start(3), n, b->red_total[3], b->dt, false, kRowIStep, b->status, st),
                 "batch row reduction"))
      return FMM_ERR_CUDA;
  }
  const CombineArgs* comb = reinterpret_cast<const CombineArgs*>(ws + L.off_comb);
  if (!cuda_ok(launch_combine_batched(comb, reinterpret_cast<const int64_t*>(ws + L.off_comb_start), b->comb_count,
                                      b->comb_total, b->dt, b->fmt, b->comb_tr, b->comb_smem, st),
               "batch combination pass") ||
      !cuda_ok(launch_convert_batched(comb + b->comb_count, reinterpret_cast<const int64_t*>(ws + L.off_copy_start),
                                      b->copy_count, b->copy_total, b->dt, b->fmt, st),
               "batch conversion pass") ||
      !cuda_ok(b->pairs ? launch_pair_gemm_batched(b->layout, reinterpret_cast<const DirectArgs*>(ws + L.off_direct),
                                                   reinterpret_cast<const int64_t*>(ws + L.off_unit_start), n,
                                                   b->unit_total, b->fmt, st)
                        : launch_direct_gemm_batched(b->layout, reinterpret_cast<const DirectArgs*>(ws + L.off_direct),
                                                     reinterpret_cast<const int64_t*>(ws + L.off_unit_start), n,
                                                     b->unit_total, b->fmt, kBatchTileN, st),
               "batch multiply") ||
      !cuda_ok(launch_out_combine_batched(reinterpret_cast<const OutArgs*>(ws + L.off_out),
                                          reinterpret_cast<const int64_t*>(ws + L.off_out_start), b->out_count,
                                          b->out_total, b->out_tr, b->out_smem, st),
               "batch output pass"))
    return FMM_ERR_CUDA;
  return FMM_OK;
}

}  // namespace fmm

using namespace fmm;

extern "C" {

fmm_status fmm_plan(fmm_plan_t* out, int levels, const fmm_rule* rules, int leaf_format) {
  if (!out || levels < 0 || levels > 16 || (levels > 0 && !rules)) return FMM_ERR_ARG;
  *out = nullptr;
  std::vector<CanonRule> cr((size_t)levels);
  for (int l = 0; l < levels; ++l) {
    fmm_status s = canonicalize(rules[l], &cr[(size_t)l]);
    if (s != FMM_OK) return s;
  }
  Plan* p = nullptr;
  fmm_status s = make_plan(cr, leaf_format, &p);
  if (s != FMM_OK) return s;
  *out = reinterpret_cast<fmm_plan_t>(p);
  return FMM_OK;
}

fmm_status fmm_plan_tree(fmm_plan_t* out, int nrules, const fmm_rule* rules, int levels, int64_t nnodes,
                         const int32_t* node_rule, int leaf_format) {
  if (!out || nrules < 1 || !rules || levels < 1 || levels > 16 || nnodes < 1 || nnodes > (1 << 20) || !node_rule)
    return FMM_ERR_ARG;
  *out = nullptr;
  std::vector<CanonRule> cr((size_t)nrules);
  for (int i = 0; i < nrules; ++i) {
    fmm_status s = canonicalize(rules[i], &cr[(size_t)i]);
    if (s != FMM_OK) return s;
  }
  const std::vector<int> nr(node_rule, node_rule + nnodes);
  Plan* p = nullptr;
  fmm_status s = make_plan(cr, leaf_format, &p, &nr, levels);
  if (s != FMM_OK) return s;
  *out = reinterpret_cast<fmm_plan_t>(p);
  return FMM_OK;
}

fmm_status fmm_rule_rotate(const fmm_rule* in, double* U, double* V, double* W, fmm_rule* out) {
  if (!in || !U || !V || !W || !out) return FMM_ERR_ARG;
  return rule_rotate(*in, U, V, W, out);
}

fmm_status fmm_rule_compose(const fmm_rule* outer, const fmm_rule* inner, double* U, double* V, double* W,
                            fmm_rule* out) {
  if (!outer || !inner || !U || !V || !W || !out) return FMM_ERR_ARG;
  return rule_compose(*outer, *inner, U, V, W, out);
}

fmm_status fmm_rule_transform(const fmm_rule* in, const double* XU, const double* XV, const double* XW, double* U,
                              double* V, double* W, fmm_rule* out) {
  if (!in || !U || !V || !W || !out) return FMM_ERR_ARG;
  return rule_transform(*in, XU, XV, XW, U, V, W, out);
}

fmm_status fmm_rule_permute(const fmm_rule* in, const int32_t* perm_i, const int32_t* perm_k, const int32_t* perm_j,
                            double* U, double* V, double* W, fmm_rule* out) {
  if (!in || !U || !V || !W || !out) return FMM_ERR_ARG;
  return rule_permute(*in, perm_i, perm_k, perm_j, U, V, W, out);
}

fmm_status fmm_plan_variants(fmm_plan_t* out, const fmm_rule* base, int levels, int selection, uint64_t seed,
                             const float* block_max_a, const float* block_max_b, int32_t* chosen,
                             int leaf_format) {
  if (!out || !base || levels < 1 || levels > 8) return FMM_ERR_ARG;
  *out = nullptr;
  CanonRule c;
  fmm_status s = canonicalize(*base, &c);
  if (s != FMM_OK) return s;
  if (brent_violations(c)) return FMM_ERR_NOT_MATMUL;
  std::vector<int> nr;
  if ((s = cg_select(c, levels, selection, seed, block_max_a, block_max_b, &nr)) != FMM_OK) return s;
  std::vector<CanonRule> table(8);
  for (int v = 0; v < 8; ++v) table[(size_t)v] = cg_variant(c, v);
  Plan* p = nullptr;
  if ((s = make_plan(table, leaf_format, &p, &nr, levels)) != FMM_OK) return s;
  if (chosen)
    for (size_t i = 0; i < nr.size(); ++i) chosen[i] = nr[i];
  *out = reinterpret_cast<fmm_plan_t>(p);
  return FMM_OK;
}

fmm_status fmm_block_max(const void* X, int dtype, int64_t rows, int64_t cols, int64_t ld, int nrb, int ncb,
                         float* out, void* stream) {
  if (!valid_dtype(dtype) || rows < 0 || cols < 0 || nrb < 1 || ncb < 1 || nrb > 64 || ncb > 64 || !out)
    return FMM_ERR_ARG;
  if (rows > 0 && cols > 0 && (!X || ld < cols)) return FMM_ERR_ARG;
  int* status = status_ptr();
  if (!status) return FMM_ERR_CUDA;
  return cuda_ok(launch_block_max(X, dtype, rows, cols, ld, nrb, ncb, out, status, as_stream(stream)), "block max")
             ? FMM_OK
             : FMM_ERR_CUDA;
}

fmm_status fmm_plan_destroy(fmm_plan_t plan) {
  destroy_plan(reinterpret_cast<Plan*>(plan));
  return FMM_OK;
}

fmm_status fmm_plan_set_schedule(fmm_plan_t plan, int schedule) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || schedule < FMM_SCHEDULE_AUTO || schedule > FMM_SCHEDULE_PASS_ACCUMULATE) return FMM_ERR_ARG;
  p->schedule = schedule;
  if (p->grad_a) p->grad_a->schedule = schedule;
  if (p->grad_b) p->grad_b->schedule = schedule;
  return FMM_OK;
}

fmm_status fmm_plan_set_between_scaling(fmm_plan_t plan, int enable) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return FMM_ERR_ARG;
  // a level-1 product's leaves are contiguous and equally many only when
  // every level's ranks agree
  if (enable && !p->level_r_uniform) return FMM_ERR_UNSUPPORTED;
  if (enable && p->levels >= 2 && !p->level1) {
    fmm_status s = make_plan({p->rules[0]}, p->leaf_format, &p->level1);
    if (s != FMM_OK) return s;
  }
  p->between = enable ? 1 : 0;
  return FMM_OK;
}

fmm_status fmm_plan_info(fmm_plan_t plan, double* q_sum, double* e_prod, int64_t* leaves, int64_t* nnz,
                         int64_t* pm, int64_t* pk, int64_t* pn) {
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  if (!p) return FMM_ERR_ARG;
  if (q_sum) *q_sum = p->q_sum;
  if (e_prod) *e_prod = p->e_prod;
  if (leaves) *leaves = p->leaves;
  if (nnz) *nnz = p->nnz;
  if (pm) *pm = p->pm;
  if (pk) *pk = p->pk;
  if (pn) *pn = p->pn;
  return FMM_OK;
}

fmm_status fmm_plan_flatten(fmm_plan_t plan, int table, double* U, double* V, double* W, int32_t* first) {
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  if (!p || table < FMM_TABLE_LEAVES || table > FMM_TABLE_GATHER) return FMM_ERR_ARG;
  if (table == FMM_TABLE_GATHER && p->gather_off < 0) return FMM_ERR_UNSUPPORTED;
  const int64_t R = p->leaves;
  const int64_t rows[3] = {p->pm * p->pk, p->pk * p->pn, p->pm * p->pn};
  const int64_t grid_cols[3] = {p->pk, p->pn, p->pn};
  double* out[3] = {U, V, W};
  if (table == FMM_TABLE_GATHER) out[0] = out[1] = nullptr;
  for (int s = 0; s < 3; ++s)
    if (out[s]) std::fill(out[s], out[s] + rows[s] * R, 0.0);
  if (first) std::fill(first, first + rows[2] * R, 0);
  // one term: coefficient c of block blk ((row << 16) | col) in leaf r
  auto put = [&](int s, int32_t blk, int64_t r, float c, bool is_first) {
    const int64_t i = (int64_t)((blk & 0x7FFFFFFF) >> 16) * grid_cols[s] + (blk & 0xFFFF);
    if (out[s]) out[s][i * R + r] += (double)c;
    if (s == 2 && first && is_first) first[i * R + r] = 1;
  };
  if (table == FMM_TABLE_LEAVES) {
    for (int64_t r = 0; r < R; ++r) {
      const LeafDesc& d = p->host[(size_t)r];
      for (int t = 0; t < d.na; ++t) put(0, d.a_blk[t], r, d.a_coef[t], false);
      for (int t = 0; t < d.nb; ++t) put(1, d.b_blk[t], r, d.b_coef[t], false);
      for (int t = 0; t < d.nc; ++t) put(2, d.c_blk[t], r, d.c_coef[t], d.c_first[t] != 0);
    }
  } else if (table == FMM_TABLE_LISTS) {
    for (int s = 0; s < 3; ++s) {
      const int32_t* start = p->lists.data() + p->list_off[s];
      const int32_t* blk = start + R + 1;
      const int32_t* coef = blk + p->list_nnz[s];
      for (int64_t r = 0; r < R; ++r)
        for (int32_t t = start[r]; t < start[r + 1]; ++t) {
          float c;
          std::memcpy(&c, &coef[t], 4);
          put(s, blk[t], r, c, (blk[t] & kFirstBit) != 0);
        }
    }
  } else {
    const int64_t nblk = rows[2];
    const int32_t* gstart = p->lists.data() + p->gather_off;
    const int32_t* gleaf = gstart + nblk + 1;
    const int32_t* gcoef = gleaf + p->list_nnz[2];
    for (int64_t k = 0; k < nblk; ++k)
      for (int32_t t = gstart[k]; t < gstart[k + 1]; ++t) {
        float c;
        std::memcpy(&c, &gcoef[t], 4);
        if (W) W[k * R + gleaf[t]] += (double)c;
        if (first && t == gstart[k]) first[k * R + gleaf[t]] = 1;
      }
  }
  return FMM_OK;
}

fmm_status fmm_plan_bound(fmm_plan_t plan, int64_t K, double normA, double normB, double eps, double* bound) {
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  if (!p || !bound || K < 0) return FMM_ERR_ARG;
  const double kl = (double)((K + p->pk - 1) / p->pk);
  *bound = (kl + p->q_sum) * kl * p->e_prod * normA * normB * eps;
  return FMM_OK;
}

fmm_status fmm_scale_outside(const void* A, const void* B, int dtype, int64_t M, int64_t K, int64_t N,
                             int64_t lda, int64_t ldb, const int32_t* d_in, int32_t* eA, int32_t* eB,
                             void* stream) {
  if (!valid_dtype(dtype) || M < 0 || K < 0 || N < 0) return FMM_ERR_ARG;
  if ((M > 0 && !eA) || (N > 0 && !eB)) return FMM_ERR_ARG;
  if ((M > 0 && K > 0 && !A) || (K > 0 && N > 0 && !B)) return FMM_ERR_ARG;
  if ((M > 0 && K > 0 && lda < K) || (K > 0 && N > 0 && ldb < N)) return FMM_ERR_SHAPE;
  int* status = status_ptr();
  if (!status) return FMM_ERR_CUDA;
  cudaStream_t st = as_stream(stream);
  // eA_i = e(max_k |A_ik| 2^d_k): row reduction of A with column shifts +d.
  if (K == 0) {
    if (launch_fill(eA, M, 0, st) != cudaSuccess) return FMM_ERR_CUDA;
    if (launch_fill(eB, N, 0, st) != cudaSuccess) return FMM_ERR_CUDA;
    return FMM_OK;
  }
  if (!cuda_ok(launch_row_exp(A, dtype, M, K, lda, d_in, +1, eA, kRowOStep, status, st), "row reduction"))
    return FMM_ERR_CUDA;
  // eB_j = e(max_k 2^-d_k |B_kj|): column reduction of B with row shifts -d.
  if (!cuda_ok(launch_col_exp(B, dtype, K, N, ldb, d_in, -1, eB, status, st), "column reduction"))
    return FMM_ERR_CUDA;
  if (launch_zero_sentinel(eB, N, st) != cudaSuccess) return FMM_ERR_CUDA;
  return FMM_OK;
}

fmm_status fmm_scale_inside(const void* A, const void* B, int dtype, int64_t M, int64_t K, int64_t N,
                            int64_t lda, int64_t ldb, const int32_t* eA, const int32_t* eB, int32_t* d,
                            void* stream) {
  if (!valid_dtype(dtype) || M < 0 || K < 0 || N < 0) return FMM_ERR_ARG;
  if (K > 0 && !d) return FMM_ERR_ARG;
  if ((M > 0 && K > 0 && !A) || (K > 0 && N > 0 && !B)) return FMM_ERR_ARG;
  if ((M > 0 && K > 0 && lda < K) || (K > 0 && N > 0 && ldb < N)) return FMM_ERR_SHAPE;
  int* status = status_ptr();
  if (!status) return FMM_ERR_CUDA;
  cudaStream_t st = as_stream(stream);
  if (K == 0) return FMM_OK;
  // d_k <- e(max_i 2^-eA_i |A_ik|): column reduction of A (kZeroExp if 0).
  if (launch_col_exp(A, dtype, M, K, lda, eA, -1, d, status, st) != cudaSuccess) return FMM_ERR_CUDA;
  // d_k <- floor((e(max_j |B_kj| 2^-eB_j) - d_k) / 2): row reduction of B.
  if (launch_row_exp(B, dtype, K, N, ldb, eB, -1, d, kRowIStep, status, st) != cudaSuccess) return FMM_ERR_CUDA;
  if (N == 0 && launch_fill(d, K, 0, st) != cudaSuccess) return FMM_ERR_CUDA;
  return FMM_OK;
}

// The step pair O, I of Alg. 3 starting from d = 0 (M, K, N > 0): the same
// exponents as fmm_scale_outside then fmm_scale_inside, in two launches
// (rows of A and column panels of B; then, per k panel, the columns of A
// and rows of B) that need no initialised outputs.
static fmm_status scale_oi_from_zero(const void* A, const void* B, int dtype, int64_t M, int64_t K, int64_t N,
                                     int64_t lda, int64_t ldb, int32_t* eA, int32_t* d, int32_t* eB,
                                     cudaStream_t st) {
  if (!valid_dtype(dtype) || !A || !B || !eA || !d || !eB) return FMM_ERR_ARG;
  if (lda < K || ldb < N) return FMM_ERR_SHAPE;
  int* status = status_ptr();
  if (!status) return FMM_ERR_CUDA;
  return cuda_ok(launch_oi_from_zero(A, B, dtype, M, K, N, lda, ldb, eA, d, eB, status, st), "O-I reductions")
             ? FMM_OK
             : FMM_ERR_CUDA;
}

fmm_status fmm_scale(const char* steps, const void* A, const void* B, int dtype, int64_t M, int64_t K, int64_t N,
                     int64_t lda, int64_t ldb, int32_t* eA, int32_t* d, int32_t* eB, void* stream) {
  if (!steps || !valid_dtype(dtype) || M < 0 || K < 0 || N < 0) return FMM_ERR_ARG;
  bool has_o = false, has_i = false;
  for (const char* c = steps; *c; ++c) {
    if (*c != 'O' && *c != 'I') return FMM_ERR_ARG;
    has_o |= *c == 'O';
    has_i |= *c == 'I';
  }
  if ((M > 0 && !eA) || (K > 0 && !d) || (N > 0 && !eB)) return FMM_ERR_ARG;
  // The steps' own checks, made before the fills below launch anything.
  if (steps[0] && ((M > 0 && K > 0 && !A) || (K > 0 && N > 0 && !B))) return FMM_ERR_ARG;
  if (steps[0] && ((M > 0 && K > 0 && lda < K) || (K > 0 && N > 0 && ldb < N))) return FMM_ERR_SHAPE;
  cudaStream_t st = as_stream(stream);
  // Every vector starts at zero (no scaling).  A vector that some step
  // overwrites completely needs no fill; and while a vector is still all
  // zeros the steps that read it are told so (no shift), which selects the
  // unshifted reductions.
  if (!has_o && (launch_fill(eA, M, 0, st) != cudaSuccess || launch_fill(eB, N, 0, st) != cudaSuccess))
    return FMM_ERR_CUDA;
  if (!has_i && launch_fill(d, K, 0, st) != cudaSuccess) return FMM_ERR_CUDA;
  bool d_zero = true, e_zero = true;
  for (const char* c = steps; *c; ++c) {
    if (c[0] == 'O' && c[1] == 'I' && d_zero && M > 0 && K > 0 && N > 0) {
      // An O step on unshifted operands followed by an I step: the I step's
      // column pass over A needs only eA, so each operand's two passes run
      // back to back (the second one mostly from L2): rows of A, columns of
      // A, columns of B, rows of B.
      fmm_status s = scale_oi_from_zero(A, B, dtype, M, K, N, lda, ldb, eA, d, eB, st);
      if (s != FMM_OK) return s;
      e_zero = d_zero = false;
      ++c;
      continue;
    }
    fmm_status s = *c == 'O'
                       ? fmm_scale_outside(A, B, dtype, M, K, N, lda, ldb, d_zero ? nullptr : d, eA, eB, stream)
                       : fmm_scale_inside(A, B, dtype, M, K, N, lda, ldb, e_zero ? nullptr : eA,
                                          e_zero ? nullptr : eB, d, stream);
    if (s != FMM_OK) return s;
    if (*c == 'O') e_zero = false;
    else d_zero = false;
  }
  return FMM_OK;
}

fmm_status fmm_scale_adaptive(const void* A, const void* B, int dtype, int64_t M, int64_t K, int64_t N,
                              int64_t lda, int64_t ldb, double tau, int max_steps, int first_inside,
                              int32_t* eA, int32_t* d, int32_t* eB, int32_t* steps_taken, void* ws,
                              size_t ws_bytes, void* stream) {
  if (!valid_dtype(dtype) || M < 0 || K < 0 || N < 0 || max_steps < 0 || max_steps > 100000) return FMM_ERR_ARG;
  if (!(tau > 0) || !std::isfinite(tau) || (first_inside != 0 && first_inside != 1)) return FMM_ERR_ARG;
  if ((M > 0 && !eA) || (K > 0 && !d) || (N > 0 && !eB)) return FMM_ERR_ARG;
  if ((M > 0 && K > 0 && !A) || (K > 0 && N > 0 && !B)) return FMM_ERR_ARG;
  if ((M > 0 && K > 0 && lda < K) || (K > 0 && N > 0 && ldb < N)) return FMM_ERR_SHAPE;
  if (!ws || (uintptr_t)ws % 16 != 0 || (int64_t)ws_bytes < 4 * (M + K + N + 64)) return FMM_ERR_WORKSPACE;
  int* status = status_ptr();
  if (!status) return FMM_ERR_CUDA;
  cudaStream_t st = as_stream(stream);
  // workspace: ctl[64] (stopped, failed, steps applied), then the exponents
  // a step computes before its test adopts them
  int* ctl = static_cast<int*>(ws);
  int* nA = ctl + 64;
  int* nB = nA + M;
  int* nD = nB + N;
  // The tests in exponent form: an O factor 2^g passes when
  // g >= -log2(1 + tau) / 2, an I factor when |g| <= log2(1 + tau) / 4.
  const double l2 = std::log2(1.0 + tau);
  const int o_lo = (int)std::max(-1e9, std::ceil(-l2 / 2)), i_hi = (int)std::min(1e9, std::floor(l2 / 4));
  if (launch_fill(ctl, 64, 0, st) != cudaSuccess || launch_fill(eA, M, 0, st) != cudaSuccess ||
      launch_fill(d, K, 0, st) != cudaSuccess || launch_fill(eB, N, 0, st) != cudaSuccess)
    return FMM_ERR_CUDA;
  if (steps_taken && launch_fill(steps_taken, 1, 0, st) != cudaSuccess) return FMM_ERR_CUDA;
  // while a vector is still all zeros its reductions run unshifted
  bool d_zero = true, e_zero = true, seen_o = false;
  for (int t = 1; t <= max_steps; ++t) {
    const bool o = ((t - 1) % 2 == 0) == (first_inside == 0);
    const bool tested = seen_o;  // every step after the first O step
    if (o) {
      // eA_i = e(max_k |A_ik| 2^d_k), eB_j = e(max_k 2^-d_k |B_kj|)
      if (K == 0) {
        if (launch_fill(nA, M, 0, st) != cudaSuccess || launch_fill(nB, N, 0, st) != cudaSuccess) return FMM_ERR_CUDA;
      } else if (!cuda_ok(launch_row_exp(A, dtype, M, K, lda, d_zero ? nullptr : d, +1, nA, kRowOStep, status, st,
                                         ctl),
                          "row reduction") ||
                 !cuda_ok(launch_col_exp(B, dtype, K, N, ldb, d_zero ? nullptr : d, -1, nB, status, st, ctl),
                          "column reduction") ||
                 launch_zero_sentinel(nB, N, st) != cudaSuccess) {
        return FMM_ERR_CUDA;
      }
      if (launch_scale_accept(nA, eA, M, o_lo, INT32_MAX, ctl, st) != cudaSuccess ||
          launch_scale_accept(nB, eB, N, o_lo, INT32_MAX, ctl, st) != cudaSuccess)
        return FMM_ERR_CUDA;
      e_zero = false;
      seen_o = true;
    } else if (K > 0) {
      // d_k = floor((e(max_j |B_kj| 2^-eB_j) - e(max_i 2^-eA_i |A_ik|)) / 2)
      if (!cuda_ok(launch_col_exp(A, dtype, M, K, lda, e_zero ? nullptr : eA, -1, nD, status, st, ctl),
                   "column reduction") ||
          !cuda_ok(launch_row_exp(B, dtype, K, N, ldb, e_zero ? nullptr : eB, -1, nD, kRowIStep, status, st, ctl),
                   "row reduction"))
        return FMM_ERR_CUDA;
      if (N == 0 && launch_fill(nD, K, 0, st) != cudaSuccess) return FMM_ERR_CUDA;
      if (launch_scale_accept(nD, d, K, -i_hi, i_hi, ctl, st) != cudaSuccess) return FMM_ERR_CUDA;
      d_zero = false;
    }
    if (launch_scale_stop(ctl, tested ? 1 : 0, t, steps_taken, st) != cudaSuccess) return FMM_ERR_CUDA;
  }
  return FMM_OK;
}

fmm_status fmm_workspace_size(fmm_plan_t plan, int64_t M, int64_t K, int64_t N, size_t* bytes) {
  if (!plan || !bytes || M < 0 || K < 0 || N < 0) return FMM_ERR_ARG;
  *bytes = ws_bytes_for(reinterpret_cast<const Plan*>(plan), M, K, N);
  return FMM_OK;
}

fmm_status fmm_multiply(fmm_plan_t plan, const void* A, int64_t lda, const void* B, int64_t ldb, float* C,
                        int64_t ldc, int64_t M, int64_t K, int64_t N, int in_dtype, const int32_t* eA,
                        const int32_t* d, const int32_t* eB, void* ws, size_t ws_bytes, void* stream) {
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  if (!p || !valid_dtype(in_dtype) || M < 0 || K < 0 || N < 0) return FMM_ERR_ARG;
  if (M > 0 && N > 0 && !C) return FMM_ERR_ARG;
  if ((M > 0 && K > 0 && !A) || (K > 0 && N > 0 && !B)) return FMM_ERR_ARG;
  if ((M > 0 && K > 0 && lda < K) || (K > 0 && N > 0 && ldb < N) || (M > 0 && N > 0 && ldc < N))
    return FMM_ERR_SHAPE;
  if (in_dtype == FMM_DT_F16 && p->leaf_format == FMM_LEAF_BF16X3) return FMM_ERR_DTYPE;
  if (ceil_div(M, p->pm) >= (1ll << 30) || ceil_div(N, p->pn) >= (1ll << 30) || ceil_div(K, p->pk) >= (1ll << 30))
    return FMM_ERR_SHAPE;
  // A: t = M (rows of A), k = K (columns): k-contiguous; rows scaled by
  // 2^-eA, columns by 2^d.  B: t = N (columns of B), k = K (rows):
  // t-contiguous; rows scaled by 2^-d, columns by 2^-eB (Algs. 1-3).
  const Source a{A, lda, in_dtype, true, M, K, p->pm, p->pk, eA, -1, d, +1};
  const Source b{B, ldb, in_dtype, false, N, K, p->pn, p->pk, d, -1, eB, -1};
  return run_plan(p, a, b, C, ldc, M, K, N, eA, eB, ws, ws_bytes, as_stream(stream));
}

fmm_status fmm_multiply_noalloc(fmm_plan_t plan, const void* A, int64_t lda, const void* B, int64_t ldb,
                                float* C, int64_t ldc, int64_t M, int64_t K, int64_t N, int in_dtype,
                                const int32_t* eA, const int32_t* d, const int32_t* eB, void* stream) {
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  if (!p || !valid_dtype(in_dtype) || M < 0 || K < 0 || N < 0) return FMM_ERR_ARG;
  if (M > 0 && N > 0 && !C) return FMM_ERR_ARG;
  if ((M > 0 && K > 0 && !A) || (K > 0 && N > 0 && !B)) return FMM_ERR_ARG;
  if ((M > 0 && K > 0 && lda < K) || (K > 0 && N > 0 && ldb < N) || (M > 0 && N > 0 && ldc < N))
    return FMM_ERR_SHAPE;
  if (in_dtype == FMM_DT_F16 && p->leaf_format == FMM_LEAF_BF16X3) return FMM_ERR_DTYPE;
  if (ceil_div(M, p->pm) >= (1ll << 30) || ceil_div(N, p->pn) >= (1ll << 30) || ceil_div(K, p->pk) >= (1ll << 30))
    return FMM_ERR_SHAPE;
  if (M == 0 || N == 0) return FMM_OK;
  if (K == 0) return run_plan(p, Source{}, Source{}, C, ldc, M, K, N, nullptr, nullptr, nullptr, 0, as_stream(stream));
  // The size check comes before any device call.  The workspace part is
  // the one of the path run_plan takes with this much room: the pass
  // schedule's combined operands and stored products (E4M3 leaves and the
  // forced pass schedules always take it), or the load-stage schedule's
  // prepared operand copies (the automatic schedule takes whichever fits,
  // the pass schedule first).
  const size_t leaf_bytes = p->host.size() * sizeof(LeafDesc);
  const size_t table_bytes = leaf_bytes + p->lists.size() * 4;
  const size_t table = (size_t)round_up((int64_t)table_bytes, 256);
  const int64_t pass_need = pass_bytes(p, M, K, N, p->pm, p->pk, p->pn);
  const int64_t stage_need = prepared_bytes(M, K, p->pm, p->pk) + prepared_bytes(N, K, p->pn, p->pk);
  const bool pass_only = p->leaf_format == FMM_LEAF_E4M3B128 || p->schedule == FMM_SCHEDULE_PASS ||
                         p->schedule == FMM_SCHEDULE_PASS_EPILOGUE || p->schedule == FMM_SCHEDULE_PASS_PRODUCTS ||
                         p->schedule == FMM_SCHEDULE_PASS_ACCUMULATE;
  const int64_t ws_need = pass_only ? pass_need
                          : p->schedule == FMM_SCHEDULE_LOAD_STAGE ? stage_need
                                                                   : std::min(pass_need, stage_need);
  const size_t need = table + (size_t)ws_need;
  if (need > FMM_NOALLOC_SCRATCH_BYTES) {
    t_last_error = "fmm_multiply_noalloc: this problem needs " + std::to_string(need) +
                   " bytes of scratch; the static scratch holds " + std::to_string(FMM_NOALLOC_SCRATCH_BYTES);
    return FMM_ERR_WORKSPACE;
  }
  char* scratch = noalloc_scratch();
  if (!scratch) return FMM_ERR_CUDA;
  cudaStream_t st = as_stream(stream);
  if (!upload_words(reinterpret_cast<uint32_t*>(scratch), p->host.data(), leaf_bytes / 4, st) ||
      !upload_words(reinterpret_cast<uint32_t*>(scratch + leaf_bytes), p->lists.data(), p->lists.size(), st))
    return FMM_ERR_CUDA;
  // Operands as in fmm_multiply.
  const Source a{A, lda, in_dtype, true, M, K, p->pm, p->pk, eA, -1, d, +1};
  const Source b{B, ldb, in_dtype, false, N, K, p->pn, p->pk, d, -1, eB, -1};
  return run_plan(p, a, b, C, ldc, M, K, N, eA, eB, scratch + table, FMM_NOALLOC_SCRATCH_BYTES - table, st,
                  reinterpret_cast<const LeafDesc*>(scratch), /*allow_between=*/false);
}

fmm_status fmm_plan_gradient(fmm_plan_t plan, int which, fmm_plan_t* out) {
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  if (!p || !out || (which != FMM_GRAD_A && which != FMM_GRAD_B)) return FMM_ERR_ARG;
  *out = nullptr;
  // the same rule transforms and plan compiler calls as the backward pass
  const bool tree = !p->node_rule.empty();
  std::vector<CanonRule> g;
  for (const auto& r : tree ? p->table : p->rules)
    g.push_back(which == FMM_GRAD_A ? rule_for_grad_a(r) : rule_for_grad_b(r));
  Plan* q = nullptr;
  fmm_status s = make_plan(g, p->leaf_format, &q, tree ? &p->node_rule : nullptr, p->levels);
  if (s != FMM_OK) return s;
  q->schedule = p->schedule;
  *out = reinterpret_cast<fmm_plan_t>(q);
  return FMM_OK;
}

fmm_status fmm_multiply_backward(fmm_plan_t plan, const float* dC, int64_t lddc, const void* A, int64_t lda,
                                 const void* B, int64_t ldb, float* dA, int64_t ldda, float* dB, int64_t lddb,
                                 int64_t M, int64_t K, int64_t N, int in_dtype, void* ws, size_t ws_bytes,
                                 void* stream) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !valid_dtype(in_dtype) || M < 0 || K < 0 || N < 0) return FMM_ERR_ARG;
  if (M > 0 && N > 0 && (!dC || lddc < N)) return FMM_ERR_ARG;
  if (in_dtype == FMM_DT_F16 && p->leaf_format == FMM_LEAF_BF16X3) return FMM_ERR_DTYPE;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!p->grad_a) {
      // a tree keeps its shape: node r of the gradient tree computes the
      // same product index as node r of the plan (the symmetry permutes
      // the operands of each product, not the products)
      const bool tree = !p->node_rule.empty();
      std::vector<CanonRule> ga, gb;
      for (const auto& r : tree ? p->table : p->rules) {
        ga.push_back(rule_for_grad_a(r));
        gb.push_back(rule_for_grad_b(r));
      }
      fmm_status s = make_plan(ga, p->leaf_format, &p->grad_a, tree ? &p->node_rule : nullptr, p->levels);
      if (s != FMM_OK) return s;
      s = make_plan(gb, p->leaf_format, &p->grad_b, tree ? &p->node_rule : nullptr, p->levels);
      if (s != FMM_OK) return s;
      p->grad_a->schedule = p->grad_b->schedule = p->schedule;
    }
  }
  cudaStream_t st = as_stream(stream);
  if (dA) {
    // dA (M x K) = dC (M x N) B^T (N x K), an <m0, n0, k0> product.  dC:
    // t = M, k = N, k-contiguous.  B^T: t = K (rows of B), k = N (columns of
    // B): k-contiguous in B's memory.
    if (M > 0 && K > 0 && (ldda < K || (N > 0 && (!B || ldb < N)))) return FMM_ERR_SHAPE;
    const Plan* g = p->grad_a;
    const Source x{dC, lddc, kF32, true, M, N, g->pm, g->pk, nullptr, 0, nullptr, 0};
    const Source y{B, ldb, in_dtype, true, K, N, g->pn, g->pk, nullptr, 0, nullptr, 0};
    fmm_status s = run_plan(g, x, y, dA, ldda, M, N, K, nullptr, nullptr, ws, ws_bytes, st);
    if (s != FMM_OK) return s;
  }
  if (dB) {
    // dB (K x N) = A^T (K x M) dC (M x N), a <k0, m0, n0> product.  A^T:
    // t = K (columns of A), k = M (rows of A): t-contiguous.  dC: t = N,
    // k = M: t-contiguous.
    if (K > 0 && N > 0 && (lddb < N || (M > 0 && (!A || lda < K)))) return FMM_ERR_SHAPE;
    const Plan* g = p->grad_b;
    const Source x{A, lda, in_dtype, false, K, M, g->pm, g->pk, nullptr, 0, nullptr, 0};
    const Source y{dC, lddc, kF32, false, N, M, g->pn, g->pk, nullptr, 0, nullptr, 0};
    fmm_status s = run_plan(g, x, y, dB, lddb, K, M, N, nullptr, nullptr, ws, ws_bytes, st);
    if (s != FMM_OK) return s;
  }
  return FMM_OK;
}

fmm_status fmm_sync_status(void* stream) {
  if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return FMM_ERR_CUDA;
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_status, sizeof(int)) != cudaSuccess) return FMM_ERR_CUDA;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_status, &zero, sizeof(int)) != cudaSuccess) return FMM_ERR_CUDA;
  if (v & kStatusTimeout) return FMM_ERR_DEVICE_TIMEOUT;
  if (v & kStatusNonfinite) return FMM_ERR_NONFINITE;
  return FMM_OK;
}

const char* fmm_status_string(fmm_status s) {
  switch (s) {
    case FMM_OK: return "ok";
    case FMM_ERR_ARG: return "invalid argument";
    case FMM_ERR_NOT_MATMUL: return "rule violates the Brent equations";
    case FMM_ERR_SHAPE: return "invalid shape or leading dimension";
    case FMM_ERR_ALIGN: return "misaligned pointer";
    case FMM_ERR_DTYPE: return "unsupported dtype / leaf format";
    case FMM_ERR_WORKSPACE: return "workspace missing or too small";
    case FMM_ERR_CUDA: return "CUDA runtime error";
    case FMM_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case FMM_ERR_NONFINITE: return "non-finite input to scaling";
    case FMM_ERR_UNSUPPORTED: return "plan outside the supported range";
  }
  return "unknown status";
}

fmm_status fmm_batch_workspace_size(const fmm_problem* problems, int count, int in_dtype, const char* steps,
                                    size_t* bytes) {
  if (!bytes) return FMM_ERR_ARG;
  fmm_status s = batch_check(problems, count, in_dtype, steps);
  if (s != FMM_OK) return s;
  BatchLayout L;
  batch_layout(problems, count, in_dtype, &L);
  *bytes = L.total;
  return FMM_OK;
}

fmm_status fmm_batch_create(fmm_batch_t* out, const fmm_problem* problems, int count, int in_dtype,
                            const char* steps, void* ws, size_t ws_bytes) {
  if (!out) return FMM_ERR_ARG;
  *out = nullptr;
  fmm_status s = batch_check(problems, count, in_dtype, steps);
  if (s != FMM_OK) return s;
  Batch* b = new Batch();
  b->count = count;
  b->dt = in_dtype;
  b->fmt = reinterpret_cast<const Plan*>(problems[0].plan)->leaf_format;
  b->steps = batch_steps(steps);
  batch_layout(problems, count, in_dtype, &b->L);
  if (!ws || (uintptr_t)ws % 256 != 0 || ws_bytes < b->L.total) {
    delete b;
    return FMM_ERR_WORKSPACE;
  }
  b->ws = static_cast<char*>(ws);
  b->status = status_ptr();
  if (!b->status) {
    delete b;
    return FMM_ERR_CUDA;
  }
  s = batch_build(b, problems);
  if (s != FMM_OK) {
    delete b;
    return s;
  }
  *out = reinterpret_cast<fmm_batch_t>(b);
  return FMM_OK;
}

fmm_status fmm_batch_run(fmm_batch_t batch, void* stream) {
  const Batch* b = reinterpret_cast<const Batch*>(batch);
  if (!b) return FMM_ERR_ARG;
  return batch_run(b, as_stream(stream));
}

fmm_status fmm_batch_partition(const int64_t* M, const int64_t* K, const int64_t* N, int count, int parts,
                               int32_t* part_of) {
  if (count < 0 || parts < 1 || (count > 0 && (!M || !K || !N || !part_of))) return FMM_ERR_ARG;
  std::vector<int> order((size_t)count);
  std::vector<double> flops((size_t)count);
  for (int i = 0; i < count; ++i) {
    if (M[i] < 0 || K[i] < 0 || N[i] < 0) return FMM_ERR_ARG;
    order[(size_t)i] = i;
    flops[(size_t)i] = 2.0 * (double)M[i] * (double)K[i] * (double)N[i];
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return flops[(size_t)a] > flops[(size_t)b]; });
  std::vector<double> load((size_t)parts, 0.0);
  for (int i : order) {
    int best = 0;
    for (int q = 1; q < parts; ++q)
      if (load[(size_t)q] < load[(size_t)best]) best = q;
    part_of[i] = best;
    load[(size_t)best] += flops[(size_t)i];
  }
  return FMM_OK;
}

fmm_status fmm_batch_destroy(fmm_batch_t batch) {
  delete reinterpret_cast<Batch*>(batch);
  return FMM_OK;
}

const char* fmm_version(void) { return "fmm-gb300 0.1 (sm_103a)"; }

const char* fmm_last_error(void) { return t_last_error.c_str(); }

}  // extern "C"
