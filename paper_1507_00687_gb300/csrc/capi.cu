// C ABI (include/fmm.h): argument validation, plan lifetime, and the
// launch sequences of the scaling steps, the forward and the backward
// multiply.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fmm.h"
#include "device.cuh"
#include "kernels.h"
#include "plan.h"

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

static uint64_t timeout_ns() {
  static uint64_t v = [] {
    const char* s = std::getenv("FMM_WAIT_TIMEOUT_NS");
    uint64_t t = s ? std::strtoull(s, nullptr, 10) : 0;
    return t ? t : (uint64_t)2000000000ull;  // 2 s per wait
  }();
  return v;
}

static int esize(int dt) { return dt == kF32 ? 4 : 2; }

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
  if (cudaMalloc(&d, bytes) != cudaSuccess) return FMM_ERR_CUDA;
  if (cudaMemcpy(d, p->host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return FMM_ERR_CUDA;
  }
  p->dev = d;
  p->device = dev;
  return FMM_OK;
}

static fmm_status make_plan(const std::vector<CanonRule>& rules, int leaf, Plan** out) {
  Plan* p = nullptr;
  fmm_status s = build_plan(rules, leaf, &p);
  if (s != FMM_OK) return s;
  if (p->max_terms > kMaxTerms) {
    destroy_plan(p);
    return FMM_ERR_UNSUPPORTED;
  }
  *out = p;
  return FMM_OK;
}

// Run the flattened plan p on operands described by (a, b) into C.
// Block extents follow from the plan's granules: leaf block = ceil(dim / granule).
static fmm_status run_plan(const Plan* p, TileOperand a, TileOperand b, float* C, int64_t ldc, int64_t M,
                           int64_t K, int64_t N, const int* eA, const int* eB, cudaStream_t st) {
  if (M == 0 || N == 0) return FMM_OK;
  if (K == 0) {
    return cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)N * 4, (size_t)M, st) == cudaSuccess ? FMM_OK
                                                                                                   : FMM_ERR_CUDA;
  }
  int* status = status_ptr();
  if (!status) return FMM_ERR_CUDA;
  if (ensure_uploaded(p) != FMM_OK) return FMM_ERR_CUDA;
  const int64_t bm = (M + p->pm - 1) / p->pm, bk = (K + p->pk - 1) / p->pk, bn = (N + p->pn - 1) / p->pn;
  a.T = M; a.K = K; a.bt = bm; a.bk = bk;
  b.T = N; b.K = K; b.bt = bn; b.bk = bk;
  // Vector loads of 8 consecutive elements (32 bytes for fp32, 16 for 16-bit
  // types) need every chunk start -- block offset + multiple of 8 elements
  // along the contiguous index, any row -- to be aligned to that size.
  auto vec = [&](const TileOperand& o) {
    const int64_t blk = o.kcontig ? o.bk : o.bt;
    const uintptr_t align = o.dtype == kF32 ? 32 : 16;
    return ((uintptr_t)o.ptr % align == 0) && (o.ld % 8 == 0) && (blk % 8 == 0) ? 1 : 0;
  };
  a.vec_ok = vec(a);
  b.vec_ok = vec(b);
  GemmArgs g{};
  g.a = a;
  g.b = b;
  g.c.C = C;
  g.c.ldc = ldc;
  g.c.M = M;
  g.c.N = N;
  g.c.bm = bm;
  g.c.bn = bn;
  g.c.eA = eA;
  g.c.eB = eB;
  g.c.vec_ok = ((uintptr_t)C % 16 == 0) && (ldc % 4 == 0) && (bn % 4 == 0) ? 1 : 0;
  g.leaves = p->dev;
  g.num_leaves = p->leaves;
  g.kl = bk;
  g.pm = p->pm;
  g.pk = p->pk;
  g.pn = p->pn;
  g.status = status;
  g.timeout_ns = timeout_ns();
  return cuda_ok(launch_fused_gemm(g, p->leaf_format, st), "fused multiply launch") ? FMM_OK : FMM_ERR_CUDA;
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

fmm_status fmm_plan_destroy(fmm_plan_t plan) {
  destroy_plan(reinterpret_cast<Plan*>(plan));
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

fmm_status fmm_scale(const char* steps, const void* A, const void* B, int dtype, int64_t M, int64_t K, int64_t N,
                     int64_t lda, int64_t ldb, int32_t* eA, int32_t* d, int32_t* eB, void* stream) {
  if (!steps) return FMM_ERR_ARG;
  for (const char* c = steps; *c; ++c)
    if (*c != 'O' && *c != 'I') return FMM_ERR_ARG;
  if ((M > 0 && !eA) || (K > 0 && !d) || (N > 0 && !eB)) return FMM_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  if (launch_fill(eA, M, 0, st) != cudaSuccess || launch_fill(d, K, 0, st) != cudaSuccess ||
      launch_fill(eB, N, 0, st) != cudaSuccess)
    return FMM_ERR_CUDA;
  for (const char* c = steps; *c; ++c) {
    fmm_status s = *c == 'O' ? fmm_scale_outside(A, B, dtype, M, K, N, lda, ldb, d, eA, eB, stream)
                             : fmm_scale_inside(A, B, dtype, M, K, N, lda, ldb, eA, eB, d, stream);
    if (s != FMM_OK) return s;
  }
  return FMM_OK;
}

// Workspace of a scaled multiply: the scaled copies A' (M x ldA') and
// B' (K x ldB') in fp32 (bf16 for bf16 inputs), leading dimensions rounded
// up to 8 elements, each 256-byte aligned.
static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
static size_t scaled_ws_bytes(int64_t M, int64_t K, int64_t N, int es) {
  return (size_t)round_up(M * round_up(K, 8) * es, 256) + (size_t)round_up(K * round_up(N, 8) * es, 256);
}

fmm_status fmm_workspace_size(fmm_plan_t plan, int64_t M, int64_t K, int64_t N, size_t* bytes) {
  if (!plan || !bytes || M < 0 || K < 0 || N < 0) return FMM_ERR_ARG;
  *bytes = scaled_ws_bytes(M, K, N, 4);
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
  if ((M + p->pm - 1) / p->pm >= (1ll << 31) || (N + p->pn - 1) / p->pn >= (1ll << 31)) return FMM_ERR_SHAPE;
  cudaStream_t st = as_stream(stream);
  const void* Aop = A;
  const void* Bop = B;
  int64_t ldA = lda, ldB = ldb;
  int dt = in_dtype;
  if ((eA || d || eB || in_dtype == FMM_DT_F16) && M > 0 && N > 0 && K > 0) {
    // Algs. 1-3: multiply A' = 2^-eA A 2^d and B' = 2^-d B 2^-eB (exact
    // copies written by one HBM-bound pass each), unscale in the epilogue.
    // fp16 inputs always take this path (as an exact widening to fp32).
    const int wdt = in_dtype == FMM_DT_BF16 ? kBF16 : kF32;
    const int es = wdt == kF32 ? 4 : 2;
    if (!ws || ws_bytes < scaled_ws_bytes(M, K, N, es) || (uintptr_t)ws % 256 != 0) return FMM_ERR_WORKSPACE;
    ldA = round_up(K, 8);
    ldB = round_up(N, 8);
    void* Ap = ws;
    void* Bp = static_cast<char*>(ws) + round_up(M * ldA * es, 256);
    if (!cuda_ok(launch_apply_exp(A, in_dtype, M, K, lda, eA, -1, d, +1, Ap, ldA, st), "apply scaling to A"))
      return FMM_ERR_CUDA;
    if (!cuda_ok(launch_apply_exp(B, in_dtype, K, N, ldb, d, -1, eB, -1, Bp, ldB, st), "apply scaling to B"))
      return FMM_ERR_CUDA;
    Aop = Ap;
    Bop = Bp;
    dt = wdt;
  }
  TileOperand a{};
  a.ptr = Aop; a.ld = ldA; a.dtype = dt; a.kcontig = 1;
  a.blk_t_shift = 16; a.blk_k_shift = 0;
  TileOperand b{};
  b.ptr = Bop; b.ld = ldB; b.dtype = dt; b.kcontig = 0;
  b.blk_t_shift = 0; b.blk_k_shift = 16;
  return run_plan(p, a, b, C, ldc, M, K, N, eA, eB, st);
}

fmm_status fmm_multiply_backward(fmm_plan_t plan, const float* dC, int64_t lddc, const void* A, int64_t lda,
                                 const void* B, int64_t ldb, float* dA, int64_t ldda, float* dB, int64_t lddb,
                                 int64_t M, int64_t K, int64_t N, int in_dtype, void* stream) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !valid_dtype(in_dtype) || M < 0 || K < 0 || N < 0) return FMM_ERR_ARG;
  if (M > 0 && N > 0 && (!dC || lddc < N)) return FMM_ERR_ARG;
  if (in_dtype == FMM_DT_F16) return FMM_ERR_DTYPE;
  if (in_dtype == FMM_DT_F16 && p->leaf_format == FMM_LEAF_BF16X3) return FMM_ERR_DTYPE;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!p->grad_a) {
      std::vector<CanonRule> ga, gb;
      for (const auto& r : p->rules) {
        ga.push_back(rule_for_grad_a(r));
        gb.push_back(rule_for_grad_b(r));
      }
      fmm_status s = make_plan(ga, p->leaf_format, &p->grad_a);
      if (s != FMM_OK) return s;
      s = make_plan(gb, p->leaf_format, &p->grad_b);
      if (s != FMM_OK) return s;
    }
  }
  cudaStream_t st = as_stream(stream);
  if (dA) {
    // dA (M x K) = dC (M x N) B^T (N x K): operand 1 is dC (k = n contiguous),
    // operand 2 is B^T, whose element (t = k, k' = n) is B[k][n] (contiguous in n).
    if (M > 0 && K > 0 && (ldda < K || (N > 0 && (!B || ldb < N)))) return FMM_ERR_SHAPE;
    TileOperand a{};
    a.ptr = dC; a.ld = lddc; a.dtype = kF32; a.kcontig = 1; a.blk_t_shift = 16; a.blk_k_shift = 0;
    TileOperand b{};
    b.ptr = B; b.ld = ldb; b.dtype = in_dtype; b.kcontig = 1; b.blk_t_shift = 0; b.blk_k_shift = 16;
    fmm_status s = run_plan(p->grad_a, a, b, dA, ldda, M, N, K, nullptr, nullptr, st);
    if (s != FMM_OK) return s;
  }
  if (dB) {
    // dB (K x N) = A^T (K x M) dC (M x N): A^T's element (t = k, k' = m) is
    // A[m][k] (contiguous in t); dC's element (t = n, k' = m) is dC[m][n].
    if (K > 0 && N > 0 && (lddb < N || (M > 0 && (!A || lda < K)))) return FMM_ERR_SHAPE;
    TileOperand a{};
    a.ptr = A; a.ld = lda; a.dtype = in_dtype; a.kcontig = 0; a.blk_t_shift = 16; a.blk_k_shift = 0;
    TileOperand b{};
    b.ptr = dC; b.ld = lddc; b.dtype = kF32; b.kcontig = 0; b.blk_t_shift = 0; b.blk_k_shift = 16;
    fmm_status s = run_plan(p->grad_b, a, b, dB, lddb, K, M, N, nullptr, nullptr, st);
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

const char* fmm_version(void) { return "fmm-gb300 0.1 (sm_103a)"; }

const char* fmm_last_error(void) { return t_last_error.c_str(); }

}  // extern "C"
