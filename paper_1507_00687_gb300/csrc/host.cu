// Host-memory pipeline (fmm_host_*): products whose operands and results
// live in host memory, with the copies of one product overlapping the
// computation of its neighbours.  Built only on the library's public
// entry points (fmm_scale, fmm_multiply) and CUDA streams and events.
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fmm.h"

namespace {

struct Slot {
  void* A = nullptr;
  void* B = nullptr;
  float* C = nullptr;
  int32_t* e = nullptr;       // eA (M), d (K), eB (N)
  cudaEvent_t in_done = nullptr;    // A copied in
  cudaEvent_t in_done_b = nullptr;  // B copied in
  cudaEvent_t used = nullptr;       // the multiply has read A, B and written C
  cudaEvent_t out_done = nullptr;   // C copied out
  bool busy = false;
};

struct Host {
  fmm_plan_t plan;
  int64_t M, K, N;
  int dtype, es;
  std::string steps;
  std::vector<Slot> slots;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t in = nullptr, in_b = nullptr, comp = nullptr, out = nullptr;  // A and B copy in on two streams
  int next = 0;
  fmm_status err = FMM_OK;
};

int elem_size(int dt) { return dt == FMM_DT_F32 ? 4 : 2; }

void release(Host* h) {
  for (Slot& s : h->slots) {
    cudaFree(s.A);
    cudaFree(s.B);
    cudaFree(s.C);
    cudaFree(s.e);
    if (s.in_done) cudaEventDestroy(s.in_done);
    if (s.in_done_b) cudaEventDestroy(s.in_done_b);
    if (s.used) cudaEventDestroy(s.used);
    if (s.out_done) cudaEventDestroy(s.out_done);
  }
  cudaFree(h->ws);
  if (h->in) cudaStreamDestroy(h->in);
  if (h->in_b) cudaStreamDestroy(h->in_b);
  if (h->comp) cudaStreamDestroy(h->comp);
  if (h->out) cudaStreamDestroy(h->out);
  delete h;
}

}  // namespace

extern "C" {

fmm_status fmm_host_create(fmm_host_t* out, fmm_plan_t plan, int64_t M, int64_t K, int64_t N, int dtype,
                           const char* steps, int depth) {
  if (!out || !plan || M < 1 || K < 1 || N < 1 || depth < 1 || depth > 4 || !steps) return FMM_ERR_ARG;
  if (dtype != FMM_DT_F32 && dtype != FMM_DT_BF16 && dtype != FMM_DT_F16) return FMM_ERR_ARG;
  for (const char* c = steps; *c; ++c)
    if (*c != 'O' && *c != 'I') return FMM_ERR_ARG;
  *out = nullptr;
  Host* h = new Host();
  h->plan = plan;
  h->M = M;
  h->K = K;
  h->N = N;
  h->dtype = dtype;
  h->es = elem_size(dtype);
  h->steps = steps;
  h->slots.resize((size_t)depth);
  bool ok = cudaStreamCreateWithFlags(&h->in, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&h->in_b, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&h->comp, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&h->out, cudaStreamNonBlocking) == cudaSuccess;
  for (Slot& s : h->slots) {
    ok = ok && cudaMalloc(&s.A, (size_t)(M * K * h->es)) == cudaSuccess &&
         cudaMalloc(&s.B, (size_t)(K * N * h->es)) == cudaSuccess &&
         cudaMalloc(reinterpret_cast<void**>(&s.C), (size_t)(M * N * 4)) == cudaSuccess &&
         cudaMalloc(reinterpret_cast<void**>(&s.e), (size_t)((M + K + N) * 4)) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.in_done_b, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.used, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s.out_done, cudaEventDisableTiming) == cudaSuccess;
  }
  size_t ws = 0;
  ok = ok && fmm_workspace_size(plan, M, K, N, &ws) == FMM_OK;
  h->ws_bytes = ws;
  ok = ok && (ws == 0 || cudaMalloc(&h->ws, ws) == cudaSuccess);
  if (!ok) {
    release(h);
    return FMM_ERR_CUDA;
  }
  *out = reinterpret_cast<fmm_host_t>(h);
  return FMM_OK;
}

fmm_status fmm_host_submit(fmm_host_t handle, const void* hA, int64_t lda, const void* hB, int64_t ldb, float* hC,
                           int64_t ldc) {
  Host* h = reinterpret_cast<Host*>(handle);
  if (!h || !hA || !hB || !hC || lda < h->K || ldb < h->N || ldc < h->N) return FMM_ERR_ARG;
  Slot& s = h->slots[(size_t)h->next];
  h->next = (h->next + 1) % (int)h->slots.size();
  const size_t es = (size_t)h->es;
  // copy in (A and B on their own streams, so two copy engines share the
  // link) once the slot's previous multiply has read A and B
  if (s.busy && (cudaStreamWaitEvent(h->in, s.used, 0) != cudaSuccess ||
                 cudaStreamWaitEvent(h->in_b, s.used, 0) != cudaSuccess))
    return FMM_ERR_CUDA;
  if (cudaMemcpy2DAsync(s.A, (size_t)h->K * es, hA, (size_t)lda * es, (size_t)h->K * es, (size_t)h->M,
                        cudaMemcpyHostToDevice, h->in) != cudaSuccess ||
      cudaEventRecord(s.in_done, h->in) != cudaSuccess ||
      cudaMemcpy2DAsync(s.B, (size_t)h->N * es, hB, (size_t)ldb * es, (size_t)h->N * es, (size_t)h->K,
                        cudaMemcpyHostToDevice, h->in_b) != cudaSuccess ||
      cudaEventRecord(s.in_done_b, h->in_b) != cudaSuccess)
    return FMM_ERR_CUDA;
  // compute once A, B are in and the slot's previous C has been copied out
  if (cudaStreamWaitEvent(h->comp, s.in_done, 0) != cudaSuccess ||
      cudaStreamWaitEvent(h->comp, s.in_done_b, 0) != cudaSuccess)
    return FMM_ERR_CUDA;
  if (s.busy && cudaStreamWaitEvent(h->comp, s.out_done, 0) != cudaSuccess) return FMM_ERR_CUDA;
  int32_t* eA = s.e;
  int32_t* d = eA + h->M;
  int32_t* eB = d + h->K;
  const bool scaled = !h->steps.empty();
  fmm_status st = FMM_OK;
  if (scaled) st = fmm_scale(h->steps.c_str(), s.A, s.B, h->dtype, h->M, h->K, h->N, h->K, h->N, eA, d, eB, h->comp);
  if (st == FMM_OK)
    st = fmm_multiply(h->plan, s.A, h->K, s.B, h->N, s.C, h->N, h->M, h->K, h->N, h->dtype, scaled ? eA : nullptr,
                      scaled ? d : nullptr, scaled ? eB : nullptr, h->ws, h->ws_bytes, h->comp);
  if (st != FMM_OK) {
    if (h->err == FMM_OK) h->err = st;
    return st;
  }
  if (cudaEventRecord(s.used, h->comp) != cudaSuccess) return FMM_ERR_CUDA;
  // copy out
  if (cudaStreamWaitEvent(h->out, s.used, 0) != cudaSuccess ||
      cudaMemcpy2DAsync(hC, (size_t)ldc * 4, s.C, (size_t)h->N * 4, (size_t)h->N * 4, (size_t)h->M,
                        cudaMemcpyDeviceToHost, h->out) != cudaSuccess ||
      cudaEventRecord(s.out_done, h->out) != cudaSuccess)
    return FMM_ERR_CUDA;
  s.busy = true;
  return FMM_OK;
}

fmm_status fmm_host_wait(fmm_host_t handle) {
  Host* h = reinterpret_cast<Host*>(handle);
  if (!h) return FMM_ERR_ARG;
  if (cudaStreamSynchronize(h->in) != cudaSuccess || cudaStreamSynchronize(h->in_b) != cudaSuccess ||
      cudaStreamSynchronize(h->out) != cudaSuccess)
    return FMM_ERR_CUDA;
  fmm_status st = fmm_sync_status(h->comp);
  if (h->err != FMM_OK) {
    st = h->err;
    h->err = FMM_OK;
  }
  return st;
}

fmm_status fmm_host_destroy(fmm_host_t handle) {
  Host* h = reinterpret_cast<Host*>(handle);
  if (!h) return FMM_OK;
  cudaStreamSynchronize(h->in);
  cudaStreamSynchronize(h->in_b);
  cudaStreamSynchronize(h->comp);
  cudaStreamSynchronize(h->out);
  release(h);
  return FMM_OK;
}

}  // extern "C"
