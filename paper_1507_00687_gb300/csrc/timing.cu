// Per-kernel timing (fmm_kernel_timing / fmm_kernel_timing_read): while
// enabled, every kernel of the selected kinds the library launches is
// bracketed by a pair of CUDA events recorded on its launching stream, so that a caller can attribute
// the device time of one library call to its kernels (combination pass,
// multiply, scaling reductions ...).  Measurement only; off by default.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fmm.h"
#include "kernels.h"

namespace fmm {
namespace {

struct Record {
  const char* kind;
  cudaEvent_t start, stop;
};

std::mutex g_mu;
int g_mask = 0;  // kinds being recorded (bits of kind_bit)
std::vector<Record> g_records;

int kind_bit(const char* kind) {
  if (std::strcmp(kind, "scale") == 0) return 2;
  if (std::strcmp(kind, "prepare") == 0) return 4;
  if (std::strcmp(kind, "combine") == 0) return 8;
  if (std::strcmp(kind, "multiply") == 0) return 16;
  return 0;
}

void release_all() {
  for (auto& r : g_records) {
    cudaEventDestroy(r.start);
    cudaEventDestroy(r.stop);
  }
  g_records.clear();
}

}  // namespace

KernelTimer::KernelTimer(const char* kind, cudaStream_t st) : kind_(kind), st_(st) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!(g_mask & kind_bit(kind))) return;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return;
  }
  cudaEventRecord(a, st);
  start_ = a;
  stop_ = b;
}

KernelTimer::~KernelTimer() {
  if (!start_) return;
  cudaEventRecord(static_cast<cudaEvent_t>(stop_), st_);
  std::lock_guard<std::mutex> lock(g_mu);
  g_records.push_back({kind_, static_cast<cudaEvent_t>(start_), static_cast<cudaEvent_t>(stop_)});
}

}  // namespace fmm

using namespace fmm;

extern "C" {

fmm_status fmm_kernel_timing(int enable) {
  if (enable < 0 || enable > 31) return FMM_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (enable) release_all();
  g_mask = enable == 1 ? 30 : enable;
  return FMM_OK;
}

fmm_status fmm_kernel_timing_read(const char* kind, double* total_ms, int64_t* launches) {
  if (!total_ms || !launches) return FMM_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  double ms = 0;
  int64_t n = 0;
  for (const auto& r : g_records) {
    if (kind && *kind && std::strcmp(kind, r.kind) != 0) continue;
    if (cudaEventSynchronize(r.stop) != cudaSuccess) return FMM_ERR_CUDA;
    float t = 0;
    if (cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess) return FMM_ERR_CUDA;
    ms += t;
    ++n;
  }
  *total_ms = ms;
  *launches = n;
  return FMM_OK;
}

}  // extern "C"
