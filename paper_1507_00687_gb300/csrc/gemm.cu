// Host dispatch of the fused multiply to its per-leaf-format kernels.
#include <cuda_runtime.h>

#include "kernels.h"

namespace fmm {

cudaError_t launch_fused_gemm_bf16(const GemmArgs& a, cudaStream_t st);
cudaError_t launch_fused_gemm_f16(const GemmArgs& a, cudaStream_t st);
cudaError_t launch_fused_gemm_bf16x3(const GemmArgs& a, cudaStream_t st);

int device_sm_count() {
  static int n[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (n[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n[dev] = v > 0 ? v : 1;
  }
  return n[dev];
}

cudaError_t launch_fused_gemm(const GemmArgs& a, int leaf_format, cudaStream_t st) {
  switch (leaf_format) {
    case FMM_LEAF_BF16: return launch_fused_gemm_bf16(a, st);
    case FMM_LEAF_F16: return launch_fused_gemm_f16(a, st);
    default: return launch_fused_gemm_bf16x3(a, st);
  }
}

}  // namespace fmm
