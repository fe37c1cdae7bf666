// Fused multiply kernels with BF16x3 leaf products.
#include "gemm.cuh"

namespace fmm {
cudaError_t launch_fused_gemm_bf16x3(const GemmArgs& a, cudaStream_t st) {
  return gemm::launch_mode<gemm::kModeBF16x3>(a, st);
}
}  // namespace fmm
