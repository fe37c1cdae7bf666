// Fused multiply kernels with BF16 leaf products.
#include "gemm.cuh"

namespace fmm {
cudaError_t launch_fused_gemm_bf16(const GemmArgs& a, cudaStream_t st) {
  return gemm::launch_mode<gemm::kModeBF16>(a, st);
}
}  // namespace fmm
