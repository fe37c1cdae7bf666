// Fused multiply kernels with F16 leaf products.
#include "gemm.cuh"

namespace fmm {
cudaError_t launch_fused_gemm_f16(const GemmArgs& a, cudaStream_t st) {
  return gemm::launch_mode<gemm::kModeF16>(a, st);
}
}  // namespace fmm
