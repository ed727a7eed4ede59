// we_warp.cu -- one warp per walker SSA kernel for large networks (placeholder until built).
#include "we_internal.cuh"

namespace we {
size_t propagate_warp_smem(const NetView &N, int block) { (void)N; (void)block; return 0; }
cudaError_t launch_propagate_warp(const PropagateParams &prm, int block, cudaStream_t st) {
  (void)prm; (void)block; (void)st;
  return cudaErrorNotSupported;
}
}  // namespace we
