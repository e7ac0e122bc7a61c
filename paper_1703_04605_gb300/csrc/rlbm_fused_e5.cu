// Fused FP32 kernel for the stencil G1,G14,G49,G51,G60,G70.
#include "rlbm_fused.cuh"
#include "rlbm_fused_launch.h"

namespace rlbm {
template <>
cudaError_t launch_fused<StencilE5>(const FusedParams& p, const void* fin, void* fout, cudaStream_t s) {
  const long long nsite = (long long)p.Nx * p.Ny;
  fused_f32_kernel<StencilE5><<<(unsigned)((nsite + 127) / 128), 128, 0, s>>>(
      p, static_cast<const float*>(fin), static_cast<float*>(fout));
  return cudaGetLastError();
}
}  // namespace rlbm
