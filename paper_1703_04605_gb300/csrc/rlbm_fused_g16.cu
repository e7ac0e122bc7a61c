// Fused FP32 kernel for the stencil G1..G6.
#include "rlbm_fused.cuh"
#include "rlbm_fused_launch.h"

namespace rlbm {
template <>
cudaError_t launch_fused<StencilG16>(const FusedParams& p, const void* fin, void* fout, cudaStream_t s) {
  const long long nsite = (long long)p.Nx * p.Ny;
  fused_f32_kernel<StencilG16><<<(unsigned)((nsite + 127) / 128), 128, 0, s>>>(
      p, static_cast<const float*>(fin), static_cast<float*>(fout));
  return cudaGetLastError();
}
}  // namespace rlbm
