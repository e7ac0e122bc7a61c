// Fused FP32 kernel for the stencil G5,G12,G14,G17,G21,G26.
#include "rlbm_fused.cuh"
#include "rlbm_fused_launch.h"

namespace rlbm {
template <>
cudaError_t launch_fused<StencilM1>(const FusedParams& p, const void* fin, void* fout, cudaStream_t s) {
  const long long nsite = (long long)p.Nx * p.Ny;
  fused_f32_kernel<StencilM1><<<(unsigned)((nsite + 127) / 128), 128, 0, s>>>(
      p, static_cast<const float*>(fin), static_cast<float*>(fout));
  return cudaGetLastError();
}
}  // namespace rlbm
