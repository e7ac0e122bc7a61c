// Fused FP32 kernel for the stencil G1..G6.
#include "rlbm_fused.cuh"
#include "rlbm_fused_launch.h"

namespace rlbm {
template <>
cudaError_t launch_fused<StencilG16>(const FusedParams& p, const void* fin, void* fout, bool bf16, cudaStream_t s) {
  const long long nsite = (long long)p.Nx * p.Ny;
  const unsigned grid = (unsigned)((nsite + 127) / 128);
  if (bf16) fused_f32_kernel<StencilG16, true><<<grid, 128, 0, s>>>(p, fin, fout);
  else fused_f32_kernel<StencilG16, false><<<grid, 128, 0, s>>>(p, fin, fout);
  return cudaGetLastError();
}
template <>
cudaError_t launch_bf16_io<StencilG16>(int what, const FusedParams& fp, const StepParams<double>& p, FieldPtrs fd,
                               void* cur, void* prev, void* ccur, void* cprev, MomentOut mo, cudaStream_t s) {
  return launch_bf16_io_impl<StencilG16>(what, fp, p, fd, cur, prev, ccur, cprev, mo, s);
}
template <>
const void* fused_kernel_fn<StencilG16>(bool bf16) {
  return fused_kernel_fn_impl<StencilG16>(bf16);
}
}  // namespace rlbm
