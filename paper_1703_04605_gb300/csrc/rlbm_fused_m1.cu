// Fused FP32 kernel for the stencil G5,G12,G14,G17,G21,G26.
#include "rlbm_fused.cuh"
#include "rlbm_persist.cuh"
#include "rlbm_fused_launch.h"

namespace rlbm {
template <>
cudaError_t launch_fused<StencilM1>(const FusedParams& p, const void* fin, void* fout, int mode, cudaStream_t s) {
  return launch_fused_impl<StencilM1>(p, fin, fout, mode, s);
}
template <>
cudaError_t launch_bf16_io<StencilM1>(int what, const FusedParams& fp, const StepParams<double>& p, FieldPtrs fd,
                               void* cur, void* prev, void* ccur, void* cprev, MomentOut mo, cudaStream_t s) {
  return launch_bf16_io_impl<StencilM1>(what, fp, p, fd, cur, prev, ccur, cprev, mo, s);
}
template <>
const void* fused_kernel_fn<StencilM1>(int mode) {
  return fused_kernel_fn_impl<StencilM1>(mode);
}
template <>
const void* persist_kernel_fn<StencilM1>(int mode) {
  return persist_kernel_fn_impl<StencilM1>(mode);
}
}  // namespace rlbm
