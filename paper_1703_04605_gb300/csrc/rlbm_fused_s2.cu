// Fused FP32 kernel for the stencil G3,G9,G10,G14,G17,G21.
#include "rlbm_fused.cuh"
#include "rlbm_persist.cuh"
#include "rlbm_fused_launch.h"

namespace rlbm {
template <>
cudaError_t launch_fused<StencilS2>(const FusedParams& p, const void* fin, void* fout, int mode, cudaStream_t s) {
  return launch_fused_impl<StencilS2>(p, fin, fout, mode, s);
}
template <>
cudaError_t launch_bf16_io<StencilS2>(int what, const FusedParams& fp, const StepParams<double>& p, FieldPtrs fd,
                               void* cur, void* prev, void* ccur, void* cprev, MomentOut mo, cudaStream_t s) {
  return launch_bf16_io_impl<StencilS2>(what, fp, p, fd, cur, prev, ccur, cprev, mo, s);
}
template <>
const void* fused_kernel_fn<StencilS2>(int mode) {
  return fused_kernel_fn_impl<StencilS2>(mode);
}
template <>
const void* persist_kernel_fn<StencilS2>(int mode) {
  return persist_kernel_fn_impl<StencilS2>(mode);
}
}  // namespace rlbm
