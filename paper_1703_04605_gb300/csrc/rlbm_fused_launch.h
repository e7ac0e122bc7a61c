// Launchers of the stencil-specialised FP32 kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "rlbm_internal.h"
#include "rlbm_stencils.h"

namespace rlbm {
template <class Def>
cudaError_t launch_fused(const FusedParams& p, const void* fin, void* fout, bool bf16, cudaStream_t s);
template <>
cudaError_t launch_fused<StencilM1>(const FusedParams&, const void*, void*, bool, cudaStream_t);
template <>
cudaError_t launch_fused<StencilG16>(const FusedParams&, const void*, void*, bool, cudaStream_t);
template <>
cudaError_t launch_fused<StencilE5>(const FusedParams&, const void*, void*, bool, cudaStream_t);
template <>
cudaError_t launch_fused<StencilS2>(const FusedParams&, const void*, void*, bool, cudaStream_t);

// Batched FP32 step over up to kBatchMax lattices of one stencil (minb: 4 or 5
// resident blocks per SM, i.e. 128 or 96 registers).
struct BatchParams;
template <class Def>
cudaError_t launch_batch(const BatchParams& bp, int minb, cudaStream_t s);
template <>
cudaError_t launch_batch<StencilM1>(const BatchParams&, int, cudaStream_t);
template <>
cudaError_t launch_batch<StencilG16>(const BatchParams&, int, cudaStream_t);
template <>
cudaError_t launch_batch<StencilE5>(const BatchParams&, int, cudaStream_t);
template <>
cudaError_t launch_batch<StencilS2>(const BatchParams&, int, cudaStream_t);
// BF16 deviation storage: what = 0 init (fields -> coefficients, S_0, S_{-1}),
// what = 1 read-out of the pull of prev.
template <class Def>
cudaError_t launch_bf16_io(int what, const FusedParams& fp, const StepParams<double>& p, FieldPtrs fd,
                           void* cur, void* prev, void* ccur, void* cprev, MomentOut mo, cudaStream_t s);
#define RLBM_DECL_BF16_IO(S)                                                                              \
  template <>                                                                                            \
  cudaError_t launch_bf16_io<S>(int, const FusedParams&, const StepParams<double>&, FieldPtrs, void*, void*, \
                                void*, void*, MomentOut, cudaStream_t);
RLBM_DECL_BF16_IO(StencilM1)
RLBM_DECL_BF16_IO(StencilG16)
RLBM_DECL_BF16_IO(StencilE5)
RLBM_DECL_BF16_IO(StencilS2)
#undef RLBM_DECL_BF16_IO
}  // namespace rlbm
