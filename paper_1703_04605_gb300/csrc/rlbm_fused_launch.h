// Launchers of the stencil-specialised FP32 kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "rlbm_stencils.h"

namespace rlbm {
struct FusedParams;
template <class Def>
cudaError_t launch_fused(const FusedParams& p, const void* fin, void* fout, cudaStream_t s);
template <>
cudaError_t launch_fused<StencilM1>(const FusedParams&, const void*, void*, cudaStream_t);
template <>
cudaError_t launch_fused<StencilG16>(const FusedParams&, const void*, void*, cudaStream_t);
template <>
cudaError_t launch_fused<StencilE5>(const FusedParams&, const void*, void*, cudaStream_t);
}  // namespace rlbm
