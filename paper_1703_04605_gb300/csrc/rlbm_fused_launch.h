// Launchers of the stencil-specialised FP32 kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "rlbm_internal.h"
#include "rlbm_stencils.h"

namespace rlbm {
// mode: 0 FP32 storage, 1 BF16 deviation storage, 2 FP32 storage with
// extended moment sums (rlbm_fused.cuh).
template <class Def>
cudaError_t launch_fused(const FusedParams& p, const void* fin, void* fout, int mode, cudaStream_t s);
template <>
cudaError_t launch_fused<StencilM1>(const FusedParams&, const void*, void*, int, cudaStream_t);
template <>
cudaError_t launch_fused<StencilG16>(const FusedParams&, const void*, void*, int, cudaStream_t);
template <>
cudaError_t launch_fused<StencilE5>(const FusedParams&, const void*, void*, int, cudaStream_t);
template <>
cudaError_t launch_fused<StencilS2>(const FusedParams&, const void*, void*, int, cudaStream_t);

// The step kernel itself (FusedParams, const void* fin, void* fout), for graph
// kernel nodes; grid (Nx Ny + 127)/128, block 128, no dynamic shared memory.
template <class Def>
const void* fused_kernel_fn(int mode);
template <>
const void* fused_kernel_fn<StencilM1>(int);
template <>
const void* fused_kernel_fn<StencilG16>(int);
template <>
const void* fused_kernel_fn<StencilE5>(int);
template <>
const void* fused_kernel_fn<StencilS2>(int);
// The persistent batched kernel of a stencil (rlbm_persist.cuh) for a storage
// variant (mode as above), taking one PersistParams; block 128, cooperative.
template <class Def>
const void* persist_kernel_fn(int mode);
template <>
const void* persist_kernel_fn<StencilM1>(int);
template <>
const void* persist_kernel_fn<StencilG16>(int);
template <>
const void* persist_kernel_fn<StencilE5>(int);
template <>
const void* persist_kernel_fn<StencilS2>(int);
// The compiled third-order kernel of kind 5..10 (FusedO3Params, const float*
// fin, float* fout), for graph kernel nodes; grid (Nx Ny + 127)/128, block
// 128, no dynamic shared memory (rlbm_fused_o3.cu).
const void* fused_o3_kernel_fn(int kind);
// Init and read-out on a compiled stencil.  BF16 deviation storage: what = 0
// init (fields -> coefficients, S_0, S_{-1}), what = 1 read-out of the pull of
// prev; FP32 storage: what = 2 init of S_0 into cur only, what = 3 read-out
// of the pull of prev, what = 4 read-out of S_0 in prev (pass cur) right after
// what = 2, before any step (ccur, cprev unused).
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
