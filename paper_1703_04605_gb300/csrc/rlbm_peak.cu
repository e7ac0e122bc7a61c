// FP64 fused multiply-add throughput of the device, measured with CUDA
// events: the denominator of the FP64 step kernels' ALU roofline.  Each
// thread runs eight independent dependent chains a = a b + c (so the pipe,
// not the FMA latency, bounds the rate); the grid fills every SM several
// times over.  b and c are loaded from global memory so that every FMA takes
// register operands: with b and c as kernel parameters (constant-bank
// operands) the same chains measured 16 % slower on GB300, below the rate
// that the step kernels themselves reach.  Not part of the method: a
// measurement helper.
#include <cuda_runtime.h>

#include "rlbm_internal.h"

namespace rlbm {
namespace {

constexpr int kChains = 8;
__device__ double g_sink[256];
__device__ double g_bc[2] = {0.9999999, 1e-7};   // b, c

__global__ void __launch_bounds__(256) fp64_fma_chains(int iters) {
  const double b = g_bc[0], c = g_bc[1];
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  // the chains stay in [1, 1.3] (fixed point c / (1 - b) = 1), so this store
  // never happens; it keeps the compiler from dropping the chains
  if (s == 12345.678) g_sink[threadIdx.x] = s;
}

}  // namespace
}  // namespace rlbm

using namespace rlbm;

extern "C" rlbm_status rlbm_fp64_fma_rate(void* cuda_stream, double* tflops) {
  if (!tflops) return RLBM_EINVAL;
  *tflops = 0.0;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return RLBM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 0.0f;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, s);
    fp64_fma_chains<<<blocks, threads, 0, s>>>(iters);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;   // first launch: warm-up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || best <= 0.0f) return RLBM_ECUDA;
  const double flops = 2.0 * kChains * (double)iters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return RLBM_OK;
}
