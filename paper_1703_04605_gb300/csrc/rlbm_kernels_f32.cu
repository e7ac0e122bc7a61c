// FP32-storage step kernel instantiations.
#include "rlbm_kernels.cuh"

namespace rlbm {

cudaError_t launch_step_f32(const StepParams<float>& p, const void* fin, void* fout, int qb,
                            cudaStream_t s) {
  const long long nsite = (long long)p.Nx * p.Ny;
  const dim3 grid((unsigned)((nsite + 127) / 128)), block(128);
  const float* in = static_cast<const float*>(fin);
  float* out = static_cast<float*>(fout);
  switch (qb) {
    case 40: step_f32_kernel<40><<<grid, block, 0, s>>>(p, in, out); break;
    case 64: step_f32_kernel<64><<<grid, block, 0, s>>>(p, in, out); break;
    case 80: step_f32_kernel<80><<<grid, block, 0, s>>>(p, in, out); break;
    case 96: step_f32_kernel<96><<<grid, block, 0, s>>>(p, in, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rlbm
