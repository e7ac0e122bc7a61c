// FP64-storage step kernel instantiations.
#include "rlbm_kernels.cuh"

namespace rlbm {

cudaError_t launch_step_f64(const StepParams<double>& p, const void* fin, void* fout, int qb,
                            cudaStream_t s) {
  const long long nsite = (long long)p.Nx * p.Ny;
  const dim3 grid((unsigned)((nsite + 127) / 128)), block(128);
  const double* in = static_cast<const double*>(fin);
  double* out = static_cast<double*>(fout);
  switch (qb) {
    case 40: step_f64_kernel<40><<<grid, block, 0, s>>>(p, in, out); break;
    case 64: step_f64_kernel<64><<<grid, block, 0, s>>>(p, in, out); break;
    case 80: step_f64_kernel<80><<<grid, block, 0, s>>>(p, in, out); break;
    case 96: step_f64_kernel<96><<<grid, block, 0, s>>>(p, in, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rlbm
