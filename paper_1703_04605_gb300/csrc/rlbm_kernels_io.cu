// Init (f = f^eq) and read-out kernels for every storage type.
#include "rlbm_kernels.cuh"

namespace rlbm {

cudaError_t launch_init(rlbm_dtype dt, const StepParams<double>& p, FieldPtrs f, void* cur, void* prev,
                        cudaStream_t s) {
  const long long nsite = (long long)p.Nx * p.Ny;
  const dim3 grid((unsigned)((nsite + 127) / 128)), block(128);
  switch (dt) {
    case RLBM_F64:
      init_kernel<double><<<grid, block, 0, s>>>(p, f, static_cast<double*>(cur), static_cast<double*>(prev));
      break;
    case RLBM_F32:
      init_kernel<float><<<grid, block, 0, s>>>(p, f, static_cast<float*>(cur), static_cast<float*>(prev));
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_moments(rlbm_dtype dt, const StepParams<double>& p, const void* prev, MomentOut mo,
                           cudaStream_t s) {
  const long long nsite = (long long)p.Nx * p.Ny;
  const dim3 grid((unsigned)((nsite + 127) / 128)), block(128);
  switch (dt) {
    case RLBM_F64:
      moments_kernel<double><<<grid, block, 0, s>>>(p, static_cast<const double*>(prev), mo);
      break;
    case RLBM_F32:
      moments_kernel<float><<<grid, block, 0, s>>>(p, static_cast<const float*>(prev), mo);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rlbm
