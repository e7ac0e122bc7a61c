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

namespace {

__global__ void __launch_bounds__(256) field_check_kernel(const double* __restrict__ n, const double* __restrict__ ux,
                                                          const double* __restrict__ uy, const double* __restrict__ uz,
                                                          const double* __restrict__ T, long long N, long long len,
                                                          double* __restrict__ part, unsigned long long* bad) {
  __shared__ double red[256];
  const long long lo = (long long)blockIdx.x * len;
  const long long hi = lo + len < N ? lo + len : N;
  double sum = 0.0;
  unsigned long long first = ~0ull;
  for (long long i = lo + threadIdx.x; i < hi; i += 256) {
    double v2 = ux[i] * ux[i] + uy[i] * uy[i];
    if (uz) v2 += uz[i] * uz[i];
    const double ni = n[i], Ti = T[i];
    if (!(ni > 0.0) || !(Ti > 0.0) || !(v2 < 1.0) || !isfinite(ni) || !isfinite(Ti)) {
      if (first == ~0ull) first = (unsigned long long)i;   // this thread's smallest
    } else {
      sum += ni;
    }
  }
  if (first != ~0ull) atomicMin(bad, first);
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

}  // namespace

int field_check_blocks(long long N) {
  const long long b = (N + 255) / 256;
  return (int)(b < kScanBlocks ? b : kScanBlocks);
}

cudaError_t launch_field_check(const double* n, const double* ux, const double* uy, const double* uz,
                               const double* T, long long N, double* part, unsigned long long* bad,
                               cudaStream_t s) {
  const int blocks = field_check_blocks(N);
  const long long len = (N + blocks - 1) / blocks;
  field_check_kernel<<<blocks, 256, 0, s>>>(n, ux, uy, uz, T, N, len, part, bad);
  return cudaGetLastError();
}

}  // namespace rlbm
