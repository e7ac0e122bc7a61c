// Host side of the field transfers of rlbm_init / rlbm3_init and the
// read-outs.  Validation of initial fields after their upload: one device
// pass over the uploaded copy finds the first site violating n > 0, T > 0,
// |u| < 1 (all finite) and sums the density per block (launch_field_check);
// the host adds the block sums in block order, so the mean density is the
// same on every run for a given lattice size.
#pragma once

#include <cstring>
#include <vector>

#include "rlbm_internal.h"

namespace rlbm {

struct FieldScan {
  size_t first_bad;   // index of the first invalid site, or N if none
  double nsum;        // sum of n over all sites (meaningful when first_bad == N)
  cudaError_t err;    // a CUDA error of the check itself
};

// d_n .. d_T: device copies of the fields (d_uz NULL in 2D); d_scan: device
// scratch of kScanBlocks + 1 doubles.  Synchronises the stream.
inline FieldScan check_fields(const double* d_n, const double* d_ux, const double* d_uy, const double* d_uz,
                              const double* d_T, size_t N, double* d_scan, cudaStream_t s) {
  FieldScan r{N, 0.0, cudaSuccess};
  unsigned long long* bad = reinterpret_cast<unsigned long long*>(d_scan + kScanBlocks);
  std::vector<double> h(kScanBlocks + 1, 0.0);
  cudaError_t e = cudaMemsetAsync(bad, 0xFF, sizeof(*bad), s);
  if (e == cudaSuccess) e = launch_field_check(d_n, d_ux, d_uy, d_uz, d_T, (long long)N, d_scan, bad, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), d_scan, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    r.err = e;
    return r;
  }
  unsigned long long first;
  std::memcpy(&first, &h[kScanBlocks], sizeof first);
  if (first < N) {
    r.first_bad = (size_t)first;
    return r;
  }
  const int nb = field_check_blocks((long long)N);
  for (int b = 0; b < nb; ++b) r.nsum += h[b];
  return r;
}

// Device alias of page-locked (mapped) host memory, NULL for any other
// memory.  The read-out kernels write such a buffer directly over the host
// link: the same bytes a staging copy would move, without the second pass.
inline double* mapped_alias(double* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? static_cast<double*>(a.devicePointer) : nullptr;
}

}  // namespace rlbm
