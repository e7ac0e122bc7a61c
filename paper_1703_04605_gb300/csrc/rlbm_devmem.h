// Device memory of a context: cudaMalloc / cudaFree, or the caller-supplied
// allocator installed by rlbm_set_allocator when the context was created
// (include/rlbm.h).  Shared by the 2D and 3D host code.  Internal.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/rlbm.h"

namespace rlbm {

struct DevMem {
  rlbm_alloc_fn alloc = nullptr;   // nullptr: cudaMalloc / cudaFree
  rlbm_free_fn release = nullptr;
  void* user = nullptr;
  int device = 0;
  cudaStream_t stream = nullptr;

  // Blocks must be aligned like cudaMalloc's (256 bytes): the kernels use
  // vector loads, and the tables are read as rows.
  static constexpr std::uintptr_t kAlign = 256;

  template <class T>
  cudaError_t get(T** p, size_t bytes) const {
    void* q = nullptr;
    if (!alloc) {
      const cudaError_t e = cudaMalloc(&q, bytes);
      *p = static_cast<T*>(q);
      return e;
    }
    q = alloc(bytes, device, stream, user);
    if (q && reinterpret_cast<std::uintptr_t>(q) % kAlign != 0) {
      release(q, user);
      q = nullptr;
    }
    *p = static_cast<T*>(q);
    return q ? cudaSuccess : cudaErrorMemoryAllocation;
  }

  void put(void* p) const {
    if (!p) return;
    if (alloc) release(p, user);
    else cudaFree(p);
  }
};

// The allocator for a context created now on the current device and stream.
DevMem current_devmem(cudaStream_t stream);

}  // namespace rlbm
