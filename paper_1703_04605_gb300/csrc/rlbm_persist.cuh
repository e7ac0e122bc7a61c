// Persistent batched step kernel (rlbm_batch_step, persistent engine).
//
// One cooperative launch advances every lattice of a batch that shares a
// compiled stencil and storage variant by nsteps steps.  The work is cut into
// units -- a tile of 128 x spt consecutive sites of one lattice at one step --
// that the launch's blocks claim from a global ticket counter in step-major
// order (all units of step k before any unit of step k + 1; inside a step the
// order is fixed, largest lattices first).  A unit of lattice l at step k may
// start only when all units of l at step k - 1 are complete: it pulls values
// they wrote, and it overwrites the buffer they read.  Each block's first
// thread waits for that with a bounded poll of the lattice's completion
// counter; a wait that runs out of polls sets ERR_TIMEOUT in the error words
// of the launch's lattices and raises an abort flag on which every block stops
// claiming, so the launch always ends.
//
// Progress: a unit waits only on units with smaller tickets, which were
// claimed by blocks that are running (the launch is cooperative, so all its
// blocks are resident) and are either computing or waiting on still smaller
// tickets; the smallest waiting ticket's predecessors are therefore complete
// or being computed.
//
// Memory order: a unit's stores, a block barrier, then the first thread's
// device-scope fence and the counter increment; on the reading side the
// counter read with acquire semantics and a block barrier before the pulls,
// which go through L2 (ld.global.cg), not the read-only path.
#pragma once

#include "rlbm_fused.cuh"

namespace rlbm {

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <class Def, bool BF, int EXL>
__global__ void __launch_bounds__(128, fused_min_blocks<Def, BF, EXL>())
    persist_kernel(const __grid_constant__ PersistParams pp) {
  __shared__ FusedParams sp;
  __shared__ int s_lat, s_tile, s_step, s_go;
  const unsigned total = (unsigned)pp.units_per_step * (unsigned)pp.nsteps;
  for (;;) {
    if (threadIdx.x == 0) {
      int go = 0;
      if (ld_relaxed_gpu(pp.abort) == 0u) {
        const unsigned t = atomicAdd(pp.ticket, 1u);
        if (t < total) {
          const unsigned k = t / (unsigned)pp.units_per_step;
          const int2 lt = pp.units[t - k * (unsigned)pp.units_per_step];
          const unsigned target = k * (unsigned)pp.lat[lt.x].ntiles + pp.wait_offset;
          go = 1;
          unsigned polls = 0;
          while (ld_acquire_gpu(pp.done + lt.x) < target) {
            if (++polls > pp.spin_limit || ld_relaxed_gpu(pp.abort) != 0u) {
              // give up: every lattice of the launch reports the timeout
              if (atomicExch(pp.abort, 1u) == 0u)
                for (int l = 0; l < pp.nlat; ++l) atomicOr(pp.lat[l].p[0].err, ERR_TIMEOUT);
              go = 0;
              break;
            }
            __nanosleep(256);
          }
          s_lat = lt.x;
          s_tile = lt.y;
          s_step = (int)k;
        }
      }
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const int l = s_lat, tile = s_tile, k = s_step;
    const PersistLattice& L = pp.lat[l];
    const int par = pp.par0[l] ^ (k & 1);
    {
      // the lattice's parameters for this parity into shared memory
      static_assert(sizeof(FusedParams) % 8 == 0, "FusedParams is copied in 8-byte words");
      const uint2* src = reinterpret_cast<const uint2*>(&L.p[par]);
      uint2* dst = reinterpret_cast<uint2*>(&sp);
      for (int q = threadIdx.x; q < (int)(sizeof(FusedParams) / 8); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    const void* fin = L.buf[par];
    void* fout = const_cast<void*>(L.buf[1 - par]);
    unsigned fl = 0;
    for (int j = 0; j < pp.spt; ++j) {
      const int site = (tile * pp.spt + j) * 128 + (int)threadIdx.x;
      if (site < L.nsite) fused_site<Def, BF, EXL, true>(sp, fin, fout, site, fl);
    }
    report(fl, sp.err);
    __syncthreads();   // every store of the unit is issued
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(pp.done + l, 1u);
    }
  }
}

// Entry point for a stencil and storage variant (mode as fused_kernel_fn_impl).
template <class Def>
const void* persist_kernel_fn_impl(int mode) {
  return mode == 1 ? (const void*)&persist_kernel<Def, true, 0>
         : mode == 2 ? (const void*)&persist_kernel<Def, false, 1>
         : mode == 3 ? (const void*)&persist_kernel<Def, false, 2>
                     : (const void*)&persist_kernel<Def, false, 0>;
}

}  // namespace rlbm
