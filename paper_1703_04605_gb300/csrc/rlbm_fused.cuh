// Stencil-specialised FP32 step kernel (sm_103a).
//
// Same step as rlbm_kernels.cuh (pull, moments, Landau frame, n = U.N, EOS,
// projections, equilibrium, Anderson-Witting relaxation; Eq. 16-20, 28, 49),
// restructured for FP32 storage:
//
//  * the folded stencil is a compile-time constant, so every per-population
//    quantity is a small exact integer (displacement, n_x, n_y, multiplicity)
//    and the moments are accumulated per group with exact integer weights;
//    the group-level constants (momenta, weights, App. A/B normalisations)
//    enter as hi/lo pairs of FP32 numbers, so no constant carries a fixed
//    FP32 rounding that would bias the conserved moments step after step;
//  * the stored value is d_i = f_i - r_i with r_i the rest-frame equilibrium
//    at density nref and T = T_R (see StepParams in rlbm_internal.h), and every
//    site quantity is carried as (FP64 reference constant, FP32 deviation):
//    n = nref + n_d, e/n = y_r + y_d, T = 1 + T_d, R = R(mbar) + dR.  The
//    FP32 deviations are small, so FP32 arithmetic on them loses nothing that
//    the FP32 storage keeps;
//  * the Landau frame is solved in FP32 on the full moments (the velocity is
//    well conditioned; the cancelling energy and density are formed from the
//    deviation moments), and FP64 enters only the EOS: one FP64 Newton step
//    with the FP64 R(zeta) table after the FP32 iterations.  The same R enters
//    the EOS and the projections, which keeps the energy of f^eq equal to the
//    Landau energy (Eq. 20, 28).
#pragma once

#include <utility>

#include "rlbm_kernels.cuh"
#include "rlbm_stencils.h"

namespace rlbm {

__device__ __forceinline__ float hl(const HL& c, float x) { return fmaf(c.hi, x, c.lo * x); }
__device__ __forceinline__ float hl_fma(const HL& c, float x, float acc) {
  return fmaf(c.hi, x, fmaf(c.lo, x, acc));
}

// wrapped source coordinate x - D (requires N >= |D|)
template <int D>
__device__ __forceinline__ int wrap_c(int x, int N) {
  int r = x - D;
  if constexpr (D > 0) r += (r < 0) ? N : 0;
  if constexpr (D < 0) r -= (r >= N) ? N : 0;
  return r;
}

template <class Def, int I>
__device__ __forceinline__ void fused_load(float (&d)[Def::Q], const float* __restrict__ fin,
                                           long long plane, long long pitch, int x, int y, int Nx, int Ny) {
  constexpr int DX = Def::F.nx[I], DY = Def::F.ny[I];
  const int xs = wrap_c<DX>(x, Nx);
  const int ys = wrap_c<DY>(y, Ny);
  d[I] = __ldg(fin + (long long)I * plane + (long long)ys * pitch + xs);
}

template <class Def, int I>
__device__ __forceinline__ void fused_acc(const float (&d)[Def::Q], float (&s)[6][6]) {
  constexpr int g = Def::F.grp[I], nx = Def::F.nx[I], ny = Def::F.ny[I];
  const float v = d[I];
  s[g][0] += v;
  if constexpr (nx != 0) s[g][1] = fmaf((float)nx, v, s[g][1]);
  if constexpr (ny != 0) s[g][2] = fmaf((float)ny, v, s[g][2]);
  if constexpr (nx != 0) s[g][3] = fmaf((float)(nx * nx), v, s[g][3]);
  if constexpr (nx != 0 && ny != 0) s[g][4] = fmaf((float)(nx * ny), v, s[g][4]);
  if constexpr (ny != 0) s[g][5] = fmaf((float)(ny * ny), v, s[g][5]);
}

template <class Def, int I>
__device__ __forceinline__ void fused_collide(const float (&d)[Def::Q], const float (&c)[6][6], float a0,
                                              float ax, float ay, float* __restrict__ out, long long plane) {
  constexpr int g = Def::F.grp[I], nx = Def::F.nx[I], ny = Def::F.ny[I], mult = Def::F.mult[I];
  // group polynomial alpha + bx nx + by ny + qxx nx^2 + qyy ny^2 + qxy nx ny
  float e = c[g][0];
  if constexpr (nx != 0) e = fmaf((float)nx, c[g][1], e);
  if constexpr (ny != 0) e = fmaf((float)ny, c[g][2], e);
  if constexpr (nx != 0) e = fmaf((float)(nx * nx), c[g][3], e);
  if constexpr (ny != 0) e = fmaf((float)(ny * ny), c[g][4], e);
  if constexpr (nx != 0 && ny != 0) e = fmaf((float)(nx * ny), c[g][5], e);
  if constexpr (mult != 1) e *= (float)mult;
  // weight p_i.U/(p_i^0 tau) = (U0 - v0 (nx Ux + ny Uy))/tau
  float om = a0;
  if constexpr (nx != 0) om = fmaf(-(float)nx, ax, om);
  if constexpr (ny != 0) om = fmaf(-(float)ny, ay, om);
  const float v = d[I];
  __stcs(out + (long long)I * plane, fmaf(om, e - v, v));
}

template <class Def, int... Is>
__device__ __forceinline__ void fused_load_all(std::integer_sequence<int, Is...>, float (&d)[Def::Q],
                                               const float* __restrict__ fin, long long plane, long long pitch,
                                               int x, int y, int Nx, int Ny) {
  (fused_load<Def, Is>(d, fin, plane, pitch, x, y, Nx, Ny), ...);
}

template <class Def, int... Is>
__device__ __forceinline__ void fused_acc_all(std::integer_sequence<int, Is...>, const float (&d)[Def::Q],
                                              float (&s)[6][6]) {
  (fused_acc<Def, Is>(d, s), ...);
}

template <class Def, int... Is>
__device__ __forceinline__ void fused_collide_all(std::integer_sequence<int, Is...>, const float (&d)[Def::Q],
                                                  const float (&c)[6][6], float a0, float ax, float ay,
                                                  float* __restrict__ out, long long plane) {
  (fused_collide<Def, Is>(d, c, a0, ax, ay, out, plane), ...);
}

// Five resident blocks of 128 threads (96 registers) for Q <= 64, four
// (128 registers) for larger stencils, whose populations would spill.
template <class Def>
__global__ void __launch_bounds__(128, Def::Q <= 64 ? 5 : 4) fused_f32_kernel(const __grid_constant__ FusedParams p,
                                                        const float* __restrict__ fin,
                                                        float* __restrict__ fout) {
  constexpr int Q = Def::Q;
  using Seq = std::make_integer_sequence<int, Q>;
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (site < p.Nx * p.Ny) {
    int x, y;
    site_of(site, p.Nx, x, y);
    float d[Q];
    fused_load_all<Def>(Seq{}, d, fin, p.plane, p.pitch, x, y, p.Nx, p.Ny);
    float s[6][6];
#pragma unroll
    for (int g = 0; g < 6; ++g)
#pragma unroll
      for (int k = 0; k < 6; ++k) s[g][k] = 0.0f;
    fused_acc_all<Def>(Seq{}, d, s);

    // deviation moments N0 Nx Ny T00 T0x T0y Txx Txy Tyy (reference excluded)
    float M[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) M[k] = 0.0f;
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      M[0] = hl_fma(p.gm[g][0], s[g][0], M[0]);
      M[3] = hl_fma(p.gm[g][1], s[g][0], M[3]);
      M[1] = hl_fma(p.gm[g][2], s[g][1], M[1]);
      M[2] = hl_fma(p.gm[g][2], s[g][2], M[2]);
      M[4] = hl_fma(p.gm[g][3], s[g][1], M[4]);
      M[5] = hl_fma(p.gm[g][3], s[g][2], M[5]);
      M[6] = hl_fma(p.gm[g][4], s[g][3], M[6]);
      M[7] = hl_fma(p.gm[g][4], s[g][4], M[7]);
      M[8] = hl_fma(p.gm[g][4], s[g][5], M[8]);
    }

    // Landau frame: FP32 Newton on the full moments.  v = T^0i/(...) is well
    // conditioned (relative error ~ FP32 rounding); the cancelling parts of the
    // energy and density are formed below from the deviation moments.
    float Mf[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Mf[k] = p.mref[k].hi + (p.mref[k].lo + M[k]);
    float vx, vy, dvx, dvy;
    {
      const float iden = __fdividef(1.0f, Mf[3] + 0.5f * (Mf[6] + Mf[8]));
      vx = Mf[4] * iden;
      vy = Mf[5] * iden;
#pragma unroll 1
      for (int it = 0; it < 8; ++it) {
        landau_newton_step_fast(Mf, vx, vy, dvx, dvy);
        if (fabsf(dvx) + fabsf(dvy) < 1e-7f) break;
      }
    }
    const float v2 = vx * vx + vy * vy;
    if (!(v2 < 1.0f)) fl |= ERR_LANDAU;
    const float sq = sqrtf(1.0f - v2);
    const float dg = __fdividef(v2, sq * (1.0f + sq));  // gamma - 1
    const float U0 = 1.0f + dg, Ux = U0 * vx, Uy = U0 * vy;
    // n = U.N = n_r + n_d
    const float Xi = M[0] - vx * M[1] - vy * M[2];
    const float nd = fmaf(dg, p.nr.lo, fmaf(dg, Xi + p.nr.hi, Xi));
    const float n = p.nr.hi + (p.nr.lo + nd);
    if (!(n > 0.0f)) fl |= ERR_DENSITY;
    // e/n = y_r + y_d
    const float ed = M[3] - M[4] * vx - M[5] * vy;
    const float yd = __fdividef(ed - fmaf(p.yr.hi, nd, p.yr.lo * nd), n);
    if (!(p.yr.hi + yd > p.mb)) fl |= ERR_EOS;
    // EOS: T = 1 + T_d solves 3 T_d + m (R(m/T) - R_r) = y_d.  FP32 Newton ...
    float Td = yd / p.cv_r, slope = p.cv_r, R32 = p.Rr.hi;
#pragma unroll 1
    for (int it = 0; it < 12; ++it) {
      const float T = 1.0f + Td;
      if (!(T > 0.0f)) {
        fl |= ERR_EOS;
        Td = 0.0f;
        break;
      }
      const float z = __fdividef(p.mb, T);
      R32 = ratio32(z, p.rt32, fl);
      const float dR = (R32 - p.Rr.hi) - p.Rr.lo;
      slope = eos_slope<float>(R32, z);
      const float step = __fdividef(3.0f * Td + p.mb * dR - yd, slope);
      Td -= step;
      if (fabsf(step) < 3e-8f) break;
    }
    // ... and one FP64 Newton step with the FP64 R(zeta) table
    float dR;
    {
      const float Tf = 1.0f + Td;
      const double T64 = 1.0 + (double)Td;
      double iT = (double)__fdividef(1.0f, Tf);
      iT = fma(iT, fma(-T64, iT, 1.0), iT);
      const double z64 = p.mb64 * iT;
      const double dR64 = ratio64(z64, p.rt64, fl) - p.Rr64;
      const double g64 = fma(3.0, (double)Td, fma(p.mb64, dR64, -(double)yd));
      const float step = __fdividef((float)g64, slope);
      Td -= step;
      const float R = p.Rr.hi + (p.Rr.lo + (float)dR64);
      const float z = (float)z64;
      const float dRdz = R * R + 3.0f * __fdividef(R, z) - 1.0f;
      dR = fmaf(dRdz, z * step / Tf, (float)dR64);     // R at the corrected T (first order)
    }
    const float R = p.Rr.hi + (p.Rr.lo + dR);
    const float T = 1.0f + Td;
    // projections without their normalisations (those live in p.gf)
    const float mr32 = fmaf(p.mb, R, 4.0f * T);          // mbar K3/K2(zeta)
    const float r0 = fmaf(p.nr.hi, dR, fmaf(p.nr.lo, dR, nd * R));   // n R - n_r R_r
    const float r1 = n * (dg - p.k21 * dR);
    const float r2 = n * Ux, r3 = n * Uy;
    const float F = fmaf(p.mY, dR, 3.0f * Td);
    const float G = fmaf(p.mb, dR, 4.0f * Td);
    const float r4 = n * (F + dg * fmaf(2.0f, mr32, p.cb00_1) + dg * dg * mr32);
    const float h = fmaf(mr32, dg, G);
    const float r5 = n * h * Ux, r6 = n * h * Uy;
    const float nm = n * mr32;
    const float r7 = nm * Uy * Uy, r8 = nm * (Uy * Uy - 2.0f * Ux * Ux), r9 = nm * Ux * Uy;
    float c[6][6];
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      const HL* a = p.gf[g];
      float al = hl(a[0], r0);
      al = hl_fma(a[1], r1, al);
      al = hl_fma(a[2], r4, al);
      al = hl_fma(a[3], r7, al);
      al = hl_fma(a[4], r8, al);
      c[g][0] = al;
      c[g][1] = hl_fma(a[5], r2, hl(a[6], r5));
      c[g][2] = hl_fma(a[5], r3, hl(a[6], r6));
      c[g][3] = hl(a[7], r7 - r8);
      c[g][4] = hl(a[8], r7);
      c[g][5] = hl(a[9], r9);
    }
    const float a0 = U0 * p.inv_tau, ax = p.v0 * Ux * p.inv_tau, ay = p.v0 * Uy * p.inv_tau;
    fused_collide_all<Def>(Seq{}, d, c, a0, ax, ay, fout + (long long)y * p.pitch + x, p.plane);
  }
  report(fl, p.err);
}

}  // namespace rlbm
