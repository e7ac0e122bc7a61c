// Third-order equilibrium: the deviations of the centred Maxwell-Juttner
// moments that weight the dual basis (shared by rlbm_kernels_o3.cu and
// rlbm_fused_o3.cu).
//
// Per unit density, with h = (e + P)/n = m R + 4T, R = K1/K2(m/T), U_z = 0
// and t = p0 - c, the moments of the twenty centred monomials (kO3Mono order)
// follow from <1> = R/m, <p^a> = U^a, <p^a p^b> = h U^a U^b - T eta^ab and
// <p^a p^b p^c> = A3 U^a U^b U^c + B3 (eta^ab U^c + eta^ac U^b + eta^bc U^a),
// A3 = m^2 + 6 T h, B3 = -T h (Eq. 4-6, 28-29, 43-44).  Their deviations from
// the values at rest and T = T_R are written out in dU = U0 - 1, dT = T - 1,
// dR = R - R(m), U_x, U_y, so every term is a deviation times an O(1) factor
// and FP32 evaluation has no cancellation.
#pragma once

#include "rlbm_internal.h"

namespace rlbm {

__device__ __forceinline__ double o3_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float o3_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double o3_rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float o3_rcp(float a) { return __fdividef(1.0f, a); }

// e_l = n dmu_l (kO3Mono order); m = m/T_R, c the centring shift of t.
template <typename R_t>
__device__ __forceinline__ void o3_deviations(R_t m, R_t c, R_t n, R_t U0, R_t Ux, R_t Uy, R_t dU, R_t dR,
                                              R_t dT, R_t T, R_t R, R_t (&e)[kO3Mono]) {
  const R_t h = o3_fma(m, R, R_t(4) * T);
  const R_t dh = o3_fma(m, dR, R_t(4) * dT);
  const R_t Th = T * h;
  const R_t Am = o3_fma(R_t(6), Th, m * m);      // A3
  const R_t hU = o3_fma(h, U0, -c);
  const R_t sdev = o3_fma(dT, hU, o3_fma(h, dU, dh));   // T (h U0 - c) - (h_r - c)
  const R_t q = o3_fma(Am, U0, -c * h);
  const R_t dRm = dR * o3_rcp(m);
  const R_t Ux2 = Ux * Ux, Uy2 = Uy * Uy, Uxy = Ux * Uy;
  e[0] = n * dRm;                                    // 1
  e[1] = n * o3_fma(-c, dRm, dU);                    // t
  e[2] = n * Ux;                                     // px
  e[3] = n * Uy;                                     // py
  e[4] = e[2] * hU;                                  // t px
  e[5] = e[3] * hU;                                  // t py
  e[6] = n * o3_fma(h, Ux2, dT);                     // px^2
  e[7] = n * o3_fma(h, Uy2, dT);                     // py^2
  e[8] = n * h * Uxy;                                // px py
  e[9] = n * dT;                                     // pz^2
  e[10] = n * o3_fma(q, Ux2, sdev);                  // t px^2
  e[11] = n * o3_fma(q, Uy2, sdev);                  // t py^2
  e[12] = n * q * Uxy;                               // t px py
  e[13] = e[2] * o3_fma(Am, Ux2, R_t(3) * Th);       // px^3
  e[14] = e[3] * o3_fma(Am, Ux2, Th);                // px^2 py
  e[15] = e[2] * o3_fma(Am, Uy2, Th);                // px py^2
  e[16] = e[3] * o3_fma(Am, Uy2, R_t(3) * Th);       // py^3
  e[17] = n * sdev;                                  // t pz^2
  e[18] = e[2] * Th;                                 // px pz^2
  e[19] = e[3] * Th;                                 // py pz^2
}

}  // namespace rlbm
