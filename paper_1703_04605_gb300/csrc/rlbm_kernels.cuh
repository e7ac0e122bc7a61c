// Device code of the relativistic lattice Boltzmann step (sm_103a).
//
// One thread owns one lattice site.  The step pulls the Q populations that
// stream into the site (Eq. 49 read backwards: f_i(x, t+1) = f*_i(x - n_i, t)),
// forms N^a and T^ab (Eq. 4-5, 18), solves the Landau frame (Eq. 20), n = U.N
// (Eq. 19), the EOS for T (Eq. 28), the projections b^(k) (App. B), the
// equilibrium (Eq. 16) and the Anderson-Witting relaxation (Eq. 49), and
// stores the post-collision populations at its own site.  The stored state
// S_t is therefore post-collision: S_t(x) = f*(x, t), and f(x, t+1) is the
// pull of S_t.
//
// Population storage is structure of arrays: plane i holds population i as
// [Ny][pitch] elements.  The per-population constants travel in the kernel
// parameter block (__grid_constant__), so the fully unrolled population loop
// reads them as constant-bank operands.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rlbm_internal.h"

namespace rlbm {

// ------------------------------------------------------------------ R(zeta)
// Small-zeta series and large-zeta asymptotic ratio, used outside the table:
//   R ~ (z/2)(1 + z^2/4 + (z^2/2)(ln(z/2) + gamma_E - 1/2))       (z -> 0)
//   R ~ P1(1/z)/P2(1/z), P_nu the Hankel asymptotic series of K_nu (z -> inf)
template <typename R_t>
__device__ __forceinline__ R_t ratio_outside(R_t z) {
  if (z < R_t(1)) {
    const R_t ge = R_t(0.57721566490153286061);
    R_t z2 = z * z;
    return R_t(0.5) * z * (R_t(1) + R_t(0.25) * z2 + R_t(0.5) * z2 * (log(R_t(0.5) * z) + ge - R_t(0.5)));
  }
  R_t u = R_t(1) / z;
  R_t p1 = R_t(1) + u * (R_t(0.375) + u * (R_t(-0.1171875) + u * R_t(0.1025390625)));
  R_t p2 = R_t(1) + u * (R_t(1.875) + u * (R_t(0.8203125) + u * R_t(-0.3076171875)));
  return p1 / p2;
}

__device__ __forceinline__ double ratio64(double z, const double* __restrict__ tab, unsigned& fl) {
  if (!(z > 0.0) || !isfinite(z)) {
    fl |= ERR_ZETA;
    return 0.5;
  }
  const long long bits = __double_as_longlong(z);
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;
  if (e < RT_EMIN || e >= RT_EMAX) return ratio_outside<double>(z);
  const int j = (int)((bits >> 49) & 7);
  const double d = __longlong_as_double(((bits & ((1LL << 49) - 1)) << 3) | 0x3FF0000000000000LL);
  const double x = 2.0 * d - 3.0;                 // exact: local variable in [-1, 1)
  const double* c = tab + ((e - RT_EMIN) * RT_SEG + j) * RT_NC64;
  double r = __ldg(c + RT_NC64 - 1);
#pragma unroll
  for (int k = RT_NC64 - 2; k >= 0; --k) r = fma(r, x, __ldg(c + k));
  return r;
}

// dR(Td) = R(mbar/(1 + Td)) - R(mbar) from the lattice's table (layout in
// rlbm_internal.h); false outside the tabulated range (or for NaN).  The
// local variable is formed exactly in FP32: 64 Td is an exact scaling and
// 64 Td - trunc(64 Td) an exact difference (the operands agree in sign and
// are within a factor of two, or the truncation is zero).
__device__ __forceinline__ bool dr_table64(float Td, const double* __restrict__ tab, double& dR) {
  if (!(fabsf(Td) < 3.5f)) return false;
  const float s = Td * 64.0f;
  const float k = truncf(s);
  const int ki = (int)k;
  int idx;
  if (Td >= 0.0f) {
    if (ki >= DR_NPOS) return false;
    idx = DR_NNEG + ki;
  } else {
    if (ki <= -DR_NNEG) return false;
    idx = DR_NNEG - 1 + ki;
  }
  const double x = (double)(s - k);
  const double* c = tab + idx * DR_NC;
  double r = __ldg(c + DR_NC - 1);
#pragma unroll
  for (int q = DR_NC - 2; q >= 0; --q) r = fma(r, x, __ldg(c + q));
  dR = r;
  return true;
}

__device__ __forceinline__ float ratio32(float z, const float* __restrict__ tab, unsigned& fl) {
  if (!(z > 0.0f) || !isfinite(z)) {
    fl |= ERR_ZETA;
    return 0.5f;
  }
  const int bits = __float_as_int(z);
  const int e = ((bits >> 23) & 0xff) - 127;
  if (e < RT_EMIN || e >= RT_EMAX) return ratio_outside<float>(z);
  const int j = (bits >> 20) & 7;
  const float d = __int_as_float(((bits & 0xFFFFF) << 3) | 0x3F800000);
  const float x = 2.0f * d - 3.0f;
  const float* c = tab + ((e - RT_EMIN) * RT_SEG + j) * RT_NC32;
  float r = __ldg(c + RT_NC32 - 1);
#pragma unroll
  for (int k = RT_NC32 - 2; k >= 0; --k) r = fmaf(r, x, __ldg(c + k));
  return r;
}

// dR/dzeta = R^2 + 3R/zeta - 1 (from K_nu' recurrences); g'(T) = 3 - zeta^2 R'
// is the specific heat per particle, in [3/2, 3]; clamped there.
template <typename R_t>
__device__ __forceinline__ R_t eos_slope(R_t R, R_t z) {
  R_t d = R_t(3) - z * (z * (R * R - R_t(1)) + R_t(3) * R);
  return fmin(fmax(d, R_t(1.5)), R_t(3));
}

// ------------------------------------------------------------ Landau frame
// T^ab U_b = e U^a with U = gamma (1, v): e = T00 - T0x vx - T0y vy and
//   Fx = T0x - Txx vx - Txy vy - e vx = 0,  Fy = T0y - Txy vx - Tyy vy - e vy = 0.
// Newton on (vx, vy) from the guess v = T^0i / (T00 + (Txx + Tyy)/2).
template <typename R_t>
struct Landau {
  R_t vx, vy;
};

template <typename R_t>
__device__ __forceinline__ void landau_newton_step(const R_t* m, R_t& vx, R_t& vy, R_t& dvx, R_t& dvy) {
  // m: N0 Nx Ny T00 T0x T0y Txx Txy Tyy
  const R_t T00 = m[3], T0x = m[4], T0y = m[5], Txx = m[6], Txy = m[7], Tyy = m[8];
  const R_t e = T00 - T0x * vx - T0y * vy;
  const R_t Fx = T0x - Txx * vx - Txy * vy - e * vx;
  const R_t Fy = T0y - Txy * vx - Tyy * vy - e * vy;
  const R_t J11 = -Txx - e + vx * T0x, J12 = -Txy + vx * T0y;
  const R_t J21 = -Txy + vy * T0x, J22 = -Tyy - e + vy * T0y;
  const R_t idet = R_t(1) / (J11 * J22 - J12 * J21);
  dvx = (J22 * Fx - J12 * Fy) * idet;
  dvy = (J11 * Fy - J21 * Fx) * idet;
  vx -= dvx;
  vy -= dvy;
}

// FP32 variant with an approximate reciprocal (the iteration corrects it).
__device__ __forceinline__ void landau_newton_step_fast(const float* m, float& vx, float& vy, float& dvx,
                                                        float& dvy) {
  const float T00 = m[3], T0x = m[4], T0y = m[5], Txx = m[6], Txy = m[7], Tyy = m[8];
  const float e = T00 - T0x * vx - T0y * vy;
  const float Fx = T0x - Txx * vx - Txy * vy - e * vx;
  const float Fy = T0y - Txy * vx - Tyy * vy - e * vy;
  const float J11 = -Txx - e + vx * T0x, J12 = -Txy + vx * T0y;
  const float J21 = -Txy + vy * T0x, J22 = -Tyy - e + vy * T0y;
  const float idet = __fdividef(1.0f, J11 * J22 - J12 * J21);
  dvx = (J22 * Fx - J12 * Fy) * idet;
  dvy = (J11 * Fy - J21 * Fx) * idet;
  vx -= dvx;
  vy -= dvy;
}

// ------------------------------------------------------------ site macros
template <typename R_t>
struct Macro {
  R_t n, U0, Ux, Uy, T, zeta, R;
  R_t dU;      // U0 - 1
  R_t F, G;    // thermal parts of b_00 and b_0a (see rlbm_internal.h)
  R_t dR;      // R - Rr
};

// Full FP64 site solve (the FP64 storage path, init and read-out).
__device__ __forceinline__ Macro<double> solve_site_f64(const double* m, const SiteConsts& sc,
                                                       const double* __restrict__ rt64, unsigned& fl) {
  double vx, vy;
  {
    const double den = m[3] + 0.5 * (m[6] + m[8]);
    vx = m[4] / den;
    vy = m[5] / den;
    double dvx, dvy;
#pragma unroll 1
    for (int it = 0; it < 16; ++it) {
      landau_newton_step<double>(m, vx, vy, dvx, dvy);
      if (fabs(dvx) + fabs(dvy) < 1e-15) break;
    }
  }
  Macro<double> o;
  const double v2 = vx * vx + vy * vy;
  if (!(v2 < 1.0)) fl |= ERR_LANDAU;
  const double e = m[3] - m[4] * vx - m[5] * vy;
  const double g = 1.0 / sqrt(1.0 - v2);
  o.U0 = g;
  o.dU = g * g * v2 / (g + 1.0);
  o.Ux = g * vx;
  o.Uy = g * vy;
  o.n = g * (m[0] - vx * m[1] - vy * m[2]);
  if (!(o.n > 0.0)) fl |= ERR_DENSITY;
  const double y = e / o.n;                      // energy per particle
  const double mb = sc.mbar;
  if (!(y > mb)) fl |= ERR_EOS;
  // Newton on g(T) = 3T + m R(m/T) - y; g is increasing and convex in T, so
  // Newton converges from any positive start (first step lands right of root).
  double T = (y - mb) / (3.0 - 1.5 * (mb * mb) / (y * y));
  double R = 0.0, z = 0.0;
#pragma unroll 1
  for (int it = 0; it < 40; ++it) {
    z = mb / T;
    R = ratio64(z, rt64, fl);
    const double gT = 3.0 * T + mb * R - y;
    const double dT = gT / eos_slope<double>(R, z);
    T -= dT;
    if (!(T > 0.0)) {
      fl |= ERR_EOS;
      T = 1.0;
      break;
    }
    if (fabs(dT) < 1e-15 * T) break;
  }
  z = mb / T;
  R = ratio64(z, rt64, fl);
  o.T = T;
  o.zeta = z;
  o.R = R;
  o.dR = R - sc.Rr;
  o.F = sc.mY * o.dR + 3.0 * (T - 1.0);
  o.G = mb * o.dR + 4.0 * (T - 1.0);
  return o;
}

// FP32 site solve with FP64 correction steps (the FP32 / BF16 storage paths).
// Landau: FP32 Newton, then one Newton step whose residual is formed in FP64
// (the FP32 Jacobian inverse is enough: the step squares an error that is
// already ~1e-7).  EOS: FP32 Newton, then one FP64 Newton step with the FP64
// R(zeta) table.  Returns FP64 macros; the caller rounds what it needs.
// m: the full moments in FP64.
__device__ __forceinline__ Macro<double> solve_site_mixed_m(const double (&m)[9], const SiteConsts& sc,
                                                           const double* __restrict__ rt64,
                                                           const float* __restrict__ rt32, unsigned& fl) {
  float mf[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) mf[k] = (float)m[k];
  float vx, vy;
  float J11, J12, J21, J22;
  {
    const float den = mf[3] + 0.5f * (mf[6] + mf[8]);
    vx = __fdividef(mf[4], den);
    vy = __fdividef(mf[5], den);
    float dvx, dvy;
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
      landau_newton_step<float>(mf, vx, vy, dvx, dvy);
      if (fabsf(dvx) + fabsf(dvy) < 2e-7f) break;
    }
    const float e = mf[3] - mf[4] * vx - mf[5] * vy;
    J11 = -mf[6] - e + vx * mf[4];
    J12 = -mf[7] + vx * mf[5];
    J21 = -mf[7] + vy * mf[4];
    J22 = -mf[8] - e + vy * mf[5];
  }
  // FP64 correction of (vx, vy)
  double Vx = vx, Vy = vy;
  {
    const double e = m[3] - m[4] * Vx - m[5] * Vy;
    const double Fx = m[4] - m[6] * Vx - m[7] * Vy - e * Vx;
    const double Fy = m[5] - m[7] * Vx - m[8] * Vy - e * Vy;
    const float idet = 1.0f / (J11 * J22 - J12 * J21);
    const float fx = (float)Fx, fy = (float)Fy;
    Vx -= (double)((J22 * fx - J12 * fy) * idet);
    Vy -= (double)((J11 * fy - J21 * fx) * idet);
  }
  Macro<double> o;
  const double v2 = Vx * Vx + Vy * Vy;
  if (!(v2 < 1.0)) fl |= ERR_LANDAU;
  const double e = m[3] - m[4] * Vx - m[5] * Vy;
  // gamma = 1/sqrt(1 - v2): FP32 seed, one FP64 Newton step for rsqrt
  const double s = 1.0 - v2;
  double g = (double)rsqrtf((float)s);
  g = g * (1.5 - 0.5 * s * g * g);
  o.U0 = g;
  o.dU = g * g * v2 / (g + 1.0);
  o.Ux = g * Vx;
  o.Uy = g * Vy;
  o.n = g * (m[0] - Vx * m[1] - Vy * m[2]);
  if (!(o.n > 0.0)) fl |= ERR_DENSITY;
  // y = e/n: FP32 reciprocal seed + one FP64 correction
  const float rn = 1.0f / (float)o.n;
  double y = e * (double)rn;
  y = y + (double)rn * (e - o.n * y);
  const double mb = sc.mbar;
  if (!(y > mb)) fl |= ERR_EOS;
  // FP32 Newton for T
  const float mbf = (float)mb, yf = (float)y;
  float Tf = (yf - mbf) / (3.0f - 1.5f * (mbf * mbf) / (yf * yf));
  float slope = 1.5f;
#pragma unroll 1
  for (int it = 0; it < 12; ++it) {
    const float z = mbf / Tf;
    const float R = ratio32(z, rt32, fl);
    slope = eos_slope<float>(R, z);
    const float dT = (3.0f * Tf + mbf * R - yf) / slope;
    Tf -= dT;
    if (!(Tf > 0.0f)) {
      fl |= ERR_EOS;
      Tf = 1.0f;
      break;
    }
    if (fabsf(dT) < 1e-7f * Tf) break;
  }
  // FP64 correction step: zeta = mb/T with an FP32 reciprocal seed
  double T = Tf;
  const float rT = 1.0f / Tf;
  double iT = (double)rT;
  iT = iT + iT * (1.0 - T * iT);
  double z = mb * iT;
  double R = ratio64(z, rt64, fl);
  const double dT = (3.0 * T + mb * R - y) / (double)slope;
  T -= dT;
  // first-order updates of zeta and R for the corrected T (errors O(dT^2))
  const double dz = z * dT * iT;
  z += dz;
  const float dRdz = (float)R * (float)R + 3.0f * (float)R * (float)iT / mbf - 1.0f;
  R += (double)dRdz * dz;
  o.T = T;
  o.zeta = z;
  o.R = R;
  o.dR = R - sc.Rr;
  o.F = sc.mY * o.dR + 3.0 * (T - 1.0);
  o.G = mb * o.dR + 4.0 * (T - 1.0);
  return o;
}

// Full moments = FP32 partial sums of the stored deviations + FP64 reference.
__device__ __forceinline__ Macro<double> solve_site_mixed(const float* mpart, const double* mref,
                                                         const SiteConsts& sc,
                                                         const double* __restrict__ rt64,
                                                         const float* __restrict__ rt32, unsigned& fl) {
  double m[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) m[k] = (double)mpart[k] + mref[k];
  return solve_site_mixed_m(m, sc, rt64, rt32, fl);
}

// n times the ten projections b^(k) (App. B), in the order of PopTable::cj.
template <typename R_t>
__device__ __forceinline__ void projections(const Macro<double>& md, const SiteConsts& sc, R_t* bn) {
  const R_t n = (R_t)md.n, U0 = (R_t)md.U0, Ux = (R_t)md.Ux, Uy = (R_t)md.Uy, dU = (R_t)md.dU;
  const R_t R = (R_t)md.R, T = (R_t)md.T;
  const R_t mr32 = (R_t)sc.mbar * R + R_t(4) * T;   // mbar K3/K2(zeta)
  bn[0] = n * R * (R_t)sc.inv_m;
  bn[1] = n * (dU - (R_t)sc.k21 * (R_t)md.dR) * (R_t)sc.iA;
  bn[2] = n * Ux * (R_t)sc.iB;
  bn[3] = n * Uy * (R_t)sc.iB;
  bn[4] = n * ((R_t)md.F + dU * (R_t(2) * mr32 + (R_t)sc.cb00_1) + dU * dU * mr32) * (R_t)sc.i3C;
  const R_t h = ((R_t)md.G + mr32 * dU) * (R_t)sc.iD;
  bn[5] = n * h * Ux;
  bn[6] = n * h * Uy;
  bn[7] = n * mr32 * Uy * Uy * (R_t)sc.i2E;
  bn[8] = n * mr32 * (Uy * Uy - R_t(2) * Ux * Ux) * (R_t)sc.i23E;
  bn[9] = n * mr32 * Ux * Uy * (R_t)sc.iE;
  (void)U0;
}

// ---------------------------------------------------------------- storage
template <typename S>
struct Store;
template <>
struct Store<double> {
  static __device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(double* p, double v) { __stcs(p, v); }
};
template <>
struct Store<float> {
  static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(float* p, float v) { __stcs(p, v); }
};

__device__ __forceinline__ void site_of(int s, int Nx, int& x, int& y) {
  y = s / Nx;
  x = s - y * Nx;
}

__device__ __forceinline__ int wrap_sub(int a, int d, int N) {
  int r = a - d;           // a in [0, N), d in [0, N)
  return r + ((r >> 31) & N);
}

__device__ __forceinline__ void report(unsigned fl, unsigned* err) {
  const unsigned any = __reduce_or_sync(0xffffffffu, fl);
  if (any && (threadIdx.x & 31) == 0) atomicOr(err, any);
}

// ------------------------------------------------------------ step kernels
// FP64 storage and arithmetic.
template <int QB>
__global__ void __launch_bounds__(128) step_f64_kernel(const __grid_constant__ StepParams<double> p,
                                                       const double* __restrict__ fin,
                                                       double* __restrict__ fout) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int nsite = p.Nx * p.Ny;
  unsigned fl = 0;
  if (s < nsite) {
    int x, y;
    site_of(s, p.Nx, x, y);
    double f[QB];
#pragma unroll
    for (int i = 0; i < QB; ++i) {
      if (i < p.Q) {
        const int xs = wrap_sub(x, p.pt.dxm[i], p.Nx);
        const int ys = wrap_sub(y, p.pt.dym[i], p.Ny);
        f[i] = Store<double>::ld(fin + i * p.plane + (long long)ys * p.pitch + xs);
      } else {
        f[i] = 0.0;
      }
    }
    double m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = 0.0;
#pragma unroll
    for (int i = 0; i < QB; ++i) {
      if (i < p.Q) {
#pragma unroll
        for (int k = 0; k < 9; ++k) m[k] = fma(f[i], p.pt.mom[k][i], m[k]);
      }
    }
    const Macro<double> md = solve_site_f64(m, p.sc, p.rt64, fl);
    double bn[NJ];
    projections<double>(md, p.sc, bn);
    const double a0 = md.U0 * p.inv_tau, ax = md.Ux * p.inv_tau, ay = md.Uy * p.inv_tau;
    double* o = fout + (long long)y * p.pitch + x;
#pragma unroll
    for (int i = 0; i < QB; ++i) {
      if (i < p.Q) {
        double feq = bn[0] * p.pt.cj[0][i];
#pragma unroll
        for (int k = 1; k < NJ; ++k) feq = fma(bn[k], p.pt.cj[k][i], feq);
        const double om = a0 - ax * p.pt.vx[i] - ay * p.pt.vy[i];
        Store<double>::st(o + i * p.plane, fma(om, feq - f[i], f[i]));
      }
    }
  }
  report(fl, p.err);
}

// FP32 storage of d_i = f_i - r_i (see StepParams), FP32 accumulation, FP64
// correction of Landau and EOS.
template <int QB>
__global__ void __launch_bounds__(128) step_f32_kernel(const __grid_constant__ StepParams<float> p,
                                                       const float* __restrict__ fin,
                                                       float* __restrict__ fout) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int nsite = p.Nx * p.Ny;
  unsigned fl = 0;
  if (s < nsite) {
    int x, y;
    site_of(s, p.Nx, x, y);
    float f[QB];
#pragma unroll
    for (int i = 0; i < QB; ++i) {
      if (i < p.Q) {
        const int xs = wrap_sub(x, p.pt.dxm[i], p.Nx);
        const int ys = wrap_sub(y, p.pt.dym[i], p.Ny);
        f[i] = Store<float>::ld(fin + i * p.plane + (long long)ys * p.pitch + xs);
      } else {
        f[i] = 0.0f;
      }
    }
    float m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = 0.0f;
#pragma unroll
    for (int i = 0; i < QB; ++i) {
      if (i < p.Q) {
#pragma unroll
        for (int k = 0; k < 9; ++k) m[k] = fmaf(f[i], p.pt.mom[k][i], m[k]);
      }
    }
    const Macro<double> md = solve_site_mixed(m, p.mref, p.sc, p.rt64, p.rt32, fl);
    float bn[NJ];
    projections<float>(md, p.sc, bn);
    // equilibrium minus the reference r_i: shift of the J^(0) coefficient, in FP64
    bn[0] = (float)(md.n * md.R * p.sc.inv_m - p.b0ref);
    const float it = (float)p.inv_tau;
    const float a0 = (float)md.U0 * it, ax = (float)md.Ux * it, ay = (float)md.Uy * it;
    float* o = fout + (long long)y * p.pitch + x;
#pragma unroll
    for (int i = 0; i < QB; ++i) {
      if (i < p.Q) {
        float feq = bn[0] * p.pt.cj[0][i];
#pragma unroll
        for (int k = 1; k < NJ; ++k) feq = fmaf(bn[k], p.pt.cj[k][i], feq);
        const float om = a0 - ax * p.pt.vx[i] - ay * p.pt.vy[i];
        Store<float>::st(o + i * p.plane, fmaf(om, feq - f[i], f[i]));
      }
    }
  }
  report(fl, p.err);
}

// ------------------------------------------------- init and read-out (FP64)
// Init: f = f^eq(n, U, T) (Eq. 16) at every site; writes S_0 (at the site)
// and S_{-1} (population i at x - n_i) so that the pull of S_{-1} is f(., 0):
// the read-out kernel always pulls from the buffer the last step read.
template <typename S>
__global__ void __launch_bounds__(128) init_kernel(const __grid_constant__ StepParams<double> p,
                                                   FieldPtrs fd, S* __restrict__ cur,
                                                   S* __restrict__ prev) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (s < p.Nx * p.Ny) {
    int x, y;
    site_of(s, p.Nx, x, y);
    const double n = fd.n[s], ux = fd.ux[s], uy = fd.uy[s], T = fd.T[s];
    const double v2 = ux * ux + uy * uy;
    if (!(v2 < 1.0)) fl |= ERR_LANDAU;
    if (!(n > 0.0)) fl |= ERR_DENSITY;
    if (!(T > 0.0)) fl |= ERR_EOS;
    const double g = 1.0 / sqrt(1.0 - v2);
    Macro<double> md;
    md.n = n;
    md.U0 = g;
    md.dU = g * g * v2 / (g + 1.0);
    md.Ux = g * ux;
    md.Uy = g * uy;
    md.T = T;
    md.zeta = p.sc.mbar / T;
    md.R = ratio64(md.zeta, p.rt64, fl);
    md.dR = md.R - p.sc.Rr;
    md.F = p.sc.mY * md.dR + 3.0 * (T - 1.0);
    md.G = p.sc.mbar * md.dR + 4.0 * (T - 1.0);
    double bn[NJ];
    projections<double>(md, p.sc, bn);
    bn[0] = n * md.R * p.sc.inv_m - p.b0ref;   // minus the reference (b0ref = 0 for FP64)
    for (int i = 0; i < p.Q; ++i) {
      double feq = bn[0] * p.pt.cj[0][i];
      for (int k = 1; k < NJ; ++k) feq = fma(bn[k], p.pt.cj[k][i], feq);
      cur[i * p.plane + (long long)y * p.pitch + x] = (S)feq;
      const int xs = wrap_sub(x, p.pt.dxm[i], p.Nx);
      const int ys = wrap_sub(y, p.pt.dym[i], p.Ny);
      prev[i * p.plane + (long long)ys * p.pitch + xs] = (S)feq;
    }
  }
  report(fl, p.err);
}

// Read-out: pull the state of time t from the buffer the last step read,
// then the FP64 site solve; writes the requested planes.
template <typename S>
__global__ void __launch_bounds__(128) moments_kernel(const __grid_constant__ StepParams<double> p,
                                                      const S* __restrict__ prev, MomentOut mo) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  const long long N = (long long)p.Nx * p.Ny;
  if (s < N) {
    int x, y;
    site_of(s, p.Nx, x, y);
    double m[9];
    for (int k = 0; k < 9; ++k) m[k] = 0.0;
    for (int i = 0; i < p.Q; ++i) {
      const int xs = wrap_sub(x, p.pt.dxm[i], p.Nx);
      const int ys = wrap_sub(y, p.pt.dym[i], p.Ny);
      const double f = (double)prev[i * p.plane + (long long)ys * p.pitch + xs];
      for (int k = 0; k < 9; ++k) m[k] = fma(f, p.pt.mom[k][i], m[k]);
    }
    for (int k = 0; k < 9; ++k) m[k] += p.mref[k];
    const Macro<double> md = solve_site_f64(m, p.sc, p.rt64, fl);
    double* out = mo.out;
    int plane = 0;
    if (mo.mask & RLBM_M_N) out[(plane++) * N + s] = md.n;
    if (mo.mask & RLBM_M_UX) out[(plane++) * N + s] = md.Ux / md.U0;
    if (mo.mask & RLBM_M_UY) out[(plane++) * N + s] = md.Uy / md.U0;
    if (mo.mask & RLBM_M_T) out[(plane++) * N + s] = md.T;
    if (mo.mask & RLBM_M_E) out[(plane++) * N + s] = m[3] - m[4] * (md.Ux / md.U0) - m[5] * (md.Uy / md.U0);
    if (mo.mask & RLBM_M_NVEC)
      for (int k = 0; k < 3; ++k) out[(plane++) * N + s] = m[k];
    if (mo.mask & RLBM_M_TMN)
      for (int k = 3; k < 9; ++k) out[(plane++) * N + s] = m[k];
  }
  report(fl, p.err);
}

}  // namespace rlbm
