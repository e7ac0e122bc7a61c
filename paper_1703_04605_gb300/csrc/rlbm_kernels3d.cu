// Native 3D lattices: the step on an Nx x Ny x Nz periodic lattice with the
// paper's unfolded stencil (Table I orbits with signed n_z), for any six-group
// second-order stencil (Sec. III C-D) and, with the thirty-monomial
// third-order equilibrium (rlbm_o3_3d.h), for any eleven-group stencil.  Per site (Eq. 16-20, 28, 49): pull,
// the 4 + 10 moments N^a, T^ab, the Landau frame T^a_b U^b = e U^a with all
// three velocity components, n = U.N, T from e/n = 3T + m K1/K2(m/T),
// the 14 projections of App. B (corrected), f^eq = n sum_k b_k w_i J_k(p_i)
// and the Anderson-Witting relaxation with weight p_i.U/(p_i^0 tau).
//
// Generic kernels: the population loop runs over a constant table in global
// memory (one 32-entry row per population, read with vector loads; every
// thread of a warp reads the same row), in two passes: the
// first pulls and accumulates the moments, the second pulls again (the values
// are in L1/L2) to relax and store, so no per-thread population array is held
// in registers whatever Q is.  The site solve is FP64; FP64 storage holds f_i,
// FP32 storage d_i = f_i - r_i with FP32 accumulation (as the generic 2D FP32
// kernel).
#include <utility>

#include "rlbm_kernels.cuh"
#include "rlbm_o3_3d.h"

namespace rlbm {
namespace {

struct Macro3 {
  double n, U0, Ux, Uy, Uz, T, R, e;
};

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

template <typename A>
__device__ __forceinline__ const A* table(const Step3Params& p);
template <>
__device__ __forceinline__ const double* table<double>(const Step3Params& p) { return p.tab64; }
template <>
__device__ __forceinline__ const float* table<float>(const Step3Params& p) { return p.tab32; }

__device__ __forceinline__ long long at3(const Step3Params& p, int x, int y, int z) {
  return ((long long)z * p.Ny + y) * p.pitch + x;
}

__device__ __forceinline__ void site3(long long s, const Step3Params& p, int& x, int& y, int& z) {
  x = (int)(s % p.Nx);
  const long long r = s / p.Nx;
  y = (int)(r % p.Ny);
  z = (int)(r / p.Ny);
}

// Four consecutive table entries (16-byte aligned) by vector loads.
__device__ __forceinline__ void ld4(const float* p, float* d) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  d[0] = v.x;
  d[1] = v.y;
  d[2] = v.z;
  d[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double* d) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  d[0] = a.x;
  d[1] = a.y;
  d[2] = b.x;
  d[3] = b.y;
}

__device__ __forceinline__ bool interior3(const Step3Params& p, int x, int y, int z) {
  const int h = p.halo;
  return x >= h && x < p.Nx - h && y >= h && y < p.Ny - h && z >= h && z < p.Nz - h;
}

// Source element of population i for the site (x, y, z): x - n_i, periodic.
__device__ __forceinline__ long long source3(const Step3Params& p, int i, int x, int y, int z) {
  return at3(p, wrap_sub(x, __ldg(p.shift + i), p.Nx), wrap_sub(y, __ldg(p.shift + p.Q + i), p.Ny),
             wrap_sub(z, __ldg(p.shift + 2 * p.Q + i), p.Nz));
}

// T from e/n = y (Eq. 28) by Newton iteration; returns T and R = K1/K2(m/T).
__device__ __forceinline__ void eos3(double y, const SiteConsts& sc, const double* __restrict__ rt64,
                                     double& T, double& R, unsigned& fl) {
  const double mb = sc.mbar;
  if (!(y > mb)) fl |= ERR_EOS;
  // g(T) = 3T + m R(m/T) - y is increasing and convex: Newton from the
  // non-relativistic estimate converges
  T = (y - mb) / (3.0 - 1.5 * (mb * mb) / (y * y));
#pragma unroll 1
  for (int it = 0; it < 40; ++it) {
    const double z = mb / T;
    R = ratio64(z, rt64, fl);
    const double dT = (3.0 * T + mb * R - y) / eos_slope<double>(R, z);
    T -= dT;
    if (!(T > 0.0)) {
      fl |= ERR_EOS;
      T = 1.0;
      break;
    }
    if (fabs(dT) < 1e-15 * T) break;
  }
  R = ratio64(mb / T, rt64, fl);
}

// Moments m = N0 Nx Ny Nz T00 T0x T0y T0z Txx Txy Txz Tyy Tyz Tzz -> n, U, T.
// Landau frame: Newton on v = U/U^0 for F(v) = T^0i - T^ij v_j - e v_i = 0
// with e = T^00 - T^0j v_j (the spatial rows of T^a_b U^b = e U^a).
__device__ __forceinline__ Macro3 solve3(const double* m, const SiteConsts& sc, const double* __restrict__ rt64,
                                         unsigned& fl) {
  const double T00 = m[4];
  const double T0[3] = {m[5], m[6], m[7]};
  const double Tij[3][3] = {{m[8], m[9], m[10]}, {m[9], m[11], m[12]}, {m[10], m[12], m[13]}};
  const double den = T00 + (m[8] + m[11] + m[13]) / 3.0;
  double v[3] = {T0[0] / den, T0[1] / den, T0[2] / den};
#pragma unroll 1
  for (int it = 0; it < 20; ++it) {
    const double e = T00 - T0[0] * v[0] - T0[1] * v[1] - T0[2] * v[2];
    double F[3], J[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      F[a] = T0[a] - Tij[a][0] * v[0] - Tij[a][1] * v[1] - Tij[a][2] * v[2] - e * v[a];
#pragma unroll
      for (int b = 0; b < 3; ++b) J[a][b] = -Tij[a][b] - (a == b ? e : 0.0) + v[a] * T0[b];
    }
    // J dv = F by Cramer's rule
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const double id = 1.0 / det;
    const double d0 = (F[0] * c00 + J[0][1] * (F[2] * J[1][2] - F[1] * J[2][2]) +
                       J[0][2] * (F[1] * J[2][1] - F[2] * J[1][1])) * id;
    const double d1 = (J[0][0] * (F[1] * J[2][2] - F[2] * J[1][2]) + F[0] * c01 +
                       J[0][2] * (F[2] * J[1][0] - F[1] * J[2][0])) * id;
    const double d2 = (J[0][0] * (F[2] * J[1][1] - F[1] * J[2][1]) + J[0][1] * (F[1] * J[2][0] - F[2] * J[1][0]) +
                       F[0] * c02) * id;
    v[0] -= d0;
    v[1] -= d1;
    v[2] -= d2;
    if (fabs(d0) + fabs(d1) + fabs(d2) < 1e-15) break;
  }
  Macro3 o;
  const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  if (!(v2 < 1.0)) fl |= ERR_LANDAU;
  const double g = 1.0 / sqrt(1.0 - v2);
  o.U0 = g;
  o.Ux = g * v[0];
  o.Uy = g * v[1];
  o.Uz = g * v[2];
  o.e = T00 - T0[0] * v[0] - T0[1] * v[1] - T0[2] * v[2];
  o.n = g * (m[0] - v[0] * m[1] - v[1] * m[2] - v[2] * m[3]);
  if (!(o.n > 0.0)) fl |= ERR_DENSITY;
  eos3(o.e / o.n, sc, rt64, o.T, o.R, fl);
  return o;
}

// The same solve for FP32 storage: the Landau and EOS Newton iterations in
// FP32, then one Newton step of each with the residual formed in FP64 (the
// Landau Jacobian of the last FP32 iterate; the FP64 R(zeta) table), which
// squares an error already near FP32 rounding.  About a tenth of the FP64
// operations of solve3, the pipe that bounds the FP32 kernel otherwise.
__device__ __forceinline__ Macro3 solve3_mixed(const double* m, const SiteConsts& sc,
                                               const double* __restrict__ rt64, const float* __restrict__ rt32,
                                               unsigned& fl) {
  float mf[14];
#pragma unroll
  for (int k = 0; k < 14; ++k) mf[k] = (float)m[k];
  const float T00 = mf[4];
  const float T0[3] = {mf[5], mf[6], mf[7]};
  const float Tij[3][3] = {{mf[8], mf[9], mf[10]}, {mf[9], mf[11], mf[12]}, {mf[10], mf[12], mf[13]}};
  const float den = T00 + (mf[8] + mf[11] + mf[13]) * (1.0f / 3.0f);
  float v[3] = {T0[0] / den, T0[1] / den, T0[2] / den};
  float J[3][3];
#pragma unroll 1
  for (int it = 0; it < 12; ++it) {
    const float e = T00 - T0[0] * v[0] - T0[1] * v[1] - T0[2] * v[2];
    float F[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      F[a] = T0[a] - Tij[a][0] * v[0] - Tij[a][1] * v[1] - Tij[a][2] * v[2] - e * v[a];
#pragma unroll
      for (int b = 0; b < 3; ++b) J[a][b] = -Tij[a][b] - (a == b ? e : 0.0f) + v[a] * T0[b];
    }
    const float c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const float c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const float c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const float id = 1.0f / (J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02);
    const float d0 = (F[0] * c00 + J[0][1] * (F[2] * J[1][2] - F[1] * J[2][2]) +
                      J[0][2] * (F[1] * J[2][1] - F[2] * J[1][1])) * id;
    const float d1 = (J[0][0] * (F[1] * J[2][2] - F[2] * J[1][2]) + F[0] * c01 +
                      J[0][2] * (F[2] * J[1][0] - F[1] * J[2][0])) * id;
    const float d2 = (J[0][0] * (F[2] * J[1][1] - F[1] * J[2][1]) + J[0][1] * (F[1] * J[2][0] - F[2] * J[1][0]) +
                      F[0] * c02) * id;
    v[0] -= d0;
    v[1] -= d1;
    v[2] -= d2;
    if (fabsf(d0) + fabsf(d1) + fabsf(d2) < 1e-7f) break;
  }
  // one Newton step with the FP64 residual
  double vd[3] = {v[0], v[1], v[2]};
  {
    const double e = m[4] - m[5] * vd[0] - m[6] * vd[1] - m[7] * vd[2];
    const double Td[3][3] = {{m[8], m[9], m[10]}, {m[9], m[11], m[12]}, {m[10], m[12], m[13]}};
    double F[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      F[a] = m[5 + a] - Td[a][0] * vd[0] - Td[a][1] * vd[1] - Td[a][2] * vd[2] - e * vd[a];
    const double c00 = (double)J[1][1] * J[2][2] - (double)J[1][2] * J[2][1];
    const double c01 = (double)J[1][2] * J[2][0] - (double)J[1][0] * J[2][2];
    const double c02 = (double)J[1][0] * J[2][1] - (double)J[1][1] * J[2][0];
    const double id = 1.0 / (J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02);
    vd[0] -= (F[0] * c00 + J[0][1] * (F[2] * J[1][2] - F[1] * J[2][2]) + J[0][2] * (F[1] * J[2][1] - F[2] * J[1][1])) * id;
    vd[1] -= (J[0][0] * (F[1] * J[2][2] - F[2] * J[1][2]) + F[0] * c01 + J[0][2] * (F[2] * J[1][0] - F[1] * J[2][0])) * id;
    vd[2] -= (J[0][0] * (F[2] * J[1][1] - F[1] * J[2][1]) + J[0][1] * (F[1] * J[2][0] - F[2] * J[1][0]) + F[0] * c02) * id;
  }
  Macro3 o;
  const double v2 = vd[0] * vd[0] + vd[1] * vd[1] + vd[2] * vd[2];
  if (!(v2 < 1.0)) fl |= ERR_LANDAU;
  const double g = 1.0 / sqrt(1.0 - v2);
  o.U0 = g;
  o.Ux = g * vd[0];
  o.Uy = g * vd[1];
  o.Uz = g * vd[2];
  o.e = m[4] - m[5] * vd[0] - m[6] * vd[1] - m[7] * vd[2];
  o.n = g * (m[0] - vd[0] * m[1] - vd[1] * m[2] - vd[2] * m[3]);
  if (!(o.n > 0.0)) fl |= ERR_DENSITY;
  // EOS: FP32 Newton with the FP32 table, one FP64 step, R at the final T
  const double y = o.e / o.n;
  const double mb = sc.mbar;
  if (!(y > mb)) fl |= ERR_EOS;
  float T = (float)((y - mb) / (3.0 - 1.5 * (mb * mb) / (y * y)));
  const float mbf = (float)mb, yf = (float)y;
  float slope = 3.0f;
#pragma unroll 1
  for (int it = 0; it < 20; ++it) {
    if (!(T > 0.0f)) {
      fl |= ERR_EOS;
      T = 1.0f;
      break;
    }
    const float z = mbf / T;
    const float R = ratio32(z, rt32, fl);
    slope = eos_slope<float>(R, z);
    const float dT = (3.0f * T + mbf * R - yf) / slope;
    T -= dT;
    if (fabsf(dT) < 3e-7f * T) break;
  }
  double Td = T;
  Td -= (3.0 * Td + mb * ratio64(mb / Td, rt64, fl) - y) / (double)slope;
  if (!(Td > 0.0)) {
    fl |= ERR_EOS;
    Td = 1.0;
  }
  o.T = Td;
  o.R = ratio64(mb / Td, rt64, fl);
  return o;
}

// n b^(k) of App. B (corrected) for the 14 polynomials, table order.
__device__ __forceinline__ void projections3(const Macro3& o, const SiteConsts& sc, double* bn) {
  const double n = o.n, U0 = o.U0, Ux = o.Ux, Uy = o.Uy, Uz = o.Uz, R = o.R, T = o.T;
  const double mr32 = sc.mbar * R + 4.0 * T;      // mbar K3/K2(zeta)
  bn[0] = n * R * sc.inv_m;
  bn[1] = n * (U0 - sc.k21 * R) * sc.iA;
  bn[2] = n * Ux * sc.iB;
  bn[3] = n * Uy * sc.iB;
  bn[4] = n * Uz * sc.iB;
  bn[5] = n * (mr32 * U0 * U0 + sc.cb00_1 * U0 + R * sc.Y - T) * sc.i3C;
  const double h = n * (mr32 * U0 - sc.mk32) * sc.iD;
  bn[6] = h * Ux;
  bn[7] = h * Uy;
  bn[8] = h * Uz;
  const double nm = n * mr32;
  bn[9] = nm * (Uy * Uy - Uz * Uz) * sc.i2E;
  bn[10] = nm * (-2.0 * Ux * Ux + Uy * Uy + Uz * Uz) * sc.i23E;
  bn[11] = nm * Ux * Uz * sc.iE;
  bn[12] = nm * Uy * Uz * sc.iE;
  bn[13] = nm * Ux * Uy * sc.iE;
}

// Pull pass: the 14 moments of the pre-collision populations at a site.
template <typename S>
__device__ __forceinline__ void moments3(const Step3Params& p, const S* __restrict__ fin, int x, int y, int z,
                                         double* md) {
  const S* tab = table<S>(p);
  S mm[14];
#pragma unroll
  for (int k = 0; k < 14; ++k) mm[k] = S(0);
  const bool in = interior3(p, x, y, z);
  const long long here = at3(p, x, y, z);
#pragma unroll 4
  for (int i = 0; i < p.Q; ++i) {
    const long long src = in ? here + __ldg(p.off + i) : source3(p, i, x, y, z);
    const S f = __ldg(fin + (long long)i * p.plane + src);
    S c[16];
    const S* row = tab + (long long)i * kRow3;
#pragma unroll
    for (int j = 0; j < 4; ++j) ld4(row + 4 * j, c + 4 * j);
#pragma unroll
    for (int k = 0; k < 14; ++k) mm[k] = fma_t(f, c[k], mm[k]);
  }
#pragma unroll
  for (int k = 0; k < 14; ++k) md[k] = (double)mm[k] + p.mref[k];
}

template <typename S>
__global__ void __launch_bounds__(128) step3d_kernel(const __grid_constant__ Step3Params p,
                                                     const S* __restrict__ fin, S* __restrict__ fout) {
  const long long nsite = (long long)p.Nx * p.Ny * p.Nz;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (s < nsite) {
    int x, y, z;
    site3(s, p, x, y, z);
    double md[14];
    moments3<S>(p, fin, x, y, z, md);
    Macro3 o;
    if constexpr (sizeof(S) == 4) o = solve3_mixed(md, p.sc, p.rt64, p.rt32, fl);
    else o = solve3(md, p.sc, p.rt64, fl);
    double bn[14];
    projections3(o, p.sc, bn);
    bn[0] -= p.b0ref;                                  // f^eq - r_i (r_i = 0 for FP64 storage)
    S b[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) b[k] = (S)bn[k];
    const S a0 = (S)(o.U0 * p.inv_tau), ax = (S)(o.Ux * p.inv_tau), ay = (S)(o.Uy * p.inv_tau),
            az = (S)(o.Uz * p.inv_tau);
    const S* tab = table<S>(p);
    const bool in = interior3(p, x, y, z);
    const long long here = at3(p, x, y, z);
    S* out = fout + here;
#pragma unroll 4
    for (int i = 0; i < p.Q; ++i) {
      const long long src = in ? here + __ldg(p.off + i) : source3(p, i, x, y, z);
      const S f = __ldg(fin + (long long)i * p.plane + src);
      S c[20];                                         // row entries 12..31
      const S* row = tab + (long long)i * kRow3 + 12;
#pragma unroll
      for (int j = 0; j < 5; ++j) ld4(row + 4 * j, c + 4 * j);
      S feq = S(0);
#pragma unroll
      for (int k = 0; k < 14; ++k) feq = fma_t(b[k], c[2 + k], feq);
      // weight p_i.U/(p_i^0 tau) = (U0 - v_i . U)/tau
      const S om = a0 - ax * c[16] - ay * c[17] - az * c[18];
      __stcs(out + (long long)i * p.plane, fma_t(om, feq - f, f));
    }
  }
  report(fl, p.err);
}

// f = f^eq(n, U, T) (Eq. 16): S_0 at the site and S_{-1} at x - n_i, so that
// the pull of S_{-1} is f(., 0) (same convention as the 2D init).
template <typename S>
__global__ void __launch_bounds__(128) init3d_kernel(const __grid_constant__ Step3Params p, Field3Ptrs fd,
                                                     S* __restrict__ cur, S* __restrict__ prev) {
  const long long nsite = (long long)p.Nx * p.Ny * p.Nz;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (s < nsite) {
    int x, y, z;
    site3(s, p, x, y, z);
    const double ux = fd.ux[s], uy = fd.uy[s], uz = fd.uz[s];
    const double g = 1.0 / sqrt(1.0 - (ux * ux + uy * uy + uz * uz));
    Macro3 o;
    o.n = fd.n[s];
    o.T = fd.T[s];
    o.U0 = g;
    o.Ux = g * ux;
    o.Uy = g * uy;
    o.Uz = g * uz;
    o.R = ratio64(p.sc.mbar / o.T, p.rt64, fl);
    double bn[14];
    projections3(o, p.sc, bn);
    bn[0] -= p.b0ref;
    const long long here = at3(p, x, y, z);
#pragma unroll 1
    for (int i = 0; i < p.Q; ++i) {
      double feq = 0.0;
#pragma unroll
      for (int k = 0; k < 14; ++k) feq = fma(bn[k], __ldg(p.tab64 + (long long)i * kRow3 + 14 + k), feq);
      cur[(long long)i * p.plane + here] = (S)feq;
      prev[(long long)i * p.plane + source3(p, i, x, y, z)] = (S)feq;
    }
  }
  report(fl, p.err);
}

// Read-out of the pre-collision state: the pull of prev, FP64 solve.
// Planes (each Nx Ny Nz doubles, x fastest) in mask order: n, u_x, u_y, T, e,
// N^a (4), T^ab (10: 00 0x 0y 0z xx xy xz yy yz zz), u_z.
template <typename S>
__global__ void __launch_bounds__(128) moments3d_kernel(const __grid_constant__ Step3Params p,
                                                        const S* __restrict__ prev, MomentOut mo) {
  const long long nsite = (long long)p.Nx * p.Ny * p.Nz;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (s < nsite) {
    int x, y, z;
    site3(s, p, x, y, z);
    double md[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) md[k] = 0.0;
    const double* tab = p.tab64;
#pragma unroll 1
    for (int i = 0; i < p.Q; ++i) {
      const double f = (double)prev[(long long)i * p.plane + source3(p, i, x, y, z)];
#pragma unroll
      for (int k = 0; k < 14; ++k) md[k] = fma(f, __ldg(tab + (long long)i * kRow3 + k), md[k]);
    }
#pragma unroll
    for (int k = 0; k < 14; ++k) md[k] += p.mref[k];
    const Macro3 o = solve3(md, p.sc, p.rt64, fl);
    double* out = mo.out;
    long long plane = 0;
    if (mo.mask & RLBM_M_N) out[(plane++) * nsite + s] = o.n;
    if (mo.mask & RLBM_M_UX) out[(plane++) * nsite + s] = o.Ux / o.U0;
    if (mo.mask & RLBM_M_UY) out[(plane++) * nsite + s] = o.Uy / o.U0;
    if (mo.mask & RLBM_M_T) out[(plane++) * nsite + s] = o.T;
    if (mo.mask & RLBM_M_E) out[(plane++) * nsite + s] = o.e;
    if (mo.mask & RLBM_M_NVEC)
      for (int k = 0; k < 4; ++k) out[(plane++) * nsite + s] = md[k];
    if (mo.mask & RLBM_M_TMN)
      for (int k = 4; k < 14; ++k) out[(plane++) * nsite + s] = md[k];
    if (mo.mask & RLBM_M_UZ) out[(plane++) * nsite + s] = o.Uz / o.U0;
  }
  report(fl, p.err);
}

// ------------------------------------------------------------ third order
// Site quantities of the third-order equilibrium (see rlbm_o3_3d.h and the
// 2D form in rlbm_o3.cuh): with h = m R + 4T, A3 = m^2 + 6 T h, B3 = -T h,
// the deviations from rest at T_R of the moments (per unit density) of
// t^a p^s1 ... p^sr are
//   r = 0:  a = 0: dR/m           a = 1: dU - c dR/m
//   r = 1:  a = 0: U_s            a = 1: U_s (h U0 - c)
//   r = 2:  a = 0: h U_s U_s' + d_ss' dT
//           a = 1: (A3 U0 - c h) U_s U_s' + d_ss' (T (h U0 - c) - (h_r - c))
//   r = 3:  A3 U_s U_s' U_s'' + T h (d_ss' U_s'' + d_ss'' U_s' + d_s's'' U_s)
// (Eq. 4-6, 28-29, 43-44; eta^ab = -delta_ab on the spatial indices).
template <typename R>
struct O3Site3 {
  R n, U[4], dU, dR, dT, m, c, h, Th, Am, hU, sdev, q;
};

template <int A, int I, int J, int K, typename R>
__device__ __forceinline__ R o3dev3(const O3Site3<R>& s) {
  constexpr int r = I + J + K;
  constexpr int i1 = I > 0 ? 1 : (J > 0 ? 2 : 3);
  constexpr int i2 = I > 1 ? 1 : (I + J > 1 ? 2 : 3);
  constexpr int i3 = I > 2 ? 1 : (I + J > 2 ? 2 : 3);
  if constexpr (r == 0) {
    return A == 0 ? s.n * s.dR / s.m : s.n * (s.dU - s.c * s.dR / s.m);
  } else if constexpr (r == 1) {
    return A == 0 ? s.n * s.U[i1] : s.n * s.U[i1] * s.hU;
  } else if constexpr (r == 2) {
    const R uu = s.U[i1] * s.U[i2];
    if constexpr (A == 0) return s.n * (s.h * uu + (i1 == i2 ? s.dT : R(0)));
    else return s.n * (s.q * uu + (i1 == i2 ? s.sdev : R(0)));
  } else {
    R v = s.Am * s.U[i1] * s.U[i2] * s.U[i3];
    if constexpr (i1 == i2) v += s.Th * s.U[i3];
    if constexpr (i1 == i3) v += s.Th * s.U[i2];
    if constexpr (i2 == i3) v += s.Th * s.U[i1];
    return s.n * v;
  }
}

template <typename R, int... L>
__device__ __forceinline__ void o3_dev3_all(std::integer_sequence<int, L...>, const O3Site3<R>& s, R* e) {
  ((e[L] = o3dev3<kO3Exp3.e[L][0], kO3Exp3.e[L][1], kO3Exp3.e[L][2], kO3Exp3.e[L][3], R>(s)), ...);
}

// e_l = n dmu_l of the thirty monomials from the FP64 site macros.
template <typename R>
__device__ __forceinline__ void o3_deviations3(const Macro3& o, double Rr, double mbar, double c, R* e) {
  O3Site3<R> s;
  const double Ua2 = o.Ux * o.Ux + o.Uy * o.Uy + o.Uz * o.Uz;
  const double dU = Ua2 / (o.U0 + 1.0);                   // U0 - 1 without cancellation
  const double dT = o.T - 1.0;
  const double h = mbar * o.R + 4.0 * o.T;
  const double dR = o.R - Rr;
  const double dh = mbar * dR + 4.0 * dT;
  const double Th = o.T * h;
  const double Am = mbar * mbar + 6.0 * Th;
  const double hU = h * o.U0 - c;
  s.n = (R)o.n;
  s.U[0] = (R)o.U0;
  s.U[1] = (R)o.Ux;
  s.U[2] = (R)o.Uy;
  s.U[3] = (R)o.Uz;
  s.dU = (R)dU;
  s.dR = (R)dR;
  s.dT = (R)dT;
  s.m = (R)mbar;
  s.c = (R)c;
  s.h = (R)h;
  s.Th = (R)Th;
  s.Am = (R)Am;
  s.hU = (R)hU;
  s.sdev = (R)(dT * hU + h * dU + dh);                    // T (h U0 - c) - (h_r - c)
  s.q = (R)(Am * o.U0 - c * h);
  o3_dev3_all<R>(std::make_integer_sequence<int, kO3Mono3>{}, s, e);
}

template <typename A>
__device__ __forceinline__ const A* wtab(const Step3O3Params& p);
template <>
__device__ __forceinline__ const double* wtab<double>(const Step3O3Params& p) { return p.w64; }
template <>
__device__ __forceinline__ const float* wtab<float>(const Step3O3Params& p) { return p.w32; }

// Third-order step (generic over the stencil): pull and moments as
// step3d_kernel, the same site solve, then f^eq_i - nref wr_i =
// n_d wr_i + sum_l e_l W_il and the Anderson-Witting relaxation.
template <typename S>
__global__ void __launch_bounds__(128) step3d_o3_kernel(const __grid_constant__ Step3O3Params q,
                                                        const S* __restrict__ fin, S* __restrict__ fout) {
  const Step3Params& p = q.b;
  const long long nsite = (long long)p.Nx * p.Ny * p.Nz;
  const long long sidx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (sidx < nsite) {
    int x, y, z;
    site3(sidx, p, x, y, z);
    double md[14];
    moments3<S>(p, fin, x, y, z, md);
    Macro3 o;
    if constexpr (sizeof(S) == 4) o = solve3_mixed(md, p.sc, p.rt64, p.rt32, fl);
    else o = solve3(md, p.sc, p.rt64, fl);
    S e[kO3Mono3];
    o3_deviations3<S>(o, p.sc.Rr, p.sc.mbar, q.c, e);
    const S dn = (S)(o.n - p.nref);
    const S a0 = (S)(o.U0 * p.inv_tau), ax = (S)(o.Ux * p.inv_tau), ay = (S)(o.Uy * p.inv_tau),
            az = (S)(o.Uz * p.inv_tau);
    const S* tab = table<S>(p);
    const S* wt = wtab<S>(q);
    const bool in = interior3(p, x, y, z);
    const long long here = at3(p, x, y, z);
    S* out = fout + here;
#pragma unroll 2
    for (int i = 0; i < p.Q; ++i) {
      const long long src = in ? here + __ldg(p.off + i) : source3(p, i, x, y, z);
      const S f = __ldg(fin + (long long)i * p.plane + src);
      S c[4];
      ld4(tab + (long long)i * kRow3 + 28, c);               // p^a/p^0
      S w[32];
      const S* row = wt + (long long)i * kRowW3;
#pragma unroll
      for (int j = 0; j < 8; ++j) ld4(row + 4 * j, w + 4 * j);
      S feq = dn * __ldg(tab + (long long)i * kRow3 + 14);
#pragma unroll
      for (int l = 0; l < kO3Mono3; ++l) feq = fma_t(e[l], w[l], feq);
      const S om = a0 - ax * c[0] - ay * c[1] - az * c[2];
      __stcs(out + (long long)i * p.plane, fma_t(om, feq - f, f));
    }
  }
  report(fl, p.err);
}

// f = f^eq(n, U, T) at third order: S_0 at the site, S_{-1} at x - n_i.
template <typename S>
__global__ void __launch_bounds__(128) init3d_o3_kernel(const __grid_constant__ Step3O3Params q, Field3Ptrs fd,
                                                        S* __restrict__ cur, S* __restrict__ prev) {
  const Step3Params& p = q.b;
  const long long nsite = (long long)p.Nx * p.Ny * p.Nz;
  const long long sidx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (sidx < nsite) {
    int x, y, z;
    site3(sidx, p, x, y, z);
    const double ux = fd.ux[sidx], uy = fd.uy[sidx], uz = fd.uz[sidx];
    const double v2 = ux * ux + uy * uy + uz * uz;
    if (!(v2 < 1.0)) fl |= ERR_LANDAU;
    const double g = 1.0 / sqrt(1.0 - v2);
    Macro3 o;
    o.n = fd.n[sidx];
    o.T = fd.T[sidx];
    if (!(o.n > 0.0)) fl |= ERR_DENSITY;
    if (!(o.T > 0.0)) fl |= ERR_EOS;
    o.U0 = g;
    o.Ux = g * ux;
    o.Uy = g * uy;
    o.Uz = g * uz;
    o.R = ratio64(p.sc.mbar / o.T, p.rt64, fl);
    double e[kO3Mono3];
    o3_deviations3<double>(o, p.sc.Rr, p.sc.mbar, q.c, e);
    const double dn = o.n - p.nref;
    const long long here = at3(p, x, y, z);
#pragma unroll 1
    for (int i = 0; i < p.Q; ++i) {
      double feq = dn * __ldg(p.tab64 + (long long)i * kRow3 + 14);
#pragma unroll
      for (int l = 0; l < kO3Mono3; ++l) feq = fma(e[l], __ldg(q.w64 + (long long)i * kRowW3 + l), feq);
      cur[(long long)i * p.plane + here] = (S)feq;
      prev[(long long)i * p.plane + source3(p, i, x, y, z)] = (S)feq;
    }
  }
  report(fl, p.err);
}

unsigned grid3(const Step3Params& p) {
  return (unsigned)(((long long)p.Nx * p.Ny * p.Nz + 127) / 128);
}

}  // namespace

cudaError_t launch_step3d(rlbm_dtype dt, const Step3Params& p, const void* fin, void* fout, cudaStream_t s) {
  if (dt == RLBM_F64)
    step3d_kernel<double><<<grid3(p), 128, 0, s>>>(p, static_cast<const double*>(fin), static_cast<double*>(fout));
  else
    step3d_kernel<float><<<grid3(p), 128, 0, s>>>(p, static_cast<const float*>(fin), static_cast<float*>(fout));
  return cudaGetLastError();
}

cudaError_t launch_init3d(rlbm_dtype dt, const Step3Params& p, Field3Ptrs f, void* cur, void* prev,
                          cudaStream_t s) {
  if (dt == RLBM_F64)
    init3d_kernel<double><<<grid3(p), 128, 0, s>>>(p, f, static_cast<double*>(cur), static_cast<double*>(prev));
  else
    init3d_kernel<float><<<grid3(p), 128, 0, s>>>(p, f, static_cast<float*>(cur), static_cast<float*>(prev));
  return cudaGetLastError();
}

cudaError_t launch_moments3d(rlbm_dtype dt, const Step3Params& p, const void* prev, MomentOut o,
                             cudaStream_t s) {
  if (dt == RLBM_F64)
    moments3d_kernel<double><<<grid3(p), 128, 0, s>>>(p, static_cast<const double*>(prev), o);
  else
    moments3d_kernel<float><<<grid3(p), 128, 0, s>>>(p, static_cast<const float*>(prev), o);
  return cudaGetLastError();
}

cudaError_t launch_step3d_o3(rlbm_dtype dt, const Step3O3Params& p, const void* fin, void* fout, cudaStream_t s) {
  if (dt == RLBM_F64)
    step3d_o3_kernel<double><<<grid3(p.b), 128, 0, s>>>(p, static_cast<const double*>(fin), static_cast<double*>(fout));
  else
    step3d_o3_kernel<float><<<grid3(p.b), 128, 0, s>>>(p, static_cast<const float*>(fin), static_cast<float*>(fout));
  return cudaGetLastError();
}

cudaError_t launch_init3d_o3(rlbm_dtype dt, const Step3O3Params& p, Field3Ptrs f, void* cur, void* prev,
                             cudaStream_t s) {
  if (dt == RLBM_F64)
    init3d_o3_kernel<double><<<grid3(p.b), 128, 0, s>>>(p, f, static_cast<double*>(cur), static_cast<double*>(prev));
  else
    init3d_o3_kernel<float><<<grid3(p.b), 128, 0, s>>>(p, f, static_cast<float*>(cur), static_cast<float*>(prev));
  return cudaGetLastError();
}

}  // namespace rlbm
