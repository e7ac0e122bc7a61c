// Stencil-specialised FP32 step for 3D lattices (the unfolded stencil known at
// compile time).  Same step and split arithmetic as the 2D kernel of
// rlbm_fused.cuh (Eq. 16-20, 28, 49): stored values d_i = f_i - r_i; group
// sums with exact integer weights; group constants as hi/lo FP32 pairs; FP32
// Landau frame (Newton on the three velocity components) and FP32 EOS
// iterations with one FP64 Newton step of the EOS.
//
// Equilibrium per group g (|n|^2 constant in a group, so the n_z^2 term of the
// App. A polynomials folds into the others):
//   f^eq_i - r_i = alpha + beta . n + q_xx n_x^2 + q_yy n_y^2 + q_xy n_x n_y
//                  + q_xz n_x n_z + q_yz n_y n_z.
// Two passes over the populations: pull and sum (keeping each value in shared
// memory), then relax and store, so only the group sums and coefficients live
// in registers.
#include "rlbm_fused.cuh"

namespace rlbm {
namespace {

// element index of the pulled value in its plane (32-bit: a plane holds
// fewer than 2^32 elements, checked when the lattice is created)
template <class D, int I>
__device__ __forceinline__ unsigned f3_src(const Fused3Params& p, int x, int y, int z) {
  constexpr int DX = D::U.nx[I], DY = D::U.ny[I], DZ = D::U.nz[I];
  return (unsigned)wrap_c<DZ>(z, p.Nz) * (unsigned)p.zstride + (unsigned)wrap_c<DY>(y, p.Ny) * (unsigned)p.pitch +
         (unsigned)wrap_c<DX>(x, p.Nx);
}

// group sums: 1, n_x, n_y, n_z, n_x^2, n_y^2, n_z^2, n_x n_y, n_x n_z, n_y n_z
template <class D, int I>
__device__ __forceinline__ void f3_acc(const Fused3Params& p, const float* __restrict__ fin, int x, int y, int z,
                                       float (&s)[6][10], float* __restrict__ keep) {
  constexpr int g = D::U.grp[I], nx = D::U.nx[I], ny = D::U.ny[I], nz = D::U.nz[I];
  const float v = __ldg(fin + f3_src<D, I>(p, x, y, z) + (size_t)(unsigned)p.plane * I);
  keep[I * 128] = v;
  s[g][0] += v;
  if constexpr (nx != 0) s[g][1] = fmaf((float)nx, v, s[g][1]);
  if constexpr (ny != 0) s[g][2] = fmaf((float)ny, v, s[g][2]);
  if constexpr (nz != 0) s[g][3] = fmaf((float)nz, v, s[g][3]);
  if constexpr (nx != 0) s[g][4] = fmaf((float)(nx * nx), v, s[g][4]);
  if constexpr (ny != 0) s[g][5] = fmaf((float)(ny * ny), v, s[g][5]);
  if constexpr (nz != 0) s[g][6] = fmaf((float)(nz * nz), v, s[g][6]);
  if constexpr (nx != 0 && ny != 0) s[g][7] = fmaf((float)(nx * ny), v, s[g][7]);
  if constexpr (nx != 0 && nz != 0) s[g][8] = fmaf((float)(nx * nz), v, s[g][8]);
  if constexpr (ny != 0 && nz != 0) s[g][9] = fmaf((float)(ny * nz), v, s[g][9]);
}

// coefficients c[g]: alpha, beta_x, beta_y, beta_z, q_xx, q_yy, q_xy, q_xz, q_yz
template <class D, int I>
__device__ __forceinline__ void f3_collide(const Fused3Params& p, const float* __restrict__ keep,
                                           const float (&c)[6][9], float a0, float ax, float ay, float az,
                                           float* __restrict__ out) {
  constexpr int g = D::U.grp[I], nx = D::U.nx[I], ny = D::U.ny[I], nz = D::U.nz[I];
  const float v = keep[I * 128];
  float e = c[g][0];
  if constexpr (nx != 0) e = fmaf((float)nx, c[g][1], e);
  if constexpr (ny != 0) e = fmaf((float)ny, c[g][2], e);
  if constexpr (nz != 0) e = fmaf((float)nz, c[g][3], e);
  if constexpr (nx != 0) e = fmaf((float)(nx * nx), c[g][4], e);
  if constexpr (ny != 0) e = fmaf((float)(ny * ny), c[g][5], e);
  if constexpr (nx != 0 && ny != 0) e = fmaf((float)(nx * ny), c[g][6], e);
  if constexpr (nx != 0 && nz != 0) e = fmaf((float)(nx * nz), c[g][7], e);
  if constexpr (ny != 0 && nz != 0) e = fmaf((float)(ny * nz), c[g][8], e);
  // weight p_i.U/(p_i^0 tau) = (U0 - v0 n_i.U)/tau
  float om = a0;
  if constexpr (nx != 0) om = fmaf(-(float)nx, ax, om);
  if constexpr (ny != 0) om = fmaf(-(float)ny, ay, om);
  if constexpr (nz != 0) om = fmaf(-(float)nz, az, om);
  __stcs(out + (size_t)(unsigned)p.plane * I, fmaf(om, e - v, v));
}

template <class D, int... Is>
__device__ __forceinline__ void f3_acc_all(std::integer_sequence<int, Is...>, const Fused3Params& p,
                                           const float* __restrict__ fin, int x, int y, int z, float (&s)[6][10],
                                           float* __restrict__ keep) {
  (f3_acc<D, Is>(p, fin, x, y, z, s, keep), ...);
}

template <class D, int... Is>
__device__ __forceinline__ void f3_collide_all(std::integer_sequence<int, Is...>, const Fused3Params& p,
                                               const float* __restrict__ keep, const float (&c)[6][9], float a0,
                                               float ax, float ay, float az, float* __restrict__ out) {
  (f3_collide<D, Is>(p, keep, c, a0, ax, ay, az, out), ...);
}

template <class D>
__global__ void __launch_bounds__(128, 4) fused3d_kernel(const __grid_constant__ Fused3Params p,
                                                         const float* __restrict__ fin, float* __restrict__ fout) {
  constexpr int Q = D::Q;
  using Seq = std::make_integer_sequence<int, Q>;
  // Nx Ny Nz < 2^31 (checked at creation): 32-bit site arithmetic
  const int nsite = p.Nx * p.Ny * p.Nz;
  const int site = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  unsigned fl = 0;
  // each thread keeps its pulled populations here between the two passes
  // (column threadIdx.x of a [Q][128] array: consecutive threads, banks)
  extern __shared__ float keep_all[];
  float* keep = keep_all + threadIdx.x;
  if (site < nsite) {
    const int r = site / p.Nx;
    const int x = site - r * p.Nx;
    const int z = r / p.Ny;
    const int y = r - z * p.Ny;
    float s[6][10];
#pragma unroll
    for (int g = 0; g < 6; ++g)
#pragma unroll
      for (int k = 0; k < 10; ++k) s[g][k] = 0.0f;
    f3_acc_all<D>(Seq{}, p, fin, x, y, z, s, keep);
    // deviation moments N0 Nx Ny Nz T00 T0x T0y T0z Txx Txy Txz Tyy Tyz Tzz
    float M[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) M[k] = 0.0f;
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      const HL* gm = p.gm[g];   // P0, P0^2, Pv, P0 Pv, Pv^2
      M[0] = hl_fma(gm[0], s[g][0], M[0]);
      M[4] = hl_fma(gm[1], s[g][0], M[4]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        M[1 + a] = hl_fma(gm[2], s[g][1 + a], M[1 + a]);
        M[5 + a] = hl_fma(gm[3], s[g][1 + a], M[5 + a]);
      }
      M[8] = hl_fma(gm[4], s[g][4], M[8]);     // xx
      M[9] = hl_fma(gm[4], s[g][7], M[9]);     // xy
      M[10] = hl_fma(gm[4], s[g][8], M[10]);   // xz
      M[11] = hl_fma(gm[4], s[g][5], M[11]);   // yy
      M[12] = hl_fma(gm[4], s[g][9], M[12]);   // yz
      M[13] = hl_fma(gm[4], s[g][6], M[13]);   // zz
    }
    // Landau frame: FP32 Newton on the full moments
    float Mf[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) Mf[k] = p.mref[k].hi + (p.mref[k].lo + M[k]);
    const float T00 = Mf[4];
    const float T0[3] = {Mf[5], Mf[6], Mf[7]};
    const float Tij[3][3] = {{Mf[8], Mf[9], Mf[10]}, {Mf[9], Mf[11], Mf[12]}, {Mf[10], Mf[12], Mf[13]}};
    float v[3];
    {
      const float iden = __fdividef(1.0f, T00 + (Mf[8] + Mf[11] + Mf[13]) * (1.0f / 3.0f));
      v[0] = T0[0] * iden;
      v[1] = T0[1] * iden;
      v[2] = T0[2] * iden;
    }
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
      const float e = T00 - T0[0] * v[0] - T0[1] * v[1] - T0[2] * v[2];
      float F[3], J[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        F[a] = T0[a] - Tij[a][0] * v[0] - Tij[a][1] * v[1] - Tij[a][2] * v[2] - e * v[a];
#pragma unroll
        for (int b = 0; b < 3; ++b) J[a][b] = -Tij[a][b] - (a == b ? e : 0.0f) + v[a] * T0[b];
      }
      const float c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      const float c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      const float c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      const float id = __fdividef(1.0f, J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02);
      const float d0 = (F[0] * c00 + J[0][1] * (F[2] * J[1][2] - F[1] * J[2][2]) +
                        J[0][2] * (F[1] * J[2][1] - F[2] * J[1][1])) * id;
      const float d1 = (J[0][0] * (F[1] * J[2][2] - F[2] * J[1][2]) + F[0] * c01 +
                        J[0][2] * (F[2] * J[1][0] - F[1] * J[2][0])) * id;
      const float d2 = (J[0][0] * (F[2] * J[1][1] - F[1] * J[2][1]) + J[0][1] * (F[1] * J[2][0] - F[2] * J[1][0]) +
                        F[0] * c02) * id;
      v[0] -= d0;
      v[1] -= d1;
      v[2] -= d2;
      // quadratic convergence: after a step below 1e-4 the error is of
      // order its square, below the FP32 rounding of v
      if (fabsf(d0) + fabsf(d1) + fabsf(d2) < 1e-4f) break;
    }
    const float v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (!(v2 < 1.0f)) fl |= ERR_LANDAU;
    const float sq = sqrtf(1.0f - v2);
    const float dg = __fdividef(v2, sq * (1.0f + sq));  // gamma - 1
    const float U0 = 1.0f + dg, Ux = U0 * v[0], Uy = U0 * v[1], Uz = U0 * v[2];
    // n = U.N = n_r + n_d, e/n = y_r + y_d from the deviation moments
    const float Xi = M[0] - v[0] * M[1] - v[1] * M[2] - v[2] * M[3];
    const float nd = fmaf(dg, p.nr.lo, fmaf(dg, Xi + p.nr.hi, Xi));
    const float n = p.nr.hi + (p.nr.lo + nd);
    if (!(n > 0.0f)) fl |= ERR_DENSITY;
    const float ed = M[4] - M[5] * v[0] - M[6] * v[1] - M[7] * v[2];
    const float yd = __fdividef(ed - fmaf(p.yr.hi, nd, p.yr.lo * nd), n);
    if (!(p.yr.hi + yd > p.mb)) fl |= ERR_EOS;
    // EOS: T = 1 + T_d solves 3 T_d + m (R(m/T) - R_r) = y_d; FP32 Newton ...
    float Td = yd / p.cv_r, slope = p.cv_r;
#pragma unroll 1
    for (int it = 0; it < 12; ++it) {
      const float T = 1.0f + Td;
      if (!(T > 0.0f)) {
        fl |= ERR_EOS;
        Td = 0.0f;
        break;
      }
      const float zz = __fdividef(p.mb, T);
      const float R32 = ratio32(zz, p.rt32, fl);
      slope = eos_slope<float>(R32, zz);
      const float step = __fdividef(3.0f * Td + p.mb * ((R32 - p.Rr.hi) - p.Rr.lo) - yd, slope);
      Td -= step;
      if (fabsf(step) < 1e-4f) break;   // the FP64 step below squares the remaining error
    }
    // ... and one FP64 Newton step: dR(Td) from the lattice's FP64 table in
    // Td, else from the R(zeta) table
    float dR;
    {
      double dR64;
      if (!dr_table64(Td, p.dr64, dR64)) dR64 = dr_from_zeta(Td, p.mb64, p.Rr64, p.rt64, fl);
      const double g64 = fma(3.0, (double)Td, fma(p.mb64, dR64, -(double)yd));
      const float step = __fdividef((float)g64, slope);
      Td -= step;
      // R at the corrected T to first order: d(dR)/dTd = (c_v - 3)/m, c_v = slope
      dR = fmaf((slope - 3.0f) * __fdividef(1.0f, p.mb), -step, (float)dR64);
    }
    const float R = p.Rr.hi + (p.Rr.lo + dR);
    const float T = 1.0f + Td;
    // projections without their normalisations (those live in p.gf)
    const float mr32 = fmaf(p.mb, R, 4.0f * T);          // mbar K3/K2(zeta)
    const float r0 = fmaf(p.nr.hi, dR, fmaf(p.nr.lo, dR, nd * R));   // n R - n_r R_r
    const float r1 = n * (dg - p.k21 * dR);
    const float F = fmaf(p.mY, dR, 3.0f * Td);
    const float G = fmaf(p.mb, dR, 4.0f * Td);
    const float r5 = n * (F + dg * fmaf(2.0f, mr32, p.cb00_1) + dg * dg * mr32);
    const float h = n * fmaf(mr32, dg, G);
    const float nm = n * mr32;
    const float r9 = nm * (Uy * Uy - Uz * Uz);
    const float r10 = nm * (Uy * Uy + Uz * Uz - 2.0f * Ux * Ux);
    const float r11 = nm * Ux * Uz, r12 = nm * Uy * Uz, r13 = nm * Ux * Uy;
    const float rU[3] = {n * Ux, n * Uy, n * Uz};
    float c[6][9];
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      const HL* a = p.gf[g];
      float al = hl(a[0], r0);
      al = hl_fma(a[1], r1, al);
      al = hl_fma(a[2], r5, al);
      al = hl_fma(a[3], r9, al);
      al = hl_fma(a[4], r10, al);
      c[g][0] = al;
#pragma unroll
      for (int b = 0; b < 3; ++b) c[g][1 + b] = hl_fma(a[5], rU[b], hl(a[6], h * (b == 0 ? Ux : b == 1 ? Uy : Uz)));
      const float k9 = hl(a[7], r9), k10 = hl(a[8], r10);
      c[g][4] = fmaf(-3.0f, k10, k9);    // q_xx
      c[g][5] = 2.0f * k9;               // q_yy
      c[g][6] = hl(a[9], r13);           // q_xy
      c[g][7] = hl(a[9], r11);           // q_xz
      c[g][8] = hl(a[9], r12);           // q_yz
    }
    const float a0 = U0 * p.inv_tau, ax = p.v0 * Ux * p.inv_tau, ay = p.v0 * Uy * p.inv_tau,
                az = p.v0 * Uz * p.inv_tau;
    float* out = fout + ((unsigned)z * (unsigned)p.zstride + (unsigned)y * (unsigned)p.pitch + (unsigned)x);
    f3_collide_all<D>(Seq{}, p, keep, c, a0, ax, ay, az, out);
  }
  report(fl, p.err);
}

template <class D>
cudaError_t launch_fused3d_impl(const Fused3Params& p, const void* fin, void* fout, cudaStream_t s) {
  constexpr int smem = D::Q * 128 * (int)sizeof(float);
  static const cudaError_t attr =
      cudaFuncSetAttribute(fused3d_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) return attr;
  const unsigned grid = (unsigned)(((long long)p.Nx * p.Ny * p.Nz + 127) / 128);
  fused3d_kernel<D><<<grid, 128, smem, s>>>(p, static_cast<const float*>(fin), static_cast<float*>(fout));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused3d(int kind, const Fused3Params& p, const void* fin, void* fout, cudaStream_t s) {
  switch (kind) {
    case 1: return launch_fused3d_impl<Stencil3M1>(p, fin, fout, s);
    case 2: return launch_fused3d_impl<Stencil3G16>(p, fin, fout, s);
    case 3: return launch_fused3d_impl<Stencil3E5>(p, fin, fout, s);
    default: return launch_fused3d_impl<Stencil3S2>(p, fin, fout, s);
  }
}

}  // namespace rlbm
