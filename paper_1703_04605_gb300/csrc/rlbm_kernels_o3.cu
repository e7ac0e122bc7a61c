// Third-order step on a periodic Nx x Ny lattice: an eleven-group stencil
// (Sec. III D) folded onto the xy plane, with the equilibrium expanded to
// third order (Eq. 14-16 with polynomials of degree <= 3, Sec. III A-B).
//
// Per site: pull the Q populations, form N^a and T^ab (Eq. 4-5, 18), solve the
// Landau frame (Eq. 20), n = U.N (Eq. 19) and T from e/n = 3T + m K1/K2(m/T)
// (Eq. 28) -- the same site solve as the second-order kernels -- then
//
//   f_i^eq = n wr_i + n sum_l dmu_l W_il                                 (*)
//
// where W_il is the dual basis of twenty centred monomials phi_l (host table,
// rlbm_stencil.h) and dmu_l the deviation, per unit density, of the moment
// of phi_l under the Maxwell-Juttner distribution (Eq. 4-6, 43-44) from its
// value at rest and T = T_R (o3_deviations, rlbm_o3.cuh).  (*) is the unique
// w_i times a polynomial of degree <= 3 whose moments against every such
// polynomial equal the continuum ones, i.e. the third-order truncation.
//
// Kernels: two passes over the populations per site (moments, then relax and
// store), table rows read with vector loads, as the generic 3D kernels.
#include "rlbm_kernels.cuh"
#include "rlbm_o3.cuh"

namespace rlbm {
namespace {

__device__ __forceinline__ double fmo(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmo(float a, float b, float c) { return fmaf(a, b, c); }

template <typename A>
__device__ __forceinline__ const A* tab_o3(const O3Params& p);
template <>
__device__ __forceinline__ const double* tab_o3<double>(const O3Params& p) { return p.tab64; }
template <>
__device__ __forceinline__ const float* tab_o3<float>(const O3Params& p) { return p.tab32; }

__device__ __forceinline__ void ld4o(const float* p, float* d) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  d[0] = v.x;
  d[1] = v.y;
  d[2] = v.z;
  d[3] = v.w;
}
__device__ __forceinline__ void ld4o(const double* p, double* d) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  d[0] = a.x;
  d[1] = a.y;
  d[2] = b.x;
  d[3] = b.y;
}

__device__ __forceinline__ bool interior_o3(const O3Params& p, int x, int y) {
  return x >= p.halo && x < p.Nx - p.halo && y >= p.halo && y < p.Ny - p.halo;
}

// Element of population plane i that streams into (x, y): x - n_i, periodic.
__device__ __forceinline__ long long source_o3(const O3Params& p, int i, int x, int y) {
  return (long long)wrap_sub(y, __ldg(p.shift + p.Q + i), p.Ny) * p.pitch + wrap_sub(x, __ldg(p.shift + i), p.Nx);
}

// n dmu_l (kO3Mono order) from the FP64 site macros; R_t = double or float.
template <typename R_t>
__device__ __forceinline__ void dmu_o3(const Macro<double>& md, const O3Params& p, R_t (&e)[kO3Mono]) {
  o3_deviations<R_t>((R_t)p.sc.mbar, (R_t)p.c, (R_t)md.n, (R_t)md.U0, (R_t)md.Ux, (R_t)md.Uy, (R_t)md.dU,
                     (R_t)md.dR, (R_t)(md.T - 1.0), (R_t)md.T, (R_t)md.R, e);
}

// Macros of an init field (n, u, T) in the form the site solve returns.
__device__ __forceinline__ Macro<double> macro_of_fields(double n, double ux, double uy, double T,
                                                        const O3Params& p, unsigned& fl) {
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
  md.F = md.G = 0.0;
  return md;
}

template <typename S>
__global__ void __launch_bounds__(128) step_o3_kernel(const __grid_constant__ O3Params p,
                                                      const S* __restrict__ fin, S* __restrict__ fout) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (s < p.Nx * p.Ny) {
    int x, y;
    site_of(s, p.Nx, x, y);
    const S* tab = tab_o3<S>(p);
    const bool in = interior_o3(p, x, y);
    const long long here = (long long)y * p.pitch + x;
    // pass 1: moments N0 Nx Ny T00 T0x T0y Txx Txy Tyy
    S mm[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) mm[k] = S(0);
#pragma unroll 4
    for (int i = 0; i < p.Q; ++i) {
      const long long src = in ? here + __ldg(p.off + i) : source_o3(p, i, x, y);
      const S f = __ldg(fin + (long long)i * p.plane + src);
      S c[12];
      const S* row = tab + (long long)i * kRowO3;
#pragma unroll
      for (int j = 0; j < 3; ++j) ld4o(row + 4 * j, c + 4 * j);
#pragma unroll
      for (int k = 0; k < 9; ++k) mm[k] = fmo(f, c[k], mm[k]);
    }
    Macro<double> md;
    if constexpr (sizeof(S) == 4) {
      md = solve_site_mixed(mm, p.mref, p.sc, p.rt64, p.rt32, fl);
    } else {
      double m9[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) m9[k] = mm[k] + p.mref[k];
      md = solve_site_f64(m9, p.sc, p.rt64, fl);
    }
    S e[kO3Mono];
    dmu_o3<S>(md, p, e);
    const S dn = (S)(md.n - p.nref);
    const S a0 = (S)(md.U0 * p.inv_tau), ax = (S)(md.Ux * p.inv_tau), ay = (S)(md.Uy * p.inv_tau);
    // pass 2: f^eq (*), relaxation with weight p_i.U/(p_i^0 tau), store at the site
    S* out = fout + here;
#pragma unroll 2
    for (int i = 0; i < p.Q; ++i) {
      const long long src = in ? here + __ldg(p.off + i) : source_o3(p, i, x, y);
      const S f = __ldg(fin + (long long)i * p.plane + src);
      S c[24];                                       // row entries 8..31
      const S* row = tab + (long long)i * kRowO3 + 8;
#pragma unroll
      for (int j = 0; j < 6; ++j) ld4o(row + 4 * j, c + 4 * j);
      S feq = dn * c[1];
#pragma unroll
      for (int l = 0; l < kO3Mono; ++l) feq = fmo(e[l], c[2 + l], feq);
      const S om = a0 - ax * c[22] - ay * c[23];
      __stcs(out + (long long)i * p.plane, fmo(om, feq - f, f));
    }
  }
  report(fl, p.err);
}

// f = f^eq(n, U, T) (Eq. 16) at every site: S_0 at the site and S_{-1} at
// x - n_i, so that the pull of S_{-1} is f(., 0) (the 2D convention).
template <typename S>
__global__ void __launch_bounds__(128) init_o3_kernel(const __grid_constant__ O3Params p, FieldPtrs fd,
                                                      S* __restrict__ cur, S* __restrict__ prev) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (s < p.Nx * p.Ny) {
    int x, y;
    site_of(s, p.Nx, x, y);
    const Macro<double> md = macro_of_fields(fd.n[s], fd.ux[s], fd.uy[s], fd.T[s], p, fl);
    double e[kO3Mono];
    dmu_o3<double>(md, p, e);
    const double dn = md.n - p.nref;
    const long long here = (long long)y * p.pitch + x;
#pragma unroll 1
    for (int i = 0; i < p.Q; ++i) {
      const double* row = p.tab64 + (long long)i * kRowO3;
      double feq = dn * __ldg(row + 9);
#pragma unroll
      for (int l = 0; l < kO3Mono; ++l) feq = fma(e[l], __ldg(row + 10 + l), feq);
      cur[(long long)i * p.plane + here] = (S)feq;
      prev[(long long)i * p.plane + source_o3(p, i, x, y)] = (S)feq;
    }
  }
  report(fl, p.err);
}

// Read-out of the pre-collision state at time t: the pull of the buffer the
// last step read, FP64 solve; planes in mask order (n, u_x, u_y, T, e, N^a,
// T^ab), as the second-order read-out.
template <typename S>
__global__ void __launch_bounds__(128) moments_o3_kernel(const __grid_constant__ O3Params p,
                                                         const S* __restrict__ prev, MomentOut mo) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  const long long N = (long long)p.Nx * p.Ny;
  if (s < N) {
    int x, y;
    site_of(s, p.Nx, x, y);
    double m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = 0.0;
#pragma unroll 1
    for (int i = 0; i < p.Q; ++i) {
      const double f = (double)prev[(long long)i * p.plane + source_o3(p, i, x, y)];
#pragma unroll
      for (int k = 0; k < 9; ++k) m[k] = fma(f, __ldg(p.tab64 + (long long)i * kRowO3 + k), m[k]);
    }
#pragma unroll
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

unsigned grid_o3(const O3Params& p) { return (unsigned)(((long long)p.Nx * p.Ny + 127) / 128); }

}  // namespace

cudaError_t launch_step_o3(rlbm_dtype dt, const O3Params& p, const void* fin, void* fout, cudaStream_t s) {
  if (dt == RLBM_F64)
    step_o3_kernel<double><<<grid_o3(p), 128, 0, s>>>(p, static_cast<const double*>(fin), static_cast<double*>(fout));
  else
    step_o3_kernel<float><<<grid_o3(p), 128, 0, s>>>(p, static_cast<const float*>(fin), static_cast<float*>(fout));
  return cudaGetLastError();
}

cudaError_t launch_init_o3(rlbm_dtype dt, const O3Params& p, FieldPtrs f, void* cur, void* prev, cudaStream_t s) {
  if (dt == RLBM_F64)
    init_o3_kernel<double><<<grid_o3(p), 128, 0, s>>>(p, f, static_cast<double*>(cur), static_cast<double*>(prev));
  else
    init_o3_kernel<float><<<grid_o3(p), 128, 0, s>>>(p, f, static_cast<float*>(cur), static_cast<float*>(prev));
  return cudaGetLastError();
}

cudaError_t launch_moments_o3(rlbm_dtype dt, const O3Params& p, const void* prev, MomentOut o, cudaStream_t s) {
  if (dt == RLBM_F64)
    moments_o3_kernel<double><<<grid_o3(p), 128, 0, s>>>(p, static_cast<const double*>(prev), o);
  else
    moments_o3_kernel<float><<<grid_o3(p), 128, 0, s>>>(p, static_cast<const float*>(prev), o);
  return cudaGetLastError();
}

}  // namespace rlbm
