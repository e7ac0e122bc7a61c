// Stencil-specialised FP32 third-order step (sm_103a).
//
// The step of rlbm_kernels_o3.cu (pull, moments, Landau frame, n = U.N, EOS,
// third-order equilibrium, Anderson-Witting relaxation) restructured like the
// second-order fused kernel (rlbm_fused.cuh):
//
//  * the folded eleven-group stencil is a compile-time constant:
//    displacements are immediates, and the moments are accumulated per group
//    with exact integer weights and folded in with hi/lo group constants;
//    the populations are pulled twice, once for the moments and once for the
//    relaxation (see O3_TWO_PASS), rather than held in registers across the
//    site solve;
//  * storage d_i = f_i - nref wr_i and the split site solve (n = n_r + n_d,
//    T = 1 + T_d, R = R(mbar) + dR, one FP64 EOS step) of split_solve;
//  * the equilibrium f_i^eq - nref wr_i = n_d wr_i + sum_l e_l W_il, with
//    e_l = n dmu_l (the deviations of the centred Maxwell-Juttner moments,
//    rlbm_o3.cuh), is evaluated once per reflection orbit: the twenty
//    centred monomials split into classes even/odd in p_x and p_y (8 even in
//    both, 5 odd in p_x only, 5 odd in p_y only, 2 odd in both), the dual
//    basis W inherits the parities, and the members (+-n_x, +-n_y) of an
//    orbit take the four class sums with the matching signs.  The W of the
//    representative enter as hi/lo pairs, so no constant carries a fixed FP32
//    rounding into the conserved moments.
#include <utility>

#include "rlbm_fused.cuh"
#include "rlbm_o3.cuh"

namespace rlbm {
namespace {

// Parity classes of the centred monomials (kO3Mono order; rlbm_internal.h).
using kEE = std::integer_sequence<int, 0, 1, 6, 7, 9, 10, 11, 17>;   // even in p_x and p_y
using kOE = std::integer_sequence<int, 2, 4, 13, 15, 18>;            // odd in p_x only
using kEO = std::integer_sequence<int, 3, 5, 14, 16, 19>;            // odd in p_y only
using kOO = std::integer_sequence<int, 8, 12>;                       // odd in both

template <class Def, int K>
__host__ __device__ constexpr bool last_of_group() {
  return K + 1 == Def::O.K || Def::O.grp[K + 1] != Def::O.grp[K];
}

// Group sums of one reflection orbit (as fused_acc_orbit) into the current
// group's s[6]; after the group's last orbit they are folded into the
// deviation moments M (N0 Nx Ny T00 T0x T0y Txx Txy Tyy) with the group's
// hi/lo momenta and cleared.
template <class Def, int K>
__device__ __forceinline__ void o3_acc_orbit(const float (&d)[Def::Q], float (&s)[6], float (&M)[9],
                                             const FusedO3Params& p) {
  constexpr int kind = Def::O.kind[K], g = Def::O.grp[K], ax = Def::O.ax[K], ay = Def::O.ay[K];
  constexpr int i0 = Def::O.idx[K][0], i1 = Def::O.idx[K][1], i2 = Def::O.idx[K][2], i3 = Def::O.idx[K][3];
  if constexpr (kind == 1) {
    s[0] += d[i0];
  } else if constexpr (kind == 2) {
    const float S = d[i0] + d[i1], D = d[i0] - d[i1];
    s[0] += S;
    s[1] = fmaf((float)ax, D, s[1]);
    s[3] = fmaf((float)(ax * ax), S, s[3]);
  } else if constexpr (kind == 3) {
    const float S = d[i0] + d[i2], D = d[i0] - d[i2];
    s[0] += S;
    s[2] = fmaf((float)ay, D, s[2]);
    s[5] = fmaf((float)(ay * ay), S, s[5]);
  } else {
    const float a = d[i0] + d[i1], b = d[i0] - d[i1], c = d[i2] + d[i3], w = d[i2] - d[i3];
    const float S = a + c;
    s[0] += S;
    s[1] = fmaf((float)ax, b + w, s[1]);
    s[2] = fmaf((float)ay, a - c, s[2]);
    s[3] = fmaf((float)(ax * ax), S, s[3]);
    s[4] = fmaf((float)(ax * ay), b - w, s[4]);
    s[5] = fmaf((float)(ay * ay), S, s[5]);
  }
  if constexpr (last_of_group<Def, K>()) {
    const HL* gm = p.gm[g];
    M[0] = hl_fma(gm[0], s[0], M[0]);
    M[3] = hl_fma(gm[1], s[0], M[3]);
    M[1] = hl_fma(gm[2], s[1], M[1]);
    M[2] = hl_fma(gm[2], s[2], M[2]);
    M[4] = hl_fma(gm[3], s[1], M[4]);
    M[5] = hl_fma(gm[3], s[2], M[5]);
    M[6] = hl_fma(gm[4], s[3], M[6]);
    M[7] = hl_fma(gm[4], s[4], M[7]);
    M[8] = hl_fma(gm[4], s[5], M[8]);
#pragma unroll
    for (int k = 0; k < 6; ++k) s[k] = 0.0f;
  }
}

// the pulled values of the collision pass: kept in registers since the
// moment pass, or pulled again (two-pass form; L1/L2 hits)
struct O3Repull {
  const float* fin;
  long long plane, pitch;
  int x, y, Nx, Ny;
};
template <class Def, int I>
__device__ __forceinline__ float o3_pop(const float (&d)[Def::Q]) {
  return d[I];
}
template <class Def, int I>
__device__ __forceinline__ float o3_pop(const O3Repull& r) {
  constexpr int DX = Def::F.nx[I], DY = Def::F.ny[I];
  const unsigned idx = (unsigned)wrap_c<DY>(r.y, r.Ny) * (unsigned)r.pitch + (unsigned)wrap_c<DX>(r.x, r.Nx);
  return __ldg(r.fin + idx + (size_t)(unsigned)r.plane * I);
}

// d_i + (p_i.U/(p_i^0 tau)) (e - d_i), stored at the site; the weight is
// (U0 - v0 (n_x U_x + n_y U_y))/tau.
template <class Def, int I, class Pops>
__device__ __forceinline__ void o3_relax(const Pops& d, float e, float a0, float ax, float ay,
                                         float* __restrict__ out, long long plane) {
  constexpr int nx = Def::F.nx[I], ny = Def::F.ny[I];
  float om = a0;
  if constexpr (nx != 0) om = fmaf(-(float)nx, ax, om);
  if constexpr (ny != 0) om = fmaf(-(float)ny, ay, om);
  const float v = o3_pop<Def, I>(d);
  __stcs(out + (size_t)(unsigned)plane * I, fmaf(om, e - v, v));   // plane < 2^32 elements
}

template <int... L>
__device__ __forceinline__ float class_sum(std::integer_sequence<int, L...>, const HL* w, const float (&e)[kO3Mono],
                                           float acc) {
  ((acc = hl_fma(w[1 + L], e[L], acc)), ...);
  return acc;
}

// Equilibrium and relaxation of the members of reflection orbit K.
template <class Def, int K, class Pops>
__device__ __forceinline__ void o3_collide_orbit(const Pops& d, const float (&e)[kO3Mono], float nd,
                                                 float a0, float ax, float ay, float* __restrict__ out,
                                                 long long plane, const FusedO3Params& p) {
  constexpr int kind = Def::O.kind[K];
  constexpr int i0 = Def::O.idx[K][0], i1 = Def::O.idx[K][1], i2 = Def::O.idx[K][2], i3 = Def::O.idx[K][3];
  const HL* w = p.ow[K];
  const float E = class_sum(kEE{}, w, e, hl(w[0], nd));
  if constexpr (kind == 1) {
    o3_relax<Def, i0, Pops>(d, E, a0, ax, ay, out, plane);
  } else if constexpr (kind == 2) {
    const float X = class_sum(kOE{}, w, e, 0.0f);
    o3_relax<Def, i0, Pops>(d, E + X, a0, ax, ay, out, plane);
    o3_relax<Def, i1, Pops>(d, E - X, a0, ax, ay, out, plane);
  } else if constexpr (kind == 3) {
    const float Y = class_sum(kEO{}, w, e, 0.0f);
    o3_relax<Def, i0, Pops>(d, E + Y, a0, ax, ay, out, plane);
    o3_relax<Def, i2, Pops>(d, E - Y, a0, ax, ay, out, plane);
  } else {
    const float X = class_sum(kOE{}, w, e, 0.0f);
    const float Y = class_sum(kEO{}, w, e, 0.0f);
    const float Z = class_sum(kOO{}, w, e, 0.0f);
    const float EP = E + Z, EM = E - Z, XP = X + Y, XM = X - Y;
    o3_relax<Def, i0, Pops>(d, EP + XP, a0, ax, ay, out, plane);   // (+, +)
    o3_relax<Def, i1, Pops>(d, EM - XM, a0, ax, ay, out, plane);   // (-, +)
    o3_relax<Def, i2, Pops>(d, EM + XM, a0, ax, ay, out, plane);   // (+, -)
    o3_relax<Def, i3, Pops>(d, EP - XP, a0, ax, ay, out, plane);   // (-, -)
  }
}

// Pull of one population (32-bit element indices, as fused_load).
template <class Def, int I>
__device__ __forceinline__ void o3_load(float (&d)[Def::Q], const void* __restrict__ fin, long long plane,
                                        long long pitch, int x, int y, int Nx, int Ny) {
  fused_load<Def, false, I>(d, fin, nullptr, plane, pitch, x, y, Nx, Ny);
}

template <class Def, int... Is>
__device__ __forceinline__ void o3_load_all(std::integer_sequence<int, Is...>, float (&d)[Def::Q],
                                            const void* __restrict__ fin, long long plane, long long pitch, int x,
                                            int y, int Nx, int Ny) {
  (o3_load<Def, Is>(d, fin, plane, pitch, x, y, Nx, Ny), ...);
}

template <class Def, int... Ks>
__device__ __forceinline__ void o3_acc_all(std::integer_sequence<int, Ks...>, const float (&d)[Def::Q],
                                           float (&s)[6], float (&M)[9], const FusedO3Params& p) {
  (o3_acc_orbit<Def, Ks>(d, s, M, p), ...);
}

template <class Def, class Pops, int... Ks>
__device__ __forceinline__ void o3_collide_all(std::integer_sequence<int, Ks...>, const Pops& d,
                                               const float (&e)[kO3Mono], float nd, float a0, float ax, float ay,
                                               float* __restrict__ out, long long plane, const FusedO3Params& p) {
  (o3_collide_orbit<Def, Ks, Pops>(d, e, nd, a0, ax, ay, out, plane, p), ...);
}

// Two passes over the populations: the moment pass pulls each value and
// folds it into the group sums, the collision pass pulls it again (an L1/L2
// hit: the block read the same lines moments earlier, 1 % extra DRAM reads)
// instead of keeping Q values in registers across the site solve.  Resident
// blocks of 128 threads per SM: four (128 registers, no spills) up to Q = 104,
// three (168 registers, at most 16 bytes spilled) for the Q = 133-149 sets.
// Measured on GB300 against one pass: 4 % faster at Q <= 104 (one pass at
// four blocks spilled 70-90 bytes; at three blocks of 168 registers it was
// 11 % slower), 8-21 % faster for the larger sets (one pass at two blocks
// of 255 registers).  Results are the same bit for bit.
constexpr bool O3_TWO_PASS = true;

template <class Def>
constexpr int o3_min_blocks() {
  return Def::Q <= 104 ? 4 : 3;
}

template <class Def>
__global__ void __launch_bounds__(128, o3_min_blocks<Def>()) fused_o3_kernel(const __grid_constant__ FusedO3Params p,
                                                          const float* __restrict__ fin, float* __restrict__ fout) {
  static_assert(Def::O.K <= kMaxOrbO3, "orbit constants exceed FusedO3Params::ow");
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (site < p.Nx * p.Ny) {
    int x, y;
    site_of(site, p.Nx, x, y);
    float s[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float M[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) M[k] = 0.0f;
    using Orb = std::make_integer_sequence<int, Def::O.K>;
    constexpr bool two_pass = O3_TWO_PASS;
    float d[two_pass ? 1 : Def::Q];
    if constexpr (two_pass) {
      float dd[Def::Q];
      o3_load_all<Def>(std::make_integer_sequence<int, Def::Q>{}, dd, fin, p.plane, p.pitch, x, y, p.Nx, p.Ny);
      o3_acc_all<Def>(Orb{}, dd, s, M, p);
    } else {
      o3_load_all<Def>(std::make_integer_sequence<int, Def::Q>{}, d, fin, p.plane, p.pitch, x, y, p.Nx, p.Ny);
      o3_acc_all<Def>(Orb{}, d, s, M, p);
    }
    const SplitSite ss = split_solve(p, M, fl);
    // e_l = n dmu_l in the small quantities dU, dT, dR, U_x, U_y (no cancellation)
    float e[kO3Mono];
    o3_deviations<float>(p.mb, p.c, ss.n, ss.U0, ss.Ux, ss.Uy, ss.dg, ss.dR, ss.Td, ss.T, ss.R, e);
    const float Ux = ss.Ux, Uy = ss.Uy;
    const float a0 = ss.U0 * p.inv_tau, ax = p.v0 * Ux * p.inv_tau, ay = p.v0 * Uy * p.inv_tau;
    float* out = fout + (long long)y * p.pitch + x;
    if constexpr (two_pass)
      o3_collide_all<Def>(Orb{}, O3Repull{fin, p.plane, p.pitch, x, y, p.Nx, p.Ny}, e, ss.nd, a0, ax, ay, out,
                          p.plane, p);
    else o3_collide_all<Def>(Orb{}, d, e, ss.nd, a0, ax, ay, out, p.plane, p);
  }
  report(fl, p.err);
}

}  // namespace

cudaError_t launch_fused_o3(int kind, const FusedO3Params& p, const void* fin, void* fout, cudaStream_t s) {
  const unsigned grid = (unsigned)(((long long)p.Nx * p.Ny + 127) / 128);
  const float* f = static_cast<const float*>(fin);
  float* g = static_cast<float*>(fout);
  if (kind == 5) fused_o3_kernel<StencilO3M5><<<grid, 128, 0, s>>>(p, f, g);
  else if (kind == 6) fused_o3_kernel<StencilO3D><<<grid, 128, 0, s>>>(p, f, g);
  else if (kind == 7) fused_o3_kernel<StencilO3E><<<grid, 128, 0, s>>>(p, f, g);
  else if (kind == 8) fused_o3_kernel<StencilO3A><<<grid, 128, 0, s>>>(p, f, g);
  else if (kind == 9) fused_o3_kernel<StencilO3B><<<grid, 128, 0, s>>>(p, f, g);
  else fused_o3_kernel<StencilO3C><<<grid, 128, 0, s>>>(p, f, g);
  return cudaGetLastError();
}

const void* fused_o3_kernel_fn(int kind) {
  if (kind == 5) return (const void*)&fused_o3_kernel<StencilO3M5>;
  if (kind == 6) return (const void*)&fused_o3_kernel<StencilO3D>;
  if (kind == 7) return (const void*)&fused_o3_kernel<StencilO3E>;
  if (kind == 8) return (const void*)&fused_o3_kernel<StencilO3A>;
  if (kind == 9) return (const void*)&fused_o3_kernel<StencilO3B>;
  return (const void*)&fused_o3_kernel<StencilO3C>;
}

}  // namespace rlbm
