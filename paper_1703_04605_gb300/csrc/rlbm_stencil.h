// Host-side construction of a second-order stencil (Sec. III C-D, App. A-C)
// and of the R(zeta) tables.  Internal to the library.
#pragma once

#include <array>
#include <string>
#include <vector>

#include "rlbm_internal.h"
#include "rlbm_o3_3d.h"

namespace rlbm {

// One population of the stencil folded onto the xy plane.
struct FoldedPop {
  int group;        // index 0..5 into the stencil's group list
  int nx, ny;       // displacement per step (lattice cells)
  int nz2;          // n_z^2 of the merged +-n_z pair
  int mult;         // 1 (n_z = 0) or 2 (merged pair)
};

struct StencilBuild {
  int groups[6];
  double mbar, v0;
  double w_group[6];          // Eq. 52 weights (FP64)
  std::vector<FoldedPop> pops;
  // per population, rounded once from binary128: mom[9] (p0, px, py, p0p0,
  // p0px, p0py, pxpx, pxpy, pypy), cj[10] = w_i J_k(p_i), vx, vy
  std::vector<std::array<double, 21>> popc;
  // the reference r_i = w_i K1/K2(mbar)/mbar (unit density, rest, T = T_R):
  // its J^(0) coefficient and its nine moments, rounded once from binary128
  double b0ref1;
  double mref1[9];
  // per group constants of the stencil-specialised kernels (see rlbm_fused.cuh):
  // gm = P0, P0^2, Pv, P0 Pv, Pv^2 with P0 = m gamma_k, Pv = m gamma_k v0;
  // gf = a0 a1 a4 a7 a8 bx2 bx5 q78 qy7 q9 (App. A/B normalisations folded in)
  double gm[6][5];
  double gf[6][10];
  // extended moment sums: per group P0 (P0 - m) and Pv (P0 - m) (kinetic
  // moments K^0, K^a = T^0a - m N^a); the reference's K^0 per unit density
  // and per particle; the largest reference population of each group
  double gk[6][2];
  double kref1, ykr1;
  double rmax1[6];
  double cv_r;          // 3 - mbar^2 R'(mbar): specific heat per particle at T_R
  int halo;
  SiteConsts sc;
};

// Vectors of group gid of Table I (full-symmetric orbit of its generator).
std::vector<std::array<int, 3>> group_orbit(int gid);

// Weights of Eq. 52 at (m, v0) in extended precision for 6 (second order) or
// 11 (third order) groups; false if singular.
bool quadrature_weights(const int* groups, int ngroups, double m, double v0, double* w);

// Widest positive-weight interval; returns number of disjoint windows (0: none).
int quadrature_window(const int* groups, int ngroups, double m, double* lo, double* hi);

// Full build: validates, solves weights, folds, App. A constants.
// Returns RLBM_OK or an error with a message.
rlbm_status build_stencil(const rlbm_stencil* st, double m, StencilBuild* out, std::string* err);

// Number of constants per population of an unfolded (3D) stencil: the 14
// momentum products p0, px, py, pz, p0p0, p0px, p0py, p0pz, pxpx, pxpy,
// pxpz, pypy, pypz, pzpz; the 14 values w_i J_k(p_i) of App. A in the order
// 1, J0, Jx, Jy, Jz, J00, J0x, J0y, J0z, (Jyy-Jzz), Jxx, Jxz, Jyz, Jxy; and
// the velocities p^a/p^0.
// (kPop3 and kMaxPop3 are defined with the device parameters.)

// One population of the unfolded stencil.
struct Pop3 {
  int group;
  int nx, ny, nz;
  std::array<double, kPop3> c;   // rounded once from binary128
};

struct StencilBuild3 {
  StencilBuild sb;                // validation, v0, weights, site constants; sb.gm are the
                                  // group momenta of the 3D kernels as well
  std::vector<Pop3> pops;
  double mref1[14];               // moments of the reference r_i at unit density
  int halo;                       // largest |n| component
  // per group constants of the stencil-specialised 3D kernel (rlbm_fused3d.cu):
  // w/m, w(P0-m k21)/A^2, w(P0^2+cJ1 P0+cJ0)/(3C^2), -|n|^2 K9, |n|^2 K10,
  // w Pv/B^2, w Pv(P0-m k32)/D^2, K9 = w Pv^2/(4E^2), K10 = w Pv^2/(12E^2),
  // K13 = w Pv^2/E^2
  double gf3[6][10];
};

// Unfolded build for 3D lattices (the paper's stencil itself, Table I orbits
// with signed n_z); same validation and weights as build_stencil.
rlbm_status build_stencil3d(const rlbm_stencil* st, double m, StencilBuild3* out, std::string* err);

// Third-order stencil folded onto the xy plane (eleven groups, Sec. III D).
// The equilibrium is f_i^eq = n w_i P(p_i) with P the polynomial of degree
// <= 3 whose moments against every monomial of degree <= 3 are those of the
// Maxwell-Juttner distribution (the third-order truncation of Eq. 14-16).
// Per population i the table row (kRowO3 entries) holds:
//   0..8   p0, px, py, p0p0, p0px, p0py, pxpx, pxpy, pypy
//   9      wr_i = w_i K1/K2(mbar)/mbar  (f^eq of the rest state at T_R, n = 1)
//   10..29 W_il = w_i (G^-1 phi(p_i))_l: the dual basis of the 20 centred
//          monomials phi_l (kO3Mono order, t = p0 - c, c = mbar K2/K1(mbar)),
//          G_lk = sum_i w_i phi_l(p_i) phi_k(p_i)
//   30, 31 px/p0, py/p0
// so that f^eq_i = n wr_i + n sum_l dmu_l W_il, dmu_l the deviation of the
// l-th centred moment (per unit density) from its value at rest and T_R.
struct StencilBuildO3 {
  int groups[11];
  double mbar, v0;
  double w_group[11];
  std::vector<FoldedPop> pops;
  std::vector<std::array<double, kRowO3>> rows;
  double mref1[9];       // moments of the reference wr_i (unit density)
  double c;              // centring shift mbar K2/K1(mbar) = <p0>_omega
  double gm[11][5];      // per group: P0, P0^2, Pv, P0 Pv, Pv^2 (P0 = m gamma, Pv = m gamma v0)
  double cv_r;           // 3 - mbar^2 R'(mbar): specific heat per particle at T_R
  int halo;
  SiteConsts sc;         // mbar, R(mbar) and the constants of the site solve
};

rlbm_status build_stencil_o3(const rlbm_stencil* st, double m, StencilBuildO3* out, std::string* err);

// Third-order stencil unfolded for 3D lattices: base.pops in the order of
// build_stencil3d with c[0..13] the momentum products, c[14] the rest-frame
// weight w_i K1/K2(mbar)/mbar and c[28..30] p^a/p^0; base.mref1 the moments of
// that weight; wrows the dual basis of the thirty monomials of kO3Exp3.
struct StencilBuild3O3 {
  StencilBuild3 base;       // base.sb holds v0, mbar and the site constants
  int groups[11];
  double w_group[11];
  double c;                 // centring shift mbar K2/K1(mbar)
  std::vector<std::array<double, kRowW3>> wrows;
};

rlbm_status build_stencil3d_o3(const rlbm_stencil* st, double m, StencilBuild3O3* out, std::string* err);

// Per-population constant table for the kernels (CT = float or double).
template <typename CT>
void fill_pop_table(const StencilBuild& sb, int Nx, int Ny, PopTable<CT>* pt);

// R(zeta) tables (built once per process).
const std::vector<double>& ratio_table64();
const std::vector<float>& ratio_table32();
double ratio_eval_host(double z, int precision);
// The lattice's dR(Td) table (layout in rlbm_internal.h), fitted from the
// FP64 R(zeta) table.
std::vector<double> dr_table(double mbar);

// Message returned by rlbm_last_error(NULL) (defined with the C ABI).
void set_global_error(const std::string& msg);

}  // namespace rlbm
