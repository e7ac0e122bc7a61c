// Internal layout shared by the host library (rlbm_host.cpp) and the CUDA
// kernels (rlbm_kernels.cuh).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/rlbm.h"

namespace rlbm {

// Largest folded stencil the kernels are compiled for.
constexpr int QMAX = 96;
// Population-count buckets with compiled kernels (register arrays of QB).
constexpr int QBUCKETS[] = {40, 64, 80, 96};

// Second-order polynomials that survive in 2D (U^z = 0), in this order:
//   0: J^(0)  1: J_0  2: J_x  3: J_y  4: J_00  5: J_0x  6: J_0y
//   7: J_xx = (p_y^2 - p_z^2)/(2E)   8: J_yy = (-2p_x^2 + p_y^2 + p_z^2)/(2 sqrt3 E)
//   9: J_xy
constexpr int NJ = 10;

// Piecewise-polynomial tables of R(zeta) = K1(zeta)/K2(zeta).  zeta in
// [2^RT_EMIN, 2^RT_EMAX) is split into octaves and each octave into
// RT_SEG equal mantissa slices; each slice holds a polynomial in the local
// variable x in [-1, 1] (monomial coefficients, lowest degree first).
constexpr int RT_EMIN = -16;
constexpr int RT_EMAX = 16;
constexpr int RT_SEG = 8;                                  // slices per octave (2^3)
constexpr int RT_NSEG = (RT_EMAX - RT_EMIN) * RT_SEG;
constexpr int RT_NC64 = 11;                                // degree 10
constexpr int RT_NC32 = 6;                                 // degree 5

// Constants of App. A and B at mbar (rounded once from binary128).
// Derived forms used by the kernels (all exact rearrangements of App. B):
//   b0  = R/mbar
//   b_0 = (U0 - k21 R)/A                = (dU - k21 (R - Rr)) iA
//   b_a = U_a / B
//   b00 = (mbar r32 U0^2 + cb00_1 U0 + R Y - T)/(sqrt3 C)
//       = (F + dU (2 mbar r32 + cb00_1) + dU^2 mbar r32) i3C,
//         F = (mbar + Y)(R - Rr) + 3 (T - 1)
//   b0a = (mbar r32 U0 - mbar k32) U_a / D = (G + mbar r32 dU) U_a iD,
//         G = mbar (R - Rr) + 4 (T - 1)
//   bxx = mbar r32 U_y^2 i2E,  byy = mbar r32 (U_y^2 - 2 U_x^2) i23E,
//   bxy = mbar r32 U_x U_y iE
// with dU = U0 - 1, r32 = K3/K2(zeta) = R + 4 T/mbar, Rr = R(mbar) = 1/k21
// (T_R = 1), F and G vanishing at T = T_R because b_00 = b_0 = 0 for the
// rest-frame weight itself.  The differences R - Rr and T - 1 are formed in
// FP64 so that the FP32 path keeps b_00, b_0 and b_0a accurate near T_R.
struct SiteConsts {
  double mbar, inv_m;
  double k21;     // K2/K1 (mbar)
  double k32;     // K3/K2 (mbar)
  double Rr;      // K1/K2 (mbar) = 1/k21
  double A, B, C, D, E;
  double iA, iB, i3C, iD, i2E, i23E, iE;
  double cb00_1;  // U_0 coefficient of b_00: 3 (1/X - 1)
  double Y;       // mbar fraction of b_00
  double mY;      // mbar + Y
  double mk32;    // mbar k32
};

// Per-population constants of one folded stencil.  Entries i >= Q are zero.
template <typename CT>
struct PopTable {
  int dxm[QMAX], dym[QMAX];   // displacement reduced mod Nx, Ny (in [0, N))
  CT mom[9][QMAX];            // p0, px, py, p0p0, p0px, p0py, pxpx, pxpy, pypy
  CT cj[NJ][QMAX];            // w_i J_k(p_i)
  CT vx[QMAX], vy[QMAX];      // p^x/p^0, p^y/p^0
};

// FP32 storage holds d_i = f_i - r_i, r_i = nref w_i K1/K2(mbar)/mbar: the
// rest-frame equilibrium at density nref and T = T_R (all b^(k>0) vanish
// there).  r_i is uniform in space, so streaming and the Anderson-Witting
// relaxation act on d_i exactly as on f_i (with f^eq_i - r_i in place of
// f^eq_i); the moments of r_i are added back in FP64.  FP64 storage holds f_i
// (nref = 0).
template <typename CT>
struct StepParams {
  int Nx, Ny, Q, halo;
  long long pitch, plane;     // elements
  double inv_tau, v0;
  double nref;                // reference density (0: plain f_i storage)
  double b0ref;               // nref K1/K2(mbar)/mbar: n b^(0) of r_i
  double mref[9];             // moments of r_i (same order as PopTable::mom)
  SiteConsts sc;
  const double* rt64;         // RT_NSEG * RT_NC64
  const float* rt32;          // RT_NSEG * RT_NC32
  unsigned* err;              // sticky device error bits
  PopTable<CT> pt;
};

// Per-lattice table of dR(Td) = R(mbar/(1 + Td)) - R(mbar) (T = 1 + Td in
// units of T_R) for the final FP64 Newton step of the FP32 kernels' EOS: one
// polynomial of degree DR_NC - 1 per slice of width 1/64 in Td, in the local
// variable x = 64 Td - trunc(64 Td) (in [0, 1) for Td >= 0, (-1, 0] below),
// which FP32 forms exactly.  Slices DR_NNEG - 1 - j cover Td in
// (-(j+1)/64, -j/64], slices DR_NNEG + k cover [k/64, (k+1)/64); outside
// (-DR_NNEG/64, DR_NPOS/64) the kernels use the R(zeta) table.
constexpr int DR_NNEG = 48;      // T > 1/4 T_R
constexpr int DR_NPOS = 192;     // T < 4 T_R
constexpr int DR_NC = 7;         // degree 6
constexpr int DR_NSEG = DR_NNEG + DR_NPOS;

// bound on the populations of the compiled second-order stencils (at most 73)
constexpr int kMaxQ2 = 80;

// Parameters of the stencil-specialised FP32 kernels (rlbm_fused.cuh).
// A constant as the sum of two FP32 numbers (about 48 significant bits).
struct HL {
  float hi, lo;
};

struct FusedParams {
  int Nx, Ny;
  long long pitch, plane;
  float inv_tau, v0;
  // FP32 constants of the projection formulas (deviation-level terms only)
  float mb, k21, mk32, cb00_1, mY;
  float cv_r;          // specific heat per particle at T_R (Newton start)
  HL Rr;               // R(mbar) = K1/K2(mbar)
  HL nr;               // reference density
  HL yr;               // reference energy per particle e_r/n_r
  HL mref[9];          // reference moments (hi/lo: no fixed rounding in the Landau solve)
  double Rr64, hr64, mb64, nr64;
  HL gm[6][5];         // per group: P0, P0^2, Pv, P0 Pv, Pv^2 (P0 = m gamma, Pv = m gamma v0)
  HL gf[6][10];        // per group: a0 a1 a4 a7 a8 bx2 bx5 q78 qy7 q9 (see host)
  // extended moment sums only: per group P0 (P0 - m), Pv (P0 - m); the
  // reference's kinetic moment K^0 and (e - m n)/n; per group the magic
  // constant 1.5 2^23 q of the exact split grid q
  HL gk[6][2];
  HL k0r, ykr;
  float exC[6];
  double gm64[6][5];   // gm in FP64 (read-out kernel)
  const double* rt64;
  const float* rt32;
  const double* dr64;  // DR_NSEG * DR_NC (the lattice's dR(Td) table)
  unsigned* err;
  // BF16 deviation storage only: per-site equilibrium reference coefficients,
  // six planes (one per group) of uint2 = 4 bf16 (alpha, beta_x, beta_y, q)
  const void* cin;
  void* cout;
  // gm as the operand pairs of the packed (f32x2) moment sums: per group
  // (P0, P0^2), (Pv, Pv), (P0 Pv, P0 Pv), (Pv^2, Pv^2), hi pair then lo pair
  float2 gm2[6][8];
  float2 gf2[3][10][2];   // groups (2j, 2j+1): gf hi pair, lo pair
  // site / Nx = (site nx_m) >> nx_sh for 0 <= site < 2^31
  unsigned nx_m;
  int nx_sh;
  // BF16 kernels: sites x in [halo, halo + inner_nx), y in [halo, halo +
  // inner_ny) pull without wrapping; there the bfloat16 value of population
  // i and its coefficient word sit doff[i] / dcoff[i] elements from the
  // site's own slot and word of plane 0.  inner_nx = inner_ny = 0 (every
  // site takes the wrapped pull) when the offsets do not fit 32 bits.
  int inner_nx, inner_ny;
  int doff[kMaxQ2], dcoff[kMaxQ2];
};

// One lattice of a persistent batch launch (device memory; rlbm_persist.cuh).
struct PersistLattice {
  FusedParams p[2];       // step parameters for S_t in buf[0] / buf[1] (BF16 coefficient planes set)
  const void* buf[2];     // population buffers
  int nsite;              // Nx Ny
  int ntiles;             // tiles of 128 spt sites
};

struct PersistParams {
  const PersistLattice* lat;
  const int2* units;      // the units of one step in claim order: (lattice, tile)
  int nlat;
  int units_per_step;
  int nsteps;
  int spt;                // sites per thread
  unsigned spin_limit;    // polls of one wait before it gives up
  unsigned wait_offset;   // added to every wait target (testing the timeout path only)
  unsigned* ticket;       // claim counter, zero at launch
  unsigned* abort;        // nonzero: stop claiming
  unsigned* done;         // per lattice: units completed in this launch, zero at launch
  const int* par0;        // per lattice: buffer holding S_t at launch (0 or 1)
};

// Device error bits (OR-ed into *err).
enum : unsigned {
  ERR_LANDAU = 1u,   // Landau frame: non-finite or |u| >= 1
  ERR_DENSITY = 2u,  // n <= 0 or non-finite
  ERR_EOS = 4u,      // e/n <= m or T <= 0 or non-finite
  ERR_ZETA = 8u,     // zeta outside the tabulated range
  ERR_TIMEOUT = 16u, // a bounded device-side wait ran out (persistent batch)
};

// Fields read by the init kernel and written by the moments kernel.
struct FieldPtrs {
  const double* n;
  const double* ux;
  const double* uy;
  const double* T;
};

struct MomentOut {
  double* out;           // device-accessible buffer (device memory or mapped
                         // page-locked host memory), planes of Nx*Ny doubles
  unsigned mask;
};

// Validation of uploaded initial fields (rlbm_init, rlbm3_init), on the
// device: block b of at most kScanBlocks scans sites [b len, (b+1) len),
// len = ceil(N / blocks); it lowers *bad (set to all ones before) to the
// smallest index violating n > 0, T > 0, |u| < 1 (all finite) and writes
// the FP64 sum of n over its sites, reduced in a fixed order, to part[b]
// (so the total, summed by the host in block order, depends on N only).
// uz may be NULL (2D).
constexpr int kScanBlocks = 1024;
int field_check_blocks(long long N);
cudaError_t launch_field_check(const double* n, const double* ux, const double* uy, const double* uz,
                               const double* T, long long N, double* part, unsigned long long* bad,
                               cudaStream_t s);

// ------------------------------------------------- third-order 2D lattices
// Eleven-group stencils folded onto the xy plane (rlbm_kernels_o3.cu); the
// table layout is described with StencilBuildO3 (rlbm_stencil.h).  Centred
// monomials of the equilibrium polynomial, t = p0 - c:
//   1, t, px, py, t px, t py, px^2, py^2, px py, pz^2, t px^2, t py^2,
//   t px py, px^3, px^2 py, px py^2, py^3, t pz^2, px pz^2, py pz^2
constexpr int kO3Mono = 20;
constexpr int kRowO3 = 32;
constexpr int kMaxPopO3 = 256;

struct O3Params {
  int Nx, Ny, Q, halo;
  long long pitch, plane;     // elements
  double inv_tau;
  double nref;                // FP32 storage holds d_i = f_i - nref wr_i; 0 for FP64
  double mref[9];             // moments of nref wr_i
  double c;                   // centring shift of t
  SiteConsts sc;
  const double* rt64;
  const float* rt32;
  const int* shift;           // [2][Q]: n_x mod Nx, n_y mod Ny
  const long long* off;       // [Q]: -(n_y pitch + n_x), source offset of an interior site
  const double* tab64;        // [Q][kRowO3]
  const float* tab32;         // [Q][kRowO3] (FP32 storage)
  unsigned* err;
};

// Stencil-specialised FP32 third-order step (rlbm_fused_o3.cu): the split
// arithmetic of FusedParams with eleven groups.  Per reflection orbit K of
// the compiled stencil, ow[K] holds the representative (+n_x, +n_y)
// population's wr_i and its twenty dual-basis values W_il (host table row
// entries 9..29, multiplicity included) as hi/lo pairs.
constexpr int kMaxOrbO3 = 44;
struct FusedO3Params {
  int Nx, Ny;
  long long pitch, plane;
  float inv_tau, v0;
  float mb, cv_r, c;
  HL Rr, nr, yr;
  HL mref[9];
  double Rr64, mb64;
  HL gm[11][5];        // per group: P0, P0^2, Pv, P0 Pv, Pv^2
  HL ow[kMaxOrbO3][21];
  const double* rt64;
  const float* rt32;
  const double* dr64;  // DR_NSEG * DR_NC (the lattice's dR(Td) table)
  unsigned* err;
};

// kind 5, 6, 7: groups {1,2,5,6,7,9,10,11,12,13,15}, {2,3,5,6,7,8,9,10,11,13,15},
// {1,2,3,6,7,8,9,10,11,13,15}; 8, 9, 10: {8,15,20,24,26,27,28,30,36,37,42},
// {4,10,15,20,24,26,27,28,30,36,37}, {4,8,14,15,16,17,18,21,22,23,26}
cudaError_t launch_fused_o3(int kind, const FusedO3Params& p, const void* fin, void* fout, cudaStream_t s);

cudaError_t launch_step_o3(rlbm_dtype dt, const O3Params& p, const void* fin, void* fout, cudaStream_t s);
cudaError_t launch_init_o3(rlbm_dtype dt, const O3Params& p, FieldPtrs f, void* cur, void* prev, cudaStream_t s);
cudaError_t launch_moments_o3(rlbm_dtype dt, const O3Params& p, const void* prev, MomentOut o, cudaStream_t s);

// ------------------------------------------------------------ 3D lattices
// Unfolded stencil on an Nx x Ny x Nz periodic lattice (rlbm_kernels3d.cu).
// Per population i, one table row of kRow3 values at [i * kRow3] (16-byte
// aligned for vector loads): entries 0..13 momentum products p0, px, py, pz,
// p0p0, p0px, p0py, p0pz, pxpx, pxpy, pxpz, pypy, pypz, pzpz; 14..27 w_i J of
// App. A in the order 1, J0, Jx, Jy, Jz, J00, J0x, J0y, J0z,
// (py^2-pz^2)/2E, (-2px^2+py^2+pz^2)/(2 sqrt3 E), Jxz, Jyz, Jxy; 28..30
// p^a/p^0; 31 zero.
constexpr int kPop3 = 31;
constexpr int kRow3 = 32;
constexpr int kMaxPop3 = 160;

struct Step3Params {
  int Nx, Ny, Nz, Q;
  long long pitch, plane;     // elements: x pitch; plane = pitch * Ny * Nz (one population)
  double inv_tau;
  double nref;                // FP32 storage holds d_i = f_i - r_i (see StepParams); 0 for FP64
  double b0ref;               // nref K1/K2(mbar)/mbar
  double mref[14];            // moments of r_i (order of the table rows 0..13)
  SiteConsts sc;
  const double* rt64;         // FP64 R(zeta) table
  const float* rt32;          // FP32 R(zeta) table (FP32 storage: solve iterations)
  const int* shift;           // [3][Q]: n_x mod Nx, n_y mod Ny, n_z mod Nz
  const long long* off;       // [Q]: -(n_z Ny pitch + n_y pitch + n_x), the source
                              // element of population i relative to a site at least
                              // halo cells from every face
  int halo;                   // largest |n| component
  const double* tab64;        // [Q][kRow3]
  const float* tab32;         // [Q][kRow3] (FP32 storage)
  unsigned* err;              // sticky device error bits
};

struct Field3Ptrs {
  const double* n;
  const double* ux;
  const double* uy;
  const double* uz;
  const double* T;
};

// Stencil-specialised FP32 3D step (rlbm_fused3d.cu): the split arithmetic of
// FusedParams for the unfolded stencil.  gm: as FusedParams; gf: the ten
// per-group constants of StencilBuild3::gf3.
struct Fused3Params {
  int Nx, Ny, Nz;
  long long pitch, zstride, plane;   // elements; zstride = pitch * Ny
  float inv_tau, v0;
  float mb, k21, cb00_1, mY, cv_r;
  HL Rr, nr, yr;
  HL mref[14];
  double Rr64, mb64;
  HL gm[6][5];
  HL gf[6][10];
  const double* rt64;
  const float* rt32;
  const double* dr64;  // DR_NSEG * DR_NC (the lattice's dR(Td) table)
  unsigned* err;
};

// kind 1..4: groups {5,12,14,17,21,26}, {1..6}, {1,14,49,51,60,70}, {3,9,10,14,17,21}
cudaError_t launch_fused3d(int kind, const Fused3Params& p, const void* fin, void* fout, cudaStream_t s);

cudaError_t launch_step3d(rlbm_dtype dt, const Step3Params& p, const void* fin, void* fout, cudaStream_t s);
cudaError_t launch_init3d(rlbm_dtype dt, const Step3Params& p, Field3Ptrs f, void* cur, void* prev,
                          cudaStream_t s);
cudaError_t launch_moments3d(rlbm_dtype dt, const Step3Params& p, const void* prev, MomentOut o,
                             cudaStream_t s);

// Kernel launchers (rlbm_kernels_*.cu).
cudaError_t launch_step_f64(const StepParams<double>& p, const void* fin, void* fout, int qb,
                            cudaStream_t s);
cudaError_t launch_step_f32(const StepParams<float>& p, const void* fin, void* fout, int qb,
                            cudaStream_t s);
cudaError_t launch_init(rlbm_dtype dt, const StepParams<double>& p, FieldPtrs f, void* cur,
                        void* prev, cudaStream_t s);
cudaError_t launch_moments(rlbm_dtype dt, const StepParams<double>& p, const void* prev,
                           MomentOut mo, cudaStream_t s);

}  // namespace rlbm
