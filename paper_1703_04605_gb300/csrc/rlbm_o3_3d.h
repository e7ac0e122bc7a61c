// Third-order scheme on native 3D lattices (unfolded eleven-group stencils):
// the monomial basis shared by the host builder (rlbm_stencil.cpp) and the
// kernels (rlbm_kernels3d.cu), and the kernels' parameters.  Internal.
#pragma once

#include "rlbm_internal.h"

namespace rlbm {

// The thirty centred monomials t^a p_x^i p_y^j p_z^k (t = p0 - c, a <= 1,
// a + i + j + k <= 3) that span the polynomials of degree <= 3 on the mass
// shell, as (a, i, j, k), lowest degree first.
constexpr int kO3Mono3 = 30;
struct O3Exp3 {
  int e[kO3Mono3][4];
};
constexpr O3Exp3 kO3Exp3 = {{
    {0, 0, 0, 0}, {1, 0, 0, 0},                                     // 1, t
    {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1},                       // p_a
    {1, 1, 0, 0}, {1, 0, 1, 0}, {1, 0, 0, 1},                       // t p_a
    {0, 2, 0, 0}, {0, 0, 2, 0}, {0, 0, 0, 2},                       // p_a p_b
    {0, 1, 1, 0}, {0, 1, 0, 1}, {0, 0, 1, 1},
    {1, 2, 0, 0}, {1, 0, 2, 0}, {1, 0, 0, 2},                       // t p_a p_b
    {1, 1, 1, 0}, {1, 1, 0, 1}, {1, 0, 1, 1},
    {0, 3, 0, 0}, {0, 0, 3, 0}, {0, 0, 0, 3},                       // p_a p_b p_c
    {0, 2, 1, 0}, {0, 2, 0, 1}, {0, 1, 2, 0}, {0, 0, 2, 1},
    {0, 1, 0, 2}, {0, 0, 1, 2}, {0, 1, 1, 1}}};

// Per population i, the dual-basis row W3[i * kRowW3 + l] = w_i (G^-1 phi(p_i))_l
// of the thirty monomials (G their Gram matrix under the weights); the main
// table row (Step3Params::tab64) keeps the momentum products at 0..13, the
// rest-frame weight w_i K1/K2(mbar)/mbar at 14 and p^a/p^0 at 28..30.
constexpr int kRowW3 = 32;

struct Step3O3Params {
  Step3Params b;          // lattice, tables, reference moments, site constants
  double c;               // centring shift mbar K2/K1(mbar)
  const double* w64;      // [Q][kRowW3]
  const float* w32;       // [Q][kRowW3] (FP32 storage)
};

cudaError_t launch_step3d_o3(rlbm_dtype dt, const Step3O3Params& p, const void* fin, void* fout, cudaStream_t s);
cudaError_t launch_init3d_o3(rlbm_dtype dt, const Step3O3Params& p, Field3Ptrs f, void* cur, void* prev,
                             cudaStream_t s);

}  // namespace rlbm
