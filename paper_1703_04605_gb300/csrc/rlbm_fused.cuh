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
//
// Extended moment sums (template flag EX, FP32 storage): the deviation
// moments N^a and K^a = T^0a - m N^a are formed to about 2^-40 relative
// instead of FP32 rounding, because on long runs of steep, sloshing flows
// (massive Sod tubes, thousands of steps) the FP32 rounding of the moment
// sums breaks mass and energy conservation by about one rounding per step
// and site, which adds up.  Each pulled d_i is split exactly into a part h_i
// on a grid of its group (a power of two well below the group's reference
// value) and a remainder l_i = d_i - h_i; sums of the h_i with integer
// weights are exact in FP32, sums of the l_i lose only the rounding of
// numbers 2^11 times smaller, and the six group sums are combined with the
// group constants by error-free products and two-sums (float-float).  The
// kinetic moments K^a are accumulated directly, so the energy above the rest
// mass, e - m n, is formed without the cancellation of e and m n.
//
// BF16 deviation storage (template flag BF; the bfloat16 values of two
// orbit partners share a 32-bit word, StencilDef::B): the stored value is
// d_i = (f_i - r_i) - ref_i(x), rounded to bfloat16, where ref_i(x) =
// mult_i (a + b_x n_x + b_y n_y + q (n_x^2 + n_y^2)) uses the equilibrium
// coefficients of the writing site x for the population's group, rounded to
// bfloat16 and stored beside the populations (four per group and site).  The
// reader rebuilds f_i - r_i = d_i + ref_i(source site) from the same stored
// numbers, so encoding and decoding agree exactly; the rest of the step is the
// FP32 path above.
#pragma once

#include <cuda_bf16.h>
#include <cstring>
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

__device__ __forceinline__ float bf_lo(unsigned u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(unsigned u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ unsigned bf_pack(float lo, float hi) {
  return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
         ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

// bfloat16 bits of a small integer (|k| < 256, exact in bfloat16)
__host__ __device__ constexpr unsigned short bf_int_bits(int k) {
  const unsigned a = k < 0 ? -k : k;
  int e = 0;
  while ((a >> (e + 1)) != 0) ++e;
  return (unsigned short)(((k < 0) ? 0x8000u : 0u) | ((unsigned)(e + 127) << 7) | ((a << (7 - e)) & 0x7fu));
}

// acc + K b with b the bfloat16 in the high (HI) or low half of w: the
// mixed-precision FMA of sm_100+ takes both bfloat16 factors straight from
// the packed word (no unpacking); K b is exact, so the result is the FP32
// fmaf(K, b, acc) bit for bit
template <int K, bool HI>
__device__ __forceinline__ float fma_kbf(unsigned w, float acc) {
  float r;
  if constexpr (HI)
    asm("{ .reg .b16 lo, hi, k; mov.b32 {lo, hi}, %1; mov.b16 k, %2; fma.rn.f32.bf16 %0, k, hi, %3; }"
        : "=f"(r) : "r"(w), "n"((int)bf_int_bits(K)), "f"(acc));
  else
    asm("{ .reg .b16 lo, hi, k; mov.b32 {lo, hi}, %1; mov.b16 k, %2; fma.rn.f32.bf16 %0, k, lo, %3; }"
        : "=f"(r) : "r"(w), "n"((int)bf_int_bits(K)), "f"(acc));
  return r;
}

// bfloat16 h + FP32 acc, one rounding (the FP32 sum of the widened h)
__device__ __forceinline__ float add_bf(unsigned short h, float acc) {
  float r;
  asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(r) : "h"(h), "f"(acc));
  return r;
}

// reference of a population from its group's packed coefficients,
// mult (alpha + |n|^2 q + n_y beta_y + n_x beta_x) in this order, with the
// multiplicity (1 or 2) folded into the exact integer factors: the members
// of a reflection orbit share the first terms, which the encoder evaluates
// once an orbit, and the decoder's chain is the same operation for operation
template <int nx, int ny, int mult>
__device__ __forceinline__ float bf_ref(uint2 c) {
  static_assert(mult == 1 || mult == 2, "folded multiplicities are 1 or 2");
  float r;
  if constexpr (mult == 1) r = bf_lo(c.x);
  else r = fma_kbf<mult, false>(c.x, 0.0f);
  if constexpr (nx * nx + ny * ny != 0) r = fma_kbf<mult * (nx * nx + ny * ny), true>(c.y, r);
  if constexpr (ny != 0) r = fma_kbf<mult * ny, false>(c.y, r);
  if constexpr (nx != 0) r = fma_kbf<mult * nx, true>(c.x, r);
  return r;
}

// CG: loads through L2 only (ld.global.cg), for kernels that read data other
// blocks of the same launch wrote (the read-only path may hold stale lines).
template <bool CG, class T>
__device__ __forceinline__ T fused_ld(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}

// Element indices: a plane holds fewer than 2^32 elements (checked when the
// lattice is created), so the index of a pulled value, y_s pitch + x_s, and
// a plane offset I plane are formed in 32-bit arithmetic; the address is then
// one wide multiply-add from the base, where 64-bit index arithmetic costs
// several integer instructions a population.
template <class Def, bool BF, int I, bool CG = false>
__device__ __forceinline__ void fused_load(float (&d)[Def::Q], const void* __restrict__ fin,
                                           const uint2* __restrict__ cin, long long plane, long long pitch,
                                           int x, int y, int Nx, int Ny) {
  constexpr int DX = Def::F.nx[I], DY = Def::F.ny[I];
  const int xs = wrap_c<DX>(x, Nx);
  const int ys = wrap_c<DY>(y, Ny);
  const unsigned idx = (unsigned)ys * (unsigned)pitch + (unsigned)xs;
  const size_t pl = (unsigned)plane;
  if constexpr (BF) {
    constexpr int g = Def::F.grp[I], mult = Def::F.mult[I], w = Def::B.word[I], hf = Def::B.half[I];
    const unsigned short h =
        fused_ld<CG>(static_cast<const unsigned short*>(fin) + 2 * (size_t)idx + hf + 2 * pl * w);
    const uint2 c = fused_ld<CG>(cin + idx + pl * g);
    d[I] = add_bf(h, bf_ref<DX, DY, mult>(c));
  } else {
    d[I] = fused_ld<CG>(static_cast<const float*>(fin) + idx + pl * I);
  }
}

// The same pull for a site whose sources need no wrapping (BF16 storage):
// the value and its coefficient word sit at fixed offsets from the site's
// own elements (fh: its half-word slot 0 of word plane 0, ch: its
// coefficient word of group 0), which takes the index arithmetic off the path.
template <class Def, int I, bool CG = false>
__device__ __forceinline__ void fused_load_inner(float (&d)[Def::Q], const unsigned short* __restrict__ fh,
                                                 const uint2* __restrict__ ch, const FusedParams& p) {
  constexpr int DX = Def::F.nx[I], DY = Def::F.ny[I], mult = Def::F.mult[I];
  const unsigned short h = fused_ld<CG>(fh + p.doff[I]);
  const uint2 c = fused_ld<CG>(ch + p.dcoff[I]);
  d[I] = add_bf(h, bf_ref<DX, DY, mult>(c));
}

// Group sums of one reflection orbit (members (+,+), (-,+), (+,-), (-,-) of
// |n_x|, |n_y|): s[g] = sum d, sum n_x d, sum n_y d, sum n_x^2 d, sum n_x n_y d,
// sum n_y^2 d, formed from the butterflies d0 +- d1, d2 +- d3.
template <class Def, int K>
__device__ __forceinline__ void fused_acc_orbit(const float (&d)[Def::Q], float (&s)[6][6]) {
  constexpr int kind = Def::O.kind[K], g = Def::O.grp[K], ax = Def::O.ax[K], ay = Def::O.ay[K];
  constexpr int i0 = Def::O.idx[K][0], i1 = Def::O.idx[K][1], i2 = Def::O.idx[K][2], i3 = Def::O.idx[K][3];
  if constexpr (kind == 1) {
    s[g][0] += d[i0];
  } else if constexpr (kind == 2) {
    const float S = d[i0] + d[i1], D = d[i0] - d[i1];
    s[g][0] += S;
    s[g][1] = fmaf((float)ax, D, s[g][1]);
    s[g][3] = fmaf((float)(ax * ax), S, s[g][3]);
  } else if constexpr (kind == 3) {
    const float S = d[i0] + d[i2], D = d[i0] - d[i2];
    s[g][0] += S;
    s[g][2] = fmaf((float)ay, D, s[g][2]);
    s[g][5] = fmaf((float)(ay * ay), S, s[g][5]);
  } else {
    const float p = d[i0] + d[i1], q = d[i0] - d[i1], r = d[i2] + d[i3], w = d[i2] - d[i3];
    const float S = p + r;
    s[g][0] += S;
    s[g][1] = fmaf((float)ax, q + w, s[g][1]);
    s[g][2] = fmaf((float)ay, p - r, s[g][2]);
    s[g][3] = fmaf((float)(ax * ax), S, s[g][3]);
    s[g][4] = fmaf((float)(ax * ay), q - w, s[g][4]);
    s[g][5] = fmaf((float)(ay * ay), S, s[g][5]);
  }
}

// ---------------------------------------------------- extended moment sums
// A value held as the unevaluated sum hi + lo of two FP32 numbers.
struct FF {
  float hi, lo;
};

// a + b = s + e exactly (two-sum; branch-free); the _rn intrinsics keep the
// compiler from contracting or reassociating these operations.
__device__ __forceinline__ float ex_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// acc += (c.hi + c.lo)(xh + xl) with xh exact: the product c.hi xh and its
// addition to acc.hi are error-free; the remaining small terms go to acc.lo.
__device__ __forceinline__ void ex_acc(FF& acc, const HL& c, float xh, float xl) {
  const float p = __fmul_rn(c.hi, xh);
  const float pe = __fmaf_rn(c.hi, xh, -p);
  float se;
  acc.hi = ex_two_sum(acc.hi, p, se);
  acc.lo += (se + pe) + fmaf(c.lo, xh, c.hi * xl);
}

// d = h + l exactly, h on the grid of spacing q, C = 1.5 2^23 q (|d| < 2^22 q)
__device__ __forceinline__ void ex_split(float d, float C, float& h, float& l) {
  h = __fsub_rn(__fadd_rn(d, C), C);
  l = __fsub_rn(d, h);
}

// Running sums of one group: sums of h and of l with weight 1 (k = 0) and,
// at level 2, with weights n_x, n_y (k = 1, 2); plain FP32 sums of d with the
// remaining weights (n_x, n_y at level 1; n_x^2, n_x n_y, n_y^2).
struct ExGroup {
  float h[3], l[3], d[5];
};

// Moments of the extended path: N^0 and K^0 (and, at level 2, N^x, N^y, K^x,
// K^y) as float-float, the others in FP32 (all deviations: the reference r_i
// excluded).
struct ExMoments {
  FF N0, Nx, Ny, K0, Kx, Ky;
  float Txx, Txy, Tyy;
};

// Level L = 1: N^0 and K^0 extended (mass and energy, the quantities whose
// drift the sloshing tubes amplify); L = 2: also momentum and its flux.
template <class Def, int L, int K>
__device__ __forceinline__ void ex_acc_orbit(const float (&d)[Def::Q], const float (&C)[6], ExGroup& s) {
  constexpr int kind = Def::O.kind[K], g = Def::O.grp[K], ax = Def::O.ax[K], ay = Def::O.ay[K];
  constexpr int i0 = Def::O.idx[K][0], i1 = Def::O.idx[K][1], i2 = Def::O.idx[K][2], i3 = Def::O.idx[K][3];
  if constexpr (kind == 1) {
    float h, l;
    ex_split(d[i0], C[g], h, l);
    s.h[0] = __fadd_rn(s.h[0], h);
    s.l[0] += l;
  } else if constexpr (kind == 2 || kind == 3) {
    constexpr int j1 = kind == 2 ? i1 : i2;
    constexpr int a = kind == 2 ? ax : ay;
    constexpr int k = kind == 2 ? 1 : 2;
    float h0, l0, h1, l1;
    ex_split(d[i0], C[g], h0, l0);
    ex_split(d[j1], C[g], h1, l1);
    const float Sh = __fadd_rn(h0, h1), Sl = l0 + l1;
    s.h[0] = __fadd_rn(s.h[0], Sh);
    s.l[0] += Sl;
    if constexpr (L >= 2) {
      s.h[k] = __fmaf_rn((float)a, __fsub_rn(h0, h1), s.h[k]);
      s.l[k] = fmaf((float)a, l0 - l1, s.l[k]);
    } else {
      s.d[k - 1] = fmaf((float)a, d[i0] - d[j1], s.d[k - 1]);
    }
    const float S = Sh + Sl;
    s.d[kind == 2 ? 2 : 4] = fmaf((float)(a * a), S, s.d[kind == 2 ? 2 : 4]);
  } else {
    float h[4], l[4];
    ex_split(d[i0], C[g], h[0], l[0]);
    ex_split(d[i1], C[g], h[1], l[1]);
    ex_split(d[i2], C[g], h[2], l[2]);
    ex_split(d[i3], C[g], h[3], l[3]);
    const float ph = __fadd_rn(h[0], h[1]), rh = __fadd_rn(h[2], h[3]);
    const float pl = l[0] + l[1], rl = l[2] + l[3];
    const float Sh = __fadd_rn(ph, rh), Sl = pl + rl;
    s.h[0] = __fadd_rn(s.h[0], Sh);
    s.l[0] += Sl;
    const float q = d[i0] - d[i1], w = d[i2] - d[i3];
    if constexpr (L >= 2) {
      const float qh = __fsub_rn(h[0], h[1]), wh = __fsub_rn(h[2], h[3]);
      const float ql = l[0] - l[1], wl = l[2] - l[3];
      s.h[1] = __fmaf_rn((float)ax, __fadd_rn(qh, wh), s.h[1]);
      s.h[2] = __fmaf_rn((float)ay, __fsub_rn(ph, rh), s.h[2]);
      s.l[1] = fmaf((float)ax, ql + wl, s.l[1]);
      s.l[2] = fmaf((float)ay, pl - rl, s.l[2]);
    } else {
      const float p = d[i0] + d[i1], r = d[i2] + d[i3];
      s.d[0] = fmaf((float)ax, q + w, s.d[0]);
      s.d[1] = fmaf((float)ay, p - r, s.d[1]);
    }
    const float S = Sh + Sl;
    s.d[2] = fmaf((float)(ax * ax), S, s.d[2]);
    s.d[3] = fmaf((float)(ax * ay), q - w, s.d[3]);
    s.d[4] = fmaf((float)(ay * ay), S, s.d[4]);
  }
}

// Last orbit of its group (the orbits run group by group).
template <class Def, int K>
__host__ __device__ constexpr bool ex_group_ends() {
  return K + 1 == Def::O.K || Def::O.grp[K + 1] != Def::O.grp[K];
}

// Orbit K, then, at the end of a group, that group's sums into the moments.
template <class Def, int L, int K>
__device__ __forceinline__ void ex_orbit_step(const float (&d)[Def::Q], const FusedParams& p,
                                              const float (&C)[6], ExGroup& s, ExMoments& M) {
  ex_acc_orbit<Def, L, K>(d, C, s);
  if constexpr (ex_group_ends<Def, K>()) {
    constexpr int g = Def::O.grp[K];
    ex_acc(M.N0, p.gm[g][0], s.h[0], s.l[0]);
    ex_acc(M.K0, p.gk[g][0], s.h[0], s.l[0]);
    if constexpr (L >= 2) {
      ex_acc(M.Nx, p.gm[g][2], s.h[1], s.l[1]);
      ex_acc(M.Kx, p.gk[g][1], s.h[1], s.l[1]);
      ex_acc(M.Ny, p.gm[g][2], s.h[2], s.l[2]);
      ex_acc(M.Ky, p.gk[g][1], s.h[2], s.l[2]);
    } else {
      M.Nx.hi = hl_fma(p.gm[g][2], s.d[0], M.Nx.hi);
      M.Kx.hi = hl_fma(p.gk[g][1], s.d[0], M.Kx.hi);
      M.Ny.hi = hl_fma(p.gm[g][2], s.d[1], M.Ny.hi);
      M.Ky.hi = hl_fma(p.gk[g][1], s.d[1], M.Ky.hi);
    }
    M.Txx = hl_fma(p.gm[g][4], s.d[2], M.Txx);
    M.Txy = hl_fma(p.gm[g][4], s.d[3], M.Txy);
    M.Tyy = hl_fma(p.gm[g][4], s.d[4], M.Tyy);
#pragma unroll
    for (int k = 0; k < 3; ++k) s.h[k] = s.l[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < 5; ++k) s.d[k] = 0.0f;
  }
}

template <class Def, int L, int... Ks>
__device__ __forceinline__ void ex_acc_all(std::integer_sequence<int, Ks...>, const float (&d)[Def::Q],
                                           const FusedParams& p, ExMoments& M) {
  float C[6];
#pragma unroll
  for (int g = 0; g < 6; ++g) C[g] = p.exC[g];
  ExGroup s;
#pragma unroll
  for (int k = 0; k < 3; ++k) s.h[k] = s.l[k] = 0.0f;
#pragma unroll
  for (int k = 0; k < 5; ++k) s.d[k] = 0.0f;
  (ex_orbit_step<Def, L, Ks>(d, p, C, s, M), ...);
}

// Relaxation and store of population I with equilibrium value e (f^eq - r).
template <class Def, bool BF, int I>
__device__ __forceinline__ void fused_relax(const float (&d)[Def::Q], float e, const uint2 (&cq)[6], float a0,
                                            float ax, float ay, void* __restrict__ out, long long plane) {
  constexpr int g = Def::F.grp[I], nx = Def::F.nx[I], ny = Def::F.ny[I], mult = Def::F.mult[I];
  // weight p_i.U/(p_i^0 tau) = (U0 - v0 (nx Ux + ny Uy))/tau
  float om = a0;
  if constexpr (nx != 0) om = fmaf(-(float)nx, ax, om);
  if constexpr (ny != 0) om = fmaf(-(float)ny, ay, om);
  const float v = d[I];
  const float vn = fmaf(om, e - v, v);
  const size_t pl = (unsigned)plane;
  if constexpr (BF) {
    // a population without an orbit partner: its own half of its word
    constexpr int w = Def::B.word[I], hf = Def::B.half[I];
    const float dv = vn - bf_ref<nx, ny, mult>(cq[g]);
    __stcs(static_cast<unsigned short*>(out) + 2 * pl * w + hf, __bfloat16_as_ushort(__float2bfloat16_rn(dv)));
  } else {
    __stcs(static_cast<float*>(out) + pl * I, vn);
  }
}

// BF16 storage: relaxation of the orbit partners I, J (one word, I in its low
// half) and one conversion and store of the pair; R2: the arithmetic as
// packed pairs (each lane the scalar operations)
template <class Def, int I, int J, bool R2>
__device__ __forceinline__ void bf_relax_pair(const float (&d)[Def::Q], float eI, float eJ, const uint2 (&cq)[6],
                                              float a0, float ax, float ay, void* __restrict__ out,
                                              long long plane) {
  constexpr int g = Def::F.grp[I], nxI = Def::F.nx[I], nyI = Def::F.ny[I], nxJ = Def::F.nx[J],
                nyJ = Def::F.ny[J], mult = Def::F.mult[I];
  static_assert(Def::B.word[I] == Def::B.word[J] && Def::B.half[I] == 0 && Def::B.half[J] == 1,
                "orbit partners share a word, the first in its low half");
  float omI = a0, omJ = a0;
  if constexpr (nxI != 0) omI = fmaf(-(float)nxI, ax, omI);
  if constexpr (nyI != 0) omI = fmaf(-(float)nyI, ay, omI);
  if constexpr (nxJ != 0) omJ = fmaf(-(float)nxJ, ax, omJ);
  if constexpr (nyJ != 0) omJ = fmaf(-(float)nyJ, ay, omJ);
  const float rI = bf_ref<nxI, nyI, mult>(cq[g]), rJ = bf_ref<nxJ, nyJ, mult>(cq[g]);
  float2 dv;
  if constexpr (R2) {
    const float2 v = make_float2(d[I], d[J]);
    const float2 t = __ffma2_rn(v, make_float2(-1.0f, -1.0f), make_float2(eI, eJ));   // e - v
    const float2 vn = __ffma2_rn(make_float2(omI, omJ), t, v);
    dv = __ffma2_rn(make_float2(rI, rJ), make_float2(-1.0f, -1.0f), vn);
  } else {
    const float vI = d[I], vJ = d[J];
    dv = make_float2(fmaf(omI, eI - vI, vI) - rI, fmaf(omJ, eJ - vJ, vJ) - rJ);
  }
  const __nv_bfloat162 b = __floats2bfloat162_rn(dv.x, dv.y);   // .x: low half
  unsigned word;
  memcpy(&word, &b, sizeof word);
  __stcs(static_cast<unsigned*>(out) + (size_t)(unsigned)plane * Def::B.word[I], word);
}

// Relaxation of two members I, J of an orbit as packed pairs (each lane the
// scalar fused_relax's operations)
template <class Def, bool BF, int I, int J>
__device__ __forceinline__ void fused_relax2(const float (&d)[Def::Q], float eI, float eJ, const uint2 (&cq)[6],
                                             float a0, float ax, float ay, void* __restrict__ out,
                                             long long plane) {
  constexpr int g = Def::F.grp[I], nxI = Def::F.nx[I], nyI = Def::F.ny[I], nxJ = Def::F.nx[J],
                nyJ = Def::F.ny[J], mult = Def::F.mult[I];
  float omI = a0, omJ = a0;
  if constexpr (nxI != 0) omI = fmaf(-(float)nxI, ax, omI);
  if constexpr (nyI != 0) omI = fmaf(-(float)nyI, ay, omI);
  if constexpr (nxJ != 0) omJ = fmaf(-(float)nxJ, ax, omJ);
  if constexpr (nyJ != 0) omJ = fmaf(-(float)nyJ, ay, omJ);
  const float2 v = make_float2(d[I], d[J]);
  const float2 t = __ffma2_rn(v, make_float2(-1.0f, -1.0f), make_float2(eI, eJ));   // e - v
  const float2 vn = __ffma2_rn(make_float2(omI, omJ), t, v);
  static_assert(!BF, "BF16 pairs go through bf_relax_pair");
  (void)cq;
  (void)mult;
  (void)g;
  const size_t pl = (unsigned)plane;
  __stcs(static_cast<float*>(out) + pl * I, vn.x);
  __stcs(static_cast<float*>(out) + pl * J, vn.y);
}

// Equilibrium of one reflection orbit: the group polynomial
// mult (c0 + c1 n_x + c2 n_y + c3 n_x^2 + c4 n_y^2 + c5 n_x n_y) split into the
// part even in both n_x and n_y and the odd terms the members share.
template <class Def, bool BF, int K, bool R2 = false>
__device__ __forceinline__ void fused_collide_orbit(const float (&d)[Def::Q], const float (&c)[6][6],
                                                    const uint2 (&cq)[6], float a0, float ax_, float ay_,
                                                    void* __restrict__ out, long long plane) {
  constexpr int kind = Def::O.kind[K], g = Def::O.grp[K], ax = Def::O.ax[K], ay = Def::O.ay[K];
  constexpr int i0 = Def::O.idx[K][0], i1 = Def::O.idx[K][1], i2 = Def::O.idx[K][2], i3 = Def::O.idx[K][3];
  constexpr float m = (float)Def::O.mult[K];
  float E0 = m * c[g][0];
  if constexpr (ax != 0) E0 = fmaf(m * (float)(ax * ax), c[g][3], E0);
  if constexpr (ay != 0) E0 = fmaf(m * (float)(ay * ay), c[g][4], E0);
  if constexpr (kind == 1) {
    fused_relax<Def, BF, i0>(d, E0, cq, a0, ax_, ay_, out, plane);
  } else if constexpr (BF && kind == 2) {
    const float X = (m * (float)ax) * c[g][1];
    bf_relax_pair<Def, i0, i1, R2>(d, E0 + X, E0 - X, cq, a0, ax_, ay_, out, plane);
  } else if constexpr (BF && kind == 3) {
    const float Y = (m * (float)ay) * c[g][2];
    bf_relax_pair<Def, i0, i2, R2>(d, E0 + Y, E0 - Y, cq, a0, ax_, ay_, out, plane);
  } else if constexpr (BF) {
    const float X = (m * (float)ax) * c[g][1], Y = (m * (float)ay) * c[g][2];
    const float Z = (m * (float)(ax * ay)) * c[g][5];
    const float EP = E0 + Z, EM = E0 - Z, XP = X + Y, XM = X - Y;
    bf_relax_pair<Def, i0, i3, R2>(d, EP + XP, EP - XP, cq, a0, ax_, ay_, out, plane);
    bf_relax_pair<Def, i1, i2, R2>(d, EM - XM, EM + XM, cq, a0, ax_, ay_, out, plane);
  } else if constexpr (kind == 2) {
    const float X = (m * (float)ax) * c[g][1];
    if constexpr (R2) {
      fused_relax2<Def, BF, i0, i1>(d, E0 + X, E0 - X, cq, a0, ax_, ay_, out, plane);
    } else {
      fused_relax<Def, BF, i0>(d, E0 + X, cq, a0, ax_, ay_, out, plane);
      fused_relax<Def, BF, i1>(d, E0 - X, cq, a0, ax_, ay_, out, plane);
    }
  } else if constexpr (kind == 3) {
    const float Y = (m * (float)ay) * c[g][2];
    if constexpr (R2) {
      fused_relax2<Def, BF, i0, i2>(d, E0 + Y, E0 - Y, cq, a0, ax_, ay_, out, plane);
    } else {
      fused_relax<Def, BF, i0>(d, E0 + Y, cq, a0, ax_, ay_, out, plane);
      fused_relax<Def, BF, i2>(d, E0 - Y, cq, a0, ax_, ay_, out, plane);
    }
  } else {
    const float X = (m * (float)ax) * c[g][1], Y = (m * (float)ay) * c[g][2];
    const float Z = (m * (float)(ax * ay)) * c[g][5];
    const float EP = E0 + Z, EM = E0 - Z, XP = X + Y, XM = X - Y;
    if constexpr (R2) {
      fused_relax2<Def, BF, i0, i3>(d, EP + XP, EP - XP, cq, a0, ax_, ay_, out, plane);
      fused_relax2<Def, BF, i1, i2>(d, EM - XM, EM + XM, cq, a0, ax_, ay_, out, plane);
    } else {
      fused_relax<Def, BF, i0>(d, EP + XP, cq, a0, ax_, ay_, out, plane);
      fused_relax<Def, BF, i1>(d, EM - XM, cq, a0, ax_, ay_, out, plane);
      fused_relax<Def, BF, i2>(d, EM + XM, cq, a0, ax_, ay_, out, plane);
      fused_relax<Def, BF, i3>(d, EP - XP, cq, a0, ax_, ay_, out, plane);
    }
  }
}

template <class Def, bool CG = false, int... Is>
__device__ __forceinline__ void fused_load_inner_all(std::integer_sequence<int, Is...>, float (&d)[Def::Q],
                                                     const unsigned short* __restrict__ fh,
                                                     const uint2* __restrict__ ch, const FusedParams& p) {
  static_assert(Def::Q <= kMaxQ2, "offset tables hold kMaxQ2 populations");
  (fused_load_inner<Def, Is, CG>(d, fh, ch, p), ...);
}

template <class Def, bool BF, bool CG = false, int... Is>
__device__ __forceinline__ void fused_load_all(std::integer_sequence<int, Is...>, float (&d)[Def::Q],
                                               const void* __restrict__ fin, const uint2* __restrict__ cin,
                                               long long plane, long long pitch, int x, int y, int Nx, int Ny) {
  (fused_load<Def, BF, Is, CG>(d, fin, cin, plane, pitch, x, y, Nx, Ny), ...);
}

template <class Def, int... Ks>
__device__ __forceinline__ void fused_acc_all(std::integer_sequence<int, Ks...>, const float (&d)[Def::Q],
                                              float (&s)[6][6]) {
  (fused_acc_orbit<Def, Ks>(d, s), ...);
}

template <class Def, bool BF, bool R2, int... Ks>
__device__ __forceinline__ void fused_collide_all(std::integer_sequence<int, Ks...>, const float (&d)[Def::Q],
                                                  const float (&c)[6][6], const uint2 (&cq)[6], float a0,
                                                  float ax, float ay, void* __restrict__ out, long long plane) {
  (fused_collide_orbit<Def, BF, Ks, R2>(d, c, cq, a0, ax, ay, out, plane), ...);
}

// Per-population forms of the two loops (the stencil's reflection orbits are
// not used): fewer values live at once, which the 96-register FP32 kernel of
// stencils with 50 <= Q <= 64 needs to avoid spills.
template <class Def, int I>
__device__ __forceinline__ void fused_acc_pop(const float (&d)[Def::Q], float (&s)[6][6]) {
  constexpr int g = Def::F.grp[I], nx = Def::F.nx[I], ny = Def::F.ny[I];
  const float v = d[I];
  s[g][0] += v;
  if constexpr (nx != 0) s[g][1] = fmaf((float)nx, v, s[g][1]);
  if constexpr (ny != 0) s[g][2] = fmaf((float)ny, v, s[g][2]);
  if constexpr (nx != 0) s[g][3] = fmaf((float)(nx * nx), v, s[g][3]);
  if constexpr (nx != 0 && ny != 0) s[g][4] = fmaf((float)(nx * ny), v, s[g][4]);
  if constexpr (ny != 0) s[g][5] = fmaf((float)(ny * ny), v, s[g][5]);
}

template <class Def, bool BF, int I>
__device__ __forceinline__ void fused_collide_pop(const float (&d)[Def::Q], const float (&c)[6][6],
                                                  const uint2 (&cq)[6], float a0, float ax, float ay,
                                                  void* __restrict__ out, long long plane) {
  constexpr int g = Def::F.grp[I], nx = Def::F.nx[I], ny = Def::F.ny[I], mult = Def::F.mult[I];
  float e = c[g][0];
  if constexpr (nx != 0) e = fmaf((float)nx, c[g][1], e);
  if constexpr (ny != 0) e = fmaf((float)ny, c[g][2], e);
  if constexpr (nx != 0) e = fmaf((float)(nx * nx), c[g][3], e);
  if constexpr (ny != 0) e = fmaf((float)(ny * ny), c[g][4], e);
  if constexpr (nx != 0 && ny != 0) e = fmaf((float)(nx * ny), c[g][5], e);
  if constexpr (mult != 1) e *= (float)mult;
  fused_relax<Def, BF, I>(d, e, cq, a0, ax, ay, out, plane);
}

// Packed (f32x2) forms of the coefficient formulas (groups in pairs) and of
// the relaxation (orbit members in pairs), and the site division by a
// multiplier: chosen per compiled stencil and storage from measurements on
// GB300.  Each is a few per cent faster on some kernels and slower on others,
// where it changes the register allocation.  Q identifies the stencil: 58
// M1, 39 G1..G6, 73 E5, 49 S2.
template <class Def, bool BF, int EXL>
struct FusedForms {
  static constexpr int Q = Def::Q;
  static constexpr bool coeffs2 = BF ? true : EXL ? (Q == 39 || Q == 49) : (Q != 73);
  static constexpr bool relax2 = BF ? (Q == 39 || Q == 49) : EXL ? false : (Q == 39 || Q == 73);
  static constexpr bool magic_div = Q == 73 || (EXL && (Q == 39 || Q == 49));
};

// Orbit form or per-population form, chosen per kernel from measurements on
// GB300: the orbit form saves about 5 instructions per population (E5 FP32
// and S2 FP32/BF16 3-4 % faster) but keeps more values live, which makes the
// 96-register FP32 kernel of M1 (Q = 58) spill and run 23 % slower.
template <class Def, bool BF>
__host__ __device__ constexpr bool fused_use_orbits() {
  return BF || Def::Q < 50 || Def::Q > 64;
}

template <class Def, int... Is>
__device__ __forceinline__ void fused_acc_pop_all(std::integer_sequence<int, Is...>, const float (&d)[Def::Q],
                                                  float (&s)[6][6]) {
  (fused_acc_pop<Def, Is>(d, s), ...);
}

template <class Def, bool BF, int... Is>
__device__ __forceinline__ void fused_collide_pop_all(std::integer_sequence<int, Is...>, const float (&d)[Def::Q],
                                                      const float (&c)[6][6], const uint2 (&cq)[6], float a0,
                                                      float ax, float ay, void* __restrict__ out, long long plane) {
  (fused_collide_pop<Def, BF, Is>(d, c, cq, a0, ax, ay, out, plane), ...);
}

// dR(Td) from the R(zeta) table, for temperatures outside the lattice's dR
// table (out of line: rare, and it keeps the common path's registers free).
static __device__ __noinline__ double dr_from_zeta(float Td, double mb64, double Rr64, const double* __restrict__ rt64,
                                            unsigned& fl) {
  const float Tf = 1.0f + Td;
  const double T64 = 1.0 + (double)Td;
  double iT = (double)__fdividef(1.0f, Tf);
  iT = fma(iT, fma(-T64, iT, 1.0), iT);
  return ratio64(mb64 * iT, rt64, fl) - Rr64;
}

// Site solve of the split arithmetic (see the header comment): from the
// deviation moments M (reference excluded) to U, n = n_r + n_d and
// T = 1 + T_d, R = R(mbar) + dR.  Landau frame by FP32 Newton on the full
// moments; EOS by FP32 Newton on the deviations and one FP64 Newton step with
// the FP64 R(zeta) table.
struct SplitSite {
  float dg, U0, Ux, Uy, n, nd, Td, dR, R, T;
};

// P: FusedParams or FusedO3Params (fields mref, nr, yr, Rr, mb, cv_r, mb64,
// Rr64, rt64, rt32).
// With EX, em holds the extended moments (M their FP32 roundings): the
// density deviation and e - m n are formed from them (see ExMoments).
template <bool EX = false, class P>
__device__ __forceinline__ SplitSite split_solve(const P& p, const float (&M)[9], unsigned& fl,
                                                 const ExMoments* em = nullptr) {
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
      // quadratic convergence: after a step below 1e-4 the error is of
      // order its square, below the FP32 rounding of v
      if (fabsf(dvx) + fabsf(dvy) < 1e-4f) break;
    }
  }
  const float v2 = vx * vx + vy * vy;
  if (!(v2 < 1.0f)) fl |= ERR_LANDAU;
  const float sq = sqrtf(1.0f - v2);
  const float dg = __fdividef(v2, sq * (1.0f + sq));  // gamma - 1
  const float U0 = 1.0f + dg, Ux = U0 * vx, Uy = U0 * vy;
  // n = U.N = n_r + n_d
  float Xi;
  if constexpr (EX) Xi = em->N0.hi + ((em->N0.lo - vx * M[1]) - vy * M[2]);
  else Xi = M[0] - vx * M[1] - vy * M[2];
  const float nd = fmaf(dg, p.nr.lo, fmaf(dg, Xi + p.nr.hi, Xi));
  const float n = p.nr.hi + (p.nr.lo + nd);
  if (!(n > 0.0f)) fl |= ERR_DENSITY;
  // e/n = y_r + y_d
  float yd;
  if constexpr (EX) {
    // W = e - m n = U0^2 (K^0 - 2 v.K + v.T.v) + m U0 ((U0 - 1) N^0 - (2 U0 - 1) v.N)
    // (no term cancels e against m n), formed as its deviation from the
    // reference W_r = K^0_r = y_r n_r (y = W/n): W - W_r = U0^2 (K^0_d -
    // 2 v.K + v.T.v) + dg (2 + dg) K^0_r + m U0 (...), so that FP32 rounding
    // is relative to deviations, as in the plain path
    const float K0d = em->K0.hi + em->K0.lo;
    const float Kx = em->Kx.hi + em->Kx.lo, Ky = em->Ky.hi + em->Ky.lo;
    const float Txx = p.mref[6].hi + (p.mref[6].lo + M[6]);
    const float Tyy = p.mref[8].hi + (p.mref[8].lo + M[8]);
    const float vTv = fmaf(vx * vx, Txx, fmaf(2.0f * vx * vy, M[7], vy * vy * Tyy));
    const float kd = fmaf(-2.0f, fmaf(vx, Kx, vy * Ky), K0d) + vTv;
    const float N0 = p.nr.hi + ((p.nr.lo + em->N0.hi) + em->N0.lo);
    const float vN = fmaf(vx, M[1], vy * M[2]);
    const float U02m1 = dg * (2.0f + dg);
    const float Wd = fmaf(U0 * U0, kd, fmaf(U02m1, p.k0r.hi, U02m1 * p.k0r.lo)) +
                     p.mb * U0 * fmaf(dg, N0, -fmaf(2.0f, dg, 1.0f) * vN);
    yd = __fdividef(Wd - fmaf(p.ykr.hi, nd, p.ykr.lo * nd), n);
  } else {
    const float ed = M[3] - M[4] * vx - M[5] * vy;
    yd = __fdividef(ed - fmaf(p.yr.hi, nd, p.yr.lo * nd), n);
  }
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
    // the FP64 step below squares the remaining error again
    if (fabsf(step) < 1e-4f) break;
  }
  // ... and one FP64 Newton step: dR(Td) from the lattice's FP64 table in
  // Td (no reciprocal, no reference subtraction), else from the R(zeta) table
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
  SplitSite o;
  o.dg = dg;
  o.U0 = U0;
  o.Ux = Ux;
  o.Uy = Uy;
  o.n = n;
  o.nd = nd;
  o.Td = Td;
  o.dR = dR;
  o.R = R;
  o.T = T;
  return o;
}

// Group coefficients c[g] of f^eq - r (the polynomial mult (c0 + c1 n_x +
// c2 n_y + c3 n_x^2 + c4 n_y^2 + c5 n_x n_y) of each group) from the split
// site state: the App. B projections in deviation form, without their
// normalisations (those and the App. A constants are folded into p.gf).
template <bool C2 = false>
__device__ __forceinline__ void fused_coeffs(const FusedParams& p, const SplitSite& ss, float (&c)[6][6]) {
  const float dg = ss.dg, Ux = ss.Ux, Uy = ss.Uy, n = ss.n, nd = ss.nd;
  const float Td = ss.Td, dR = ss.dR, R = ss.R, T = ss.T;
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
  if constexpr (C2) {
    // groups (2j, 2j + 1) as packed pairs; each lane is the scalar form below
    const float r78 = r7 - r8;
    const float2 R0 = make_float2(r0, r0), R1 = make_float2(r1, r1), R2 = make_float2(r2, r2);
    const float2 R3 = make_float2(r3, r3), R4 = make_float2(r4, r4), R5 = make_float2(r5, r5);
    const float2 R6 = make_float2(r6, r6), R7 = make_float2(r7, r7), R8 = make_float2(r8, r8);
    const float2 R9 = make_float2(r9, r9), R78 = make_float2(r78, r78);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float2(*a)[2] = p.gf2[j];   // a[q][0]: hi pair, a[q][1]: lo pair
      float2 al = __ffma2_rn(a[0][0], R0, __fmul2_rn(a[0][1], R0));
      al = __ffma2_rn(a[1][0], R1, __ffma2_rn(a[1][1], R1, al));
      al = __ffma2_rn(a[2][0], R4, __ffma2_rn(a[2][1], R4, al));
      al = __ffma2_rn(a[3][0], R7, __ffma2_rn(a[3][1], R7, al));
      al = __ffma2_rn(a[4][0], R8, __ffma2_rn(a[4][1], R8, al));
      const float2 h5 = __ffma2_rn(a[6][0], R5, __fmul2_rn(a[6][1], R5));
      const float2 h6 = __ffma2_rn(a[6][0], R6, __fmul2_rn(a[6][1], R6));
      const float2 b1 = __ffma2_rn(a[5][0], R2, __ffma2_rn(a[5][1], R2, h5));
      const float2 b2 = __ffma2_rn(a[5][0], R3, __ffma2_rn(a[5][1], R3, h6));
      const float2 q3 = __ffma2_rn(a[7][0], R78, __fmul2_rn(a[7][1], R78));
      const float2 q4 = __ffma2_rn(a[8][0], R7, __fmul2_rn(a[8][1], R7));
      const float2 q5 = __ffma2_rn(a[9][0], R9, __fmul2_rn(a[9][1], R9));
      const float2 cc[6] = {al, b1, b2, q3, q4, q5};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        c[2 * j][k] = cc[k].x;
        c[2 * j + 1][k] = cc[k].y;
      }
    }
  } else {
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
  }
}

// One site update (see the header comment); p describes the lattice.
template <class Def, bool BF, int EXL = 0, bool CG = false>
__device__ __forceinline__ void fused_site(const FusedParams& p, const void* __restrict__ fin,
                                           void* __restrict__ fout, int site, unsigned& fl) {
  static_assert(!(BF && EXL), "extended moment sums are for FP32 storage");
  constexpr int Q = Def::Q;
  using Seq = std::make_integer_sequence<int, Q>;
  {
    int x, y;
    if constexpr (FusedForms<Def, BF, EXL>::magic_div) {
      // y = site / Nx by the multiplier of the lattice (exact for site < 2^31)
      y = (int)(((unsigned long long)(unsigned)site * p.nx_m) >> p.nx_sh);
      x = site - y * p.Nx;
    } else {
      site_of(site, p.Nx, x, y);
    }
    float d[Q];
    const unsigned here = (unsigned)y * (unsigned)p.pitch + (unsigned)x;
    if constexpr (BF) {
      constexpr int H = Def::halo;
      if ((unsigned)(x - H) < (unsigned)p.inner_nx && (unsigned)(y - H) < (unsigned)p.inner_ny)
        fused_load_inner_all<Def, CG>(Seq{}, d, static_cast<const unsigned short*>(fin) + 2 * (size_t)here,
                                      static_cast<const uint2*>(p.cin) + here, p);
      else
        fused_load_all<Def, true, CG>(Seq{}, d, fin, static_cast<const uint2*>(p.cin), p.plane, p.pitch, x, y,
                                      p.Nx, p.Ny);
    } else {
      fused_load_all<Def, BF, CG>(Seq{}, d, fin, static_cast<const uint2*>(p.cin), p.plane, p.pitch, x, y, p.Nx,
                                  p.Ny);
    }
    using Orb = std::make_integer_sequence<int, Def::O.K>;
    // deviation moments N0 Nx Ny T00 T0x T0y Txx Txy Tyy (reference excluded)
    float M[9];
    SplitSite ss;
    if constexpr (EXL > 0) {
      ExMoments em;
      em.N0 = em.Nx = em.Ny = em.K0 = em.Kx = em.Ky = FF{0.0f, 0.0f};
      em.Txx = em.Txy = em.Tyy = 0.0f;
      ex_acc_all<Def, EXL>(Orb{}, d, p, em);
      M[0] = em.N0.hi + em.N0.lo;
      M[1] = em.Nx.hi + em.Nx.lo;
      M[2] = em.Ny.hi + em.Ny.lo;
      M[3] = fmaf(p.mb, M[0], em.K0.hi + em.K0.lo);
      M[4] = fmaf(p.mb, M[1], em.Kx.hi + em.Kx.lo);
      M[5] = fmaf(p.mb, M[2], em.Ky.hi + em.Ky.lo);
      M[6] = em.Txx;
      M[7] = em.Txy;
      M[8] = em.Tyy;
      ss = split_solve<true>(p, M, fl, &em);
    } else {
      float s[6][6];
#pragma unroll
      for (int g = 0; g < 6; ++g)
#pragma unroll
        for (int k = 0; k < 6; ++k) s[g][k] = 0.0f;
      if constexpr (fused_use_orbits<Def, BF>()) fused_acc_all<Def>(Orb{}, d, s);
      else fused_acc_pop_all<Def>(Seq{}, d, s);
      // M = sum_g gm[g] s[g] in hi/lo form; eight of the nine sums as four
      // packed pairs (each lane the same two fmaf as the scalar form)
      float2 A = make_float2(0.0f, 0.0f), B = A, C = A, D = A;
      M[8] = 0.0f;
#pragma unroll
      for (int g = 0; g < 6; ++g) {
        const float2 s00 = make_float2(s[g][0], s[g][0]), s12 = make_float2(s[g][1], s[g][2]);
        const float2 s34 = make_float2(s[g][3], s[g][4]);
        A = __ffma2_rn(p.gm2[g][0], s00, __ffma2_rn(p.gm2[g][1], s00, A));   // N0, T00
        B = __ffma2_rn(p.gm2[g][2], s12, __ffma2_rn(p.gm2[g][3], s12, B));   // Nx, Ny
        C = __ffma2_rn(p.gm2[g][4], s12, __ffma2_rn(p.gm2[g][5], s12, C));   // T0x, T0y
        D = __ffma2_rn(p.gm2[g][6], s34, __ffma2_rn(p.gm2[g][7], s34, D));   // Txx, Txy
        M[8] = hl_fma(p.gm[g][4], s[g][5], M[8]);                            // Tyy
      }
      M[0] = A.x;
      M[3] = A.y;
      M[1] = B.x;
      M[2] = B.y;
      M[4] = C.x;
      M[5] = C.y;
      M[6] = D.x;
      M[7] = D.y;
      ss = split_solve(p, M, fl);
    }
    const float U0 = ss.U0, Ux = ss.Ux, Uy = ss.Uy;
    float c[6][6];
    fused_coeffs<FusedForms<Def, BF, EXL>::coeffs2>(p, ss, c);
    const float a0 = U0 * p.inv_tau, ax = p.v0 * Ux * p.inv_tau, ay = p.v0 * Uy * p.inv_tau;
    uint2 cq[6];
    if constexpr (BF) {
      // this site's reference coefficients, rounded once and stored for the readers
      const size_t pl = (unsigned)p.plane;
#pragma unroll
      for (int g = 0; g < 6; ++g) {
        cq[g].x = bf_pack(c[g][0], c[g][1]);
        cq[g].y = bf_pack(c[g][2], 0.5f * (c[g][3] + c[g][4]));
        __stcs(static_cast<uint2*>(p.cout) + here + pl * g, cq[g]);
      }
    }
    // BF16: the site's word of word plane 0 (two bfloat16 halves)
    void* out = BF ? static_cast<void*>(static_cast<unsigned*>(fout) + here)
                   : static_cast<void*>(static_cast<float*>(fout) + here);
    if constexpr (fused_use_orbits<Def, BF>())
      fused_collide_all<Def, BF, FusedForms<Def, BF, EXL>::relax2>(Orb{}, d, c, cq, a0, ax, ay, out, p.plane);
    else fused_collide_pop_all<Def, BF>(Seq{}, d, c, cq, a0, ax, ay, out, p.plane);
  }
}

// Resident blocks of 128 threads per SM (so registers per thread), measured
// per stencil size on GB300: Q <= 40: 6 in FP32 (80 registers), 5 in BF16;
// Q <= 64: 5 in FP32 (96 registers), 4 in BF16; larger stencils 4 (128
// registers), where fewer registers would spill.
template <class Def, bool BF, int EXL = 0>
constexpr int fused_min_blocks() {
  return Def::Q <= 40 ? ((BF || EXL) ? 5 : 6) : ((Def::Q <= 64 && !BF && EXL < 2) ? 5 : 4);
}

template <class Def, bool BF, int EXL = 0>
__global__ void __launch_bounds__(128, fused_min_blocks<Def, BF, EXL>()) fused_f32_kernel(const __grid_constant__ FusedParams p,
                                                        const void* __restrict__ fin,
                                                        void* __restrict__ fout) {
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (site < p.Nx * p.Ny) fused_site<Def, BF, EXL>(p, fin, fout, site, fl);
  report(fl, p.err);
}

// Entry point of the step kernel of a stencil, for CUDA graph kernel nodes
// (rlbm_batch_step); the node's grid is (Nx Ny + 127)/128 blocks of 128.
// mode: 0 FP32, 1 BF16 deviation, 2 / 3 FP32 with extended moment sums of
// level 1 / 2.
template <class Def>
const void* fused_kernel_fn_impl(int mode) {
  return mode == 1 ? (const void*)&fused_f32_kernel<Def, true>
         : mode == 2 ? (const void*)&fused_f32_kernel<Def, false, 1>
         : mode == 3 ? (const void*)&fused_f32_kernel<Def, false, 2>
                     : (const void*)&fused_f32_kernel<Def, false>;
}

template <class Def>
cudaError_t launch_fused_impl(const FusedParams& p, const void* fin, void* fout, int mode, cudaStream_t s) {
  const long long nsite = (long long)p.Nx * p.Ny;
  const unsigned grid = (unsigned)((nsite + 127) / 128);
  if (mode == 1) fused_f32_kernel<Def, true><<<grid, 128, 0, s>>>(p, fin, fout);
  else if (mode == 2) fused_f32_kernel<Def, false, 1><<<grid, 128, 0, s>>>(p, fin, fout);
  else if (mode == 3) fused_f32_kernel<Def, false, 2><<<grid, 128, 0, s>>>(p, fin, fout);
  else fused_f32_kernel<Def, false><<<grid, 128, 0, s>>>(p, fin, fout);
  return cudaGetLastError();
}

}  // namespace rlbm

namespace rlbm {

// ---------------------------------------------------- BF16 init and read-out
// Group coefficients of f^eq - r at one site from its fields, in FP64 (same
// definitions as the step kernel: r0..r9 and the folded constants p.gf).
__device__ __forceinline__ void fp64_group_coeffs(const FusedParams& p, const SiteConsts& sc, double n,
                                                  double ux, double uy, double T, double (&c)[6][6],
                                                  unsigned& fl) {
  const double v2 = ux * ux + uy * uy;
  const double g = 1.0 / sqrt(1.0 - v2);
  const double dU = g * g * v2 / (g + 1.0);
  const double Ux = g * ux, Uy = g * uy;
  const double R = ratio64(sc.mbar / T, p.rt64, fl);
  const double dR = R - sc.Rr;
  const double mr32 = sc.mbar * R + 4.0 * T;
  const double F = sc.mY * dR + 3.0 * (T - 1.0);
  const double G = sc.mbar * dR + 4.0 * (T - 1.0);
  const double r0 = n * R - p.nr64 * sc.Rr;
  const double r1 = n * (dU - sc.k21 * dR);
  const double r2 = n * Ux, r3 = n * Uy;
  const double r4 = n * (F + dU * (2.0 * mr32 + sc.cb00_1) + dU * dU * mr32);
  const double h = G + mr32 * dU;
  const double r5 = n * h * Ux, r6 = n * h * Uy;
  const double r7 = n * mr32 * Uy * Uy, r8 = n * mr32 * (Uy * Uy - 2.0 * Ux * Ux), r9 = n * mr32 * Ux * Uy;
  for (int k = 0; k < 6; ++k) {
    double a[10];
    for (int q = 0; q < 10; ++q) a[q] = (double)p.gf[k][q].hi + (double)p.gf[k][q].lo;
    c[k][0] = a[0] * r0 + a[1] * r1 + a[2] * r4 + a[3] * r7 + a[4] * r8;
    c[k][1] = a[5] * r2 + a[6] * r5;
    c[k][2] = a[5] * r3 + a[6] * r6;
    c[k][3] = a[7] * (r7 - r8);
    c[k][4] = a[8] * r7;
    c[k][5] = a[9] * r9;
  }
}

__device__ __forceinline__ uint2 bf_coeffs(const double (&c)[6][6], int g) {
  uint2 q;
  q.x = bf_pack((float)c[g][0], (float)c[g][1]);
  q.y = bf_pack((float)c[g][2], (float)(0.5 * (c[g][3] + c[g][4])));
  return q;
}

__device__ __forceinline__ double bf_ref_rt(uint2 c, int nx, int ny, int mult) {
  return mult * ((double)bf_lo(c.x) + nx * (double)bf_hi(c.x) + ny * (double)bf_lo(c.y) +
                 (nx * nx + ny * ny) * (double)bf_hi(c.y));
}

// Init, phase 1: reference coefficients of every site into both buffers.
template <class Def>
__global__ void __launch_bounds__(128) bf16_init_coeffs(const __grid_constant__ FusedParams p, SiteConsts sc,
                                                        FieldPtrs fd, uint2* __restrict__ c0,
                                                        uint2* __restrict__ c1) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (s < p.Nx * p.Ny) {
    int x, y;
    site_of(s, p.Nx, x, y);
    double c[6][6];
    fp64_group_coeffs(p, sc, fd.n[s], fd.ux[s], fd.uy[s], fd.T[s], c, fl);
    const long long here = (long long)y * p.pitch + x;
    for (int g = 0; g < 6; ++g) {
      const uint2 q = bf_coeffs(c, g);
      c0[(long long)g * p.plane + here] = q;
      c1[(long long)g * p.plane + here] = q;
    }
  }
  report(fl, p.err);
}

// Init, phase 2: S_0 at the site and S_{-1} at x - n_i (see init_kernel).
template <class Def>
__global__ void __launch_bounds__(128) bf16_init_pops(const __grid_constant__ FusedParams p, SiteConsts sc,
                                                      FieldPtrs fd, const uint2* __restrict__ coef,
                                                      unsigned short* __restrict__ cur,
                                                      unsigned short* __restrict__ prev) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (s < p.Nx * p.Ny) {
    int x, y;
    site_of(s, p.Nx, x, y);
    double c[6][6];
    fp64_group_coeffs(p, sc, fd.n[s], fd.ux[s], fd.uy[s], fd.T[s], c, fl);
    const long long here = (long long)y * p.pitch + x;
    constexpr Folded F = Def::F;   // local copies: indexed at run time below
    constexpr BfWords B = Def::B;
    for (int i = 0; i < Def::Q; ++i) {
      const int g = F.grp[i], nx = F.nx[i], ny = F.ny[i], mult = F.mult[i];
      const double fr = mult * (c[g][0] + nx * c[g][1] + ny * c[g][2] + nx * nx * c[g][3] + ny * ny * c[g][4] +
                                nx * ny * c[g][5]);
      const uint2 own = coef[(long long)g * p.plane + here];
      cur[2 * ((long long)B.word[i] * p.plane + here) + B.half[i]] =
          __bfloat16_as_ushort(__double2bfloat16(fr - bf_ref_rt(own, nx, ny, mult)));
      int xs = x - nx, ys = y - ny;
      xs = ((xs % p.Nx) + p.Nx) % p.Nx;
      ys = ((ys % p.Ny) + p.Ny) % p.Ny;
      const long long there = (long long)ys * p.pitch + xs;
      const uint2 rem = coef[(long long)g * p.plane + there];
      prev[2 * ((long long)B.word[i] * p.plane + there) + B.half[i]] =
          __bfloat16_as_ushort(__double2bfloat16(fr - bf_ref_rt(rem, nx, ny, mult)));
    }
  }
  report(fl, p.err);
}

// Read-out: decode the pull of S_{t-1} with its coefficients, FP64 solve.
template <class Def>
__global__ void __launch_bounds__(128) bf16_moments(const __grid_constant__ StepParams<double> p,
                                                    const unsigned short* __restrict__ prev,
                                                    const uint2* __restrict__ cprev, MomentOut mo) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  const long long N = (long long)p.Nx * p.Ny;
  if (s < N) {
    int x, y;
    site_of(s, p.Nx, x, y);
    double m[9];
    for (int k = 0; k < 9; ++k) m[k] = 0.0;
    constexpr Folded F = Def::F;   // local copies: indexed at run time below
    constexpr BfWords B = Def::B;
    for (int i = 0; i < Def::Q; ++i) {
      const int g = F.grp[i], nx = F.nx[i], ny = F.ny[i], mult = F.mult[i];
      const int xs = wrap_sub(x, p.pt.dxm[i], p.Nx);
      const int ys = wrap_sub(y, p.pt.dym[i], p.Ny);
      const long long there = (long long)ys * p.pitch + xs;
      const unsigned short h = prev[2 * ((long long)B.word[i] * p.plane + there) + B.half[i]];
      const double f = (double)__uint_as_float((unsigned)h << 16) +
                       bf_ref_rt(cprev[(long long)g * p.plane + there], nx, ny, mult);
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

// ---------------------------------------------------- FP32 init and read-out
// Init of FP32 storage on a compiled stencil: per site the step kernel's own
// equilibrium of the given fields (split site state with the FP64 dR(Td)
// table, FP32 projections and group coefficients, FP32 group polynomials),
// written to S_0 at the site and to S_{-1} at x - n_i (see init_kernel).
template <class Def, bool PREV, int... Is>
__device__ __forceinline__ void f32_init_pops(std::integer_sequence<int, Is...>, const float (&c)[6][6],
                                              float* __restrict__ cur, float* __restrict__ prev,
                                              long long plane, long long pitch, int x, int y, int Nx, int Ny) {
  // 32-bit element indices (a plane holds fewer than 2^32 elements)
  const unsigned here = (unsigned)y * (unsigned)pitch + (unsigned)x;
  const size_t pl = (unsigned)plane;
  (
      [&] {
        constexpr int i = Is;
        constexpr int g = Def::F.grp[i], nx = Def::F.nx[i], ny = Def::F.ny[i], mult = Def::F.mult[i];
        float e = c[g][0];
        if constexpr (nx != 0) e = fmaf((float)nx, c[g][1], e);
        if constexpr (ny != 0) e = fmaf((float)ny, c[g][2], e);
        if constexpr (nx != 0) e = fmaf((float)(nx * nx), c[g][3], e);
        if constexpr (ny != 0) e = fmaf((float)(ny * ny), c[g][4], e);
        if constexpr (nx != 0 && ny != 0) e = fmaf((float)(nx * ny), c[g][5], e);
        if constexpr (mult != 1) e *= (float)mult;
        cur[here + pl * i] = e;
        if constexpr (PREV) {
          // population i of S_{-1} sits at x - n_i: the first pull brings it back
          const unsigned xs = (unsigned)wrap_c<nx>(x, Nx), ys = (unsigned)wrap_c<ny>(y, Ny);
          prev[ys * (unsigned)pitch + xs + pl * i] = e;
        }
      }(),
      ...);
}

// PREV: also write S_{-1} (the copy whose pull is the initial state) into
// prev; without it the read-out of the freshly initialised state reads cur
// in place (f32_moments_kernel<Def, false>) and the first step overwrites
// prev anyway.
template <class Def, bool PREV>
__global__ void __launch_bounds__(128) f32_init_kernel(const __grid_constant__ FusedParams p, SiteConsts sc,
                                                       FieldPtrs fd, float* __restrict__ cur,
                                                       float* __restrict__ prev) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  if (s < p.Nx * p.Ny) {
    int x, y;
    site_of(s, p.Nx, x, y);
    const double n = fd.n[s], ux = fd.ux[s], uy = fd.uy[s], T = fd.T[s];
    if (!(ux * ux + uy * uy < 1.0)) fl |= ERR_LANDAU;
    if (!(n > 0.0)) fl |= ERR_DENSITY;
    if (!(T > 0.0)) fl |= ERR_EOS;
    // the split site state of the fields, as the step kernel holds it
    SplitSite ss;
    const float vx = (float)ux, vy = (float)uy;
    const float v2 = vx * vx + vy * vy;
    const float sq = sqrtf(fmaxf(1.0f - v2, 0.0f));
    ss.dg = __fdividef(v2, sq * (1.0f + sq));
    ss.U0 = 1.0f + ss.dg;
    ss.Ux = ss.U0 * vx;
    ss.Uy = ss.U0 * vy;
    ss.nd = (float)(n - p.nr64);
    ss.n = (float)n;
    ss.Td = (float)(T - 1.0);
    ss.T = (float)T;
    double dR64;
    if (!dr_table64(ss.Td, p.dr64, dR64)) dR64 = dr_from_zeta(ss.Td, p.mb64, p.Rr64, p.rt64, fl);
    ss.dR = (float)dR64;
    ss.R = p.Rr.hi + (p.Rr.lo + ss.dR);
    float c[6][6];
    fused_coeffs(p, ss, c);
    (void)sc;
    f32_init_pops<Def, PREV>(std::make_integer_sequence<int, Def::Q>{}, c, cur, prev, p.plane, p.pitch, x, y, p.Nx,
                       p.Ny);
  }
  report(fl, p.err);
}

// Read-out of FP32 storage on a compiled stencil: the pull of S_{t-1}, the
// step kernel's extended moment sums (level 2: N^a and K^a to about 2^-40,
// the spatial stress in FP32) and its split site solve (deviations from the
// reference in FP32, the EOS finished by an FP64 Newton step), so n and T
// carry FP32 rounding of their deviations from the reference only.  The
// moment planes are assembled in FP64 from the float-float sums.
// PULL: the state at t is the pull of S_{t-1} in prev; otherwise (right
// after f32_init_kernel<Def, false>) it is S_0 in prev read in place.
template <class Def, bool PULL>
__global__ void __launch_bounds__(128) f32_moments_kernel(const __grid_constant__ FusedParams fp,
                                                          const __grid_constant__ StepParams<double> p,
                                                          const float* __restrict__ prev, MomentOut mo) {
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0;
  const long long N = (long long)p.Nx * p.Ny;
  if (site < N) {
    int x, y;
    site_of(site, p.Nx, x, y);
    float d[Def::Q];
    if constexpr (PULL) {
      fused_load_all<Def, false>(std::make_integer_sequence<int, Def::Q>{}, d, prev, nullptr, p.plane, p.pitch, x,
                                 y, p.Nx, p.Ny);
    } else {
      const unsigned here = (unsigned)y * (unsigned)p.pitch + (unsigned)x;
      const size_t pl = (unsigned)p.plane;
#pragma unroll
      for (int i = 0; i < Def::Q; ++i) d[i] = __ldg(prev + here + pl * i);
    }
    ExMoments em;
    em.N0 = em.Nx = em.Ny = em.K0 = em.Kx = em.Ky = FF{0.0f, 0.0f};
    em.Txx = em.Txy = em.Tyy = 0.0f;
    ex_acc_all<Def, 2>(std::make_integer_sequence<int, Def::O.K>{}, d, fp, em);
    float M[9];
    M[0] = em.N0.hi + em.N0.lo;
    M[1] = em.Nx.hi + em.Nx.lo;
    M[2] = em.Ny.hi + em.Ny.lo;
    M[3] = fmaf(fp.mb, M[0], em.K0.hi + em.K0.lo);
    M[4] = fmaf(fp.mb, M[1], em.Kx.hi + em.Kx.lo);
    M[5] = fmaf(fp.mb, M[2], em.Ky.hi + em.Ky.lo);
    M[6] = em.Txx;
    M[7] = em.Txy;
    M[8] = em.Tyy;
    const SplitSite ss = split_solve<true>(fp, M, fl, &em);
    // FP64 moments: reference + float-float deviations
    const double N0 = (double)em.N0.hi + (double)em.N0.lo, Nx = (double)em.Nx.hi + (double)em.Nx.lo;
    const double Ny = (double)em.Ny.hi + (double)em.Ny.lo, K0 = (double)em.K0.hi + (double)em.K0.lo;
    const double Kx = (double)em.Kx.hi + (double)em.Kx.lo, Ky = (double)em.Ky.hi + (double)em.Ky.lo;
    double m[9];
    m[0] = p.mref[0] + N0;
    m[1] = p.mref[1] + Nx;
    m[2] = p.mref[2] + Ny;
    m[3] = p.mref[3] + fma(fp.mb64, N0, K0);
    m[4] = p.mref[4] + fma(fp.mb64, Nx, Kx);
    m[5] = p.mref[5] + fma(fp.mb64, Ny, Ky);
    m[6] = p.mref[6] + (double)em.Txx;
    m[7] = p.mref[7] + (double)em.Txy;
    m[8] = p.mref[8] + (double)em.Tyy;
    const double vx = (double)ss.Ux / (double)ss.U0, vy = (double)ss.Uy / (double)ss.U0;
    double* out = mo.out;
    int plane = 0;
    if (mo.mask & RLBM_M_N) out[(plane++) * N + site] = fp.nr64 + (double)ss.nd;
    if (mo.mask & RLBM_M_UX) out[(plane++) * N + site] = vx;
    if (mo.mask & RLBM_M_UY) out[(plane++) * N + site] = vy;
    if (mo.mask & RLBM_M_T) out[(plane++) * N + site] = 1.0 + (double)ss.Td;
    if (mo.mask & RLBM_M_E) out[(plane++) * N + site] = m[3] - m[4] * vx - m[5] * vy;
    if (mo.mask & RLBM_M_NVEC)
      for (int k = 0; k < 3; ++k) out[(plane++) * N + site] = m[k];
    if (mo.mask & RLBM_M_TMN)
      for (int k = 3; k < 9; ++k) out[(plane++) * N + site] = m[k];
  }
  report(fl, p.err);
}

// what: 0 BF16 init, 1 BF16 read-out, 2 FP32 init, 3 FP32 read-out.
template <class Def>
cudaError_t launch_bf16_io_impl(int what, const FusedParams& fp, const StepParams<double>& p, FieldPtrs fd,
                                void* cur, void* prev, void* ccur, void* cprev, MomentOut mo, cudaStream_t s) {
  const long long nsite = (long long)p.Nx * p.Ny;
  const unsigned grid = (unsigned)((nsite + 127) / 128);
  if (what == 2) {
    f32_init_kernel<Def, false><<<grid, 128, 0, s>>>(fp, p.sc, fd, static_cast<float*>(cur), static_cast<float*>(prev));
    return cudaGetLastError();
  }
  if (what == 3) {
    f32_moments_kernel<Def, true><<<grid, 128, 0, s>>>(fp, p, static_cast<const float*>(prev), mo);
    return cudaGetLastError();
  }
  if (what == 4) {
    f32_moments_kernel<Def, false><<<grid, 128, 0, s>>>(fp, p, static_cast<const float*>(prev), mo);
    return cudaGetLastError();
  }
  if (what == 0) {
    bf16_init_coeffs<Def><<<grid, 128, 0, s>>>(fp, p.sc, fd, static_cast<uint2*>(ccur), static_cast<uint2*>(cprev));
    bf16_init_pops<Def><<<grid, 128, 0, s>>>(fp, p.sc, fd, static_cast<const uint2*>(ccur),
                                             static_cast<unsigned short*>(cur), static_cast<unsigned short*>(prev));
  } else {
    bf16_moments<Def><<<grid, 128, 0, s>>>(p, static_cast<const unsigned short*>(prev),
                                           static_cast<const uint2*>(cprev), mo);
  }
  return cudaGetLastError();
}

}  // namespace rlbm
