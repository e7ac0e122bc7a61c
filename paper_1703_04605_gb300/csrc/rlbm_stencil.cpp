// Stencil construction on the host: Table I groups, Bessel functions and
// rest-frame moments in binary128, the weights of Eq. 52, the positive-weight
// window search (Sec. III D), the App. A constants and the fold onto 2D.
#include "rlbm_stencil.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <set>
#include <type_traits>

#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 qf;
static inline qf q_exp(qf x) { return expq(x); }
static inline qf q_sqrt(qf x) { return sqrtq(x); }
static inline qf q_abs(qf x) { return fabsq(x); }
static inline qf q_cos(qf x) { return cosq(x); }
static const qf q_pi = 4 * atanq((qf)1);
#else
// On AArch64 Linux long double is IEEE binary128.
static_assert(LDBL_MANT_DIG == 113, "long double must be binary128 on this platform");
typedef long double qf;
static inline qf q_exp(qf x) { return expl(x); }
static inline qf q_sqrt(qf x) { return sqrtl(x); }
static inline qf q_abs(qf x) { return fabsl(x); }
static inline qf q_cos(qf x) { return cosl(x); }
static const qf q_pi = 3.141592653589793238462643383279502884L;
#endif

namespace rlbm {

// ------------------------------------------------------------------ Table I
// Generating vector (a >= b >= c >= 0) of each of the 84 full-symmetric
// groups of Table I (App. C), in table order.
static const int kTableI[84][3] = {
    {0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {1, 1, 1}, {2, 0, 0}, {2, 1, 0}, {2, 2, 0}, {2, 1, 1},
    {2, 2, 1}, {2, 2, 2}, {3, 0, 0}, {3, 1, 0}, {3, 2, 0}, {3, 3, 0}, {3, 1, 1}, {3, 2, 1},
    {3, 2, 2}, {3, 3, 1}, {3, 3, 2}, {3, 3, 3}, {4, 0, 0}, {4, 1, 0}, {4, 2, 0}, {4, 3, 0},
    {4, 4, 0}, {4, 1, 1}, {4, 2, 1}, {4, 3, 1}, {4, 4, 1}, {4, 2, 2}, {4, 3, 2}, {4, 4, 2},
    {4, 3, 3}, {4, 4, 3}, {4, 4, 4}, {5, 0, 0}, {5, 1, 0}, {5, 2, 0}, {5, 3, 0}, {5, 4, 0},
    {5, 5, 0}, {5, 1, 1}, {5, 2, 1}, {5, 3, 1}, {5, 4, 1}, {5, 5, 1}, {5, 2, 2}, {5, 3, 2},
    {5, 4, 2}, {5, 5, 2}, {5, 3, 3}, {5, 4, 3}, {5, 5, 3}, {5, 4, 4}, {5, 5, 4}, {5, 5, 5},
    {6, 0, 0}, {6, 1, 0}, {6, 2, 0}, {6, 3, 0}, {6, 4, 0}, {6, 5, 0}, {6, 6, 0}, {6, 1, 1},
    {6, 2, 1}, {6, 3, 1}, {6, 4, 1}, {6, 5, 1}, {6, 6, 1}, {6, 2, 2}, {6, 3, 2}, {6, 4, 2},
    {6, 5, 2}, {6, 6, 2}, {6, 3, 3}, {6, 4, 3}, {6, 5, 3}, {6, 6, 3}, {6, 4, 4}, {6, 5, 4},
    {6, 6, 4}, {6, 5, 5}, {6, 6, 5}, {6, 6, 6}};

std::vector<std::array<int, 3>> group_orbit(int gid) {
  std::set<std::array<int, 3>> out;
  const int* b = kTableI[gid - 1];
  int perm[3] = {0, 1, 2};
  do {
    for (int s = 0; s < 8; ++s) {
      std::array<int, 3> v;
      for (int a = 0; a < 3; ++a) v[a] = ((s >> a) & 1 ? -1 : 1) * b[perm[a]];
      out.insert(v);
    }
  } while (std::next_permutation(perm, perm + 3));
  return std::vector<std::array<int, 3>>(out.begin(), out.end());
}

static int group_len2(int gid) {
  const int* b = kTableI[gid - 1];
  return b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
}

// ------------------------------------------------------- Bessel functions
// Exponentially scaled K_nu(x) e^x = int_0^inf exp(-x (cosh t - 1)) cosh(nu t) dt,
// trapezoidal rule (geometric convergence for this entire, even integrand;
// Trefethen & Weideman, SIAM Rev. 56, 2014).  The step keeps both the
// small-x strip error exp(-pi^2/(2h)) and the large-x error
// exp(-2 pi^2/(h^2 x)) below the working precision.
template <typename F>
static F trap_step(double x, double digits) {
  const double D = digits * 2.302585092994046 + 10.0;
  const double h1 = M_PI * M_PI / (2.0 * D);
  const double h2 = std::sqrt(2.0 * M_PI * M_PI / (D * x));
  return (F)std::min(h1, h2);
}

// Scaled K1, K2, K3 at x in binary128.
static void bessel_k123_scaled(qf x, qf* k1, qf* k2, qf* k3, double digits = 36.0) {
  const qf h = trap_step<qf>((double)x, digits);
  qf s1 = 0, s2 = 0, s3 = 0;
  const qf tiny = (qf)1e-38;
  for (long j = 0;; ++j) {
    const qf t = h * (qf)j;
    const qf E = q_exp(t), iE = 1 / E;
    const qf cm1 = (E + iE) / 2 - 1;            // cosh t - 1 (exact enough in binary128)
    const qf g = q_exp(-x * cm1);
    const qf c1 = (E + iE) / 2, c2 = (E * E + iE * iE) / 2, c3 = (E * E * E + iE * iE * iE) / 2;
    const qf wgt = (j == 0) ? (qf)0.5 : (qf)1;
    const qf a1 = wgt * g * c1, a2 = wgt * g * c2, a3 = wgt * g * c3;
    s1 += a1;
    s2 += a2;
    s3 += a3;
    if (j > 4 && a3 < tiny * s3 && x * cm1 > (qf)5) break;
    if (j > 2000000) break;
  }
  *k1 = s1 * h;
  *k2 = s2 * h;
  *k3 = s3 * h;
}

// R(x) = K1(x)/K2(x) in binary128 (shares the exponential scaling).
static qf bessel_ratio_q(qf x, double digits = 36.0) {
  qf k1, k2, k3;
  bessel_k123_scaled(x, &k1, &k2, &k3, digits);
  return k1 / k2;
}

// Rest-frame moments <phi> = int omega phi d^3p/p0 (Eq. 36, 40-41, T_R = 1)
// of the eleven monomials that fix a quadrature (Sec. III D): the first six
// (1, p0, px^2, p0 px^2, px^4, px^2 py^2) for second order, all eleven (plus
// p0 px^4, p0 px^2 py^2, px^6, px^4 py^2, px^2 py^2 pz^2) for third order.
// In rapidity chi: d^3p/p0 = m^2 sinh^2 chi dchi dOmega and N_R = 4 pi m K1(m):
//   <p0^a |p|^b * ang> = ang int e^{-m cosh} (m cosh)^a (m sinh)^(b+2) dchi / (m K1(m)),
// with angular means 1, 1, 1/3, 1/3, 1/5, 1/15, 1/5, 1/15, 1/7, 1/35, 1/105.
constexpr int kMom = 11;
static void rest_moments_q_uncached(qf m, qf out[kMom]);

// The moments depend on m only; the last few are kept (window searches and
// stencil builds ask for the same m many times).
static void rest_moments_q(qf m, qf* out, int K) {
  struct Entry {
    qf m;
    qf v[kMom];
  };
  static thread_local Entry cache[8];
  static thread_local int used = 0, next = 0;
  for (int i = 0; i < used; ++i)
    if (cache[i].m == m) {
      for (int k = 0; k < K; ++k) out[k] = cache[i].v[k];
      return;
    }
  Entry& e = cache[next];
  rest_moments_q_uncached(m, e.v);
  e.m = m;
  for (int k = 0; k < K; ++k) out[k] = e.v[k];
  next = (next + 1) % 8;
  if (used < 8) ++used;
}

static void rest_moments_q_uncached(qf m, qf out[kMom]) {
  const qf h = trap_step<qf>((double)m, 36.0);
  // radial integrals of (m cosh)^a (m sinh)^b: (a,b) = (0,0) (1,0) (0,2) (1,2) (0,4) (1,4) (0,6)
  qf s[7] = {0, 0, 0, 0, 0, 0, 0};
  const qf tiny = (qf)1e-38;
  for (long j = 0;; ++j) {
    const qf t = h * (qf)j;
    const qf E = q_exp(t), iE = 1 / E;
    const qf ch = (E + iE) / 2, sh = (E - iE) / 2;
    const qf g = q_exp(-m * (ch - 1)) * ((j == 0) ? (qf)0.5 : (qf)1);
    const qf p0 = m * ch, p = m * sh, p2 = p * p;
    const qf base = g * p2;            // measure m^2 sinh^2
    s[0] += base;
    s[1] += base * p0;
    s[2] += base * p2;
    s[3] += base * p0 * p2;
    s[4] += base * p2 * p2;
    s[5] += base * p0 * p2 * p2;
    s[6] += base * p2 * p2 * p2;
    if (j > 4 && base * p2 * p2 * p2 * p0 < tiny * s[6] && m * (ch - 1) > (qf)5) break;
    if (j > 2000000) break;
  }
  qf k1, k2, k3;
  bessel_k123_scaled(m, &k1, &k2, &k3);   // same e^{m} scaling as the integrals
  const qf norm = h / (m * k1);
  const int src[kMom] = {0, 1, 2, 3, 4, 4, 5, 5, 6, 6, 6};
  const qf ang[kMom] = {1, 1, (qf)1 / 3, (qf)1 / 3, (qf)1 / 5, (qf)1 / 15,
                        (qf)1 / 5, (qf)1 / 15, (qf)1 / 7, (qf)1 / 35, (qf)1 / 105};
  for (int k = 0; k < kMom; ++k) out[k] = s[src[k]] * norm * ang[k];
}

// ------------------------------------------------------------ Eq. 52 solve
// Integer sums over the vectors of one group: count and the sums of n_x^2,
// n_x^4, n_x^2 n_y^2, n_x^6, n_x^4 n_y^2, n_x^2 n_y^2 n_z^2 (the orbit is
// symmetric, so these fix all eleven monomials).
struct GroupSums {
  int cnt, sx2, sx4, sx2y2, sx6, sx4y2, sx2y2z2, len2;
};

static GroupSums group_sums(int gid) {
  GroupSums g{0, 0, 0, 0, 0, 0, 0, group_len2(gid)};
  for (const auto& v : group_orbit(gid)) {
    const int x2 = v[0] * v[0], y2 = v[1] * v[1], z2 = v[2] * v[2];
    g.cnt += 1;
    g.sx2 += x2;
    g.sx4 += x2 * x2;
    g.sx2y2 += x2 * y2;
    g.sx6 += x2 * x2 * x2;
    g.sx4y2 += x2 * x2 * y2;
    g.sx2y2z2 += x2 * y2 * z2;
  }
  return g;
}

// Column k of A(v0) (K = 6 or 11 rows): sums over group k of the monomials at
// the momenta p = m gamma_k (1, v0 n) of Eq. 48.
template <typename F, int K>
static bool build_system(const GroupSums* gs, F m, F v0, F A[K][K]) {
  for (int k = 0; k < K; ++k) {
    const F s = 1 - v0 * v0 * (F)gs[k].len2;
    if (!(s > 0)) return false;
    F gam;
    if constexpr (std::is_same<F, double>::value) gam = 1 / std::sqrt(s);
    else gam = 1 / q_sqrt(s);
    const F p0 = m * gam, ps = m * gam * v0, ps2 = ps * ps, ps4 = ps2 * ps2;
    A[0][k] = (F)gs[k].cnt;
    A[1][k] = (F)gs[k].cnt * p0;
    A[2][k] = ps2 * (F)gs[k].sx2;
    A[3][k] = p0 * ps2 * (F)gs[k].sx2;
    A[4][k] = ps4 * (F)gs[k].sx4;
    A[5][k] = ps4 * (F)gs[k].sx2y2;
    if constexpr (K == 11) {
      A[6][k] = p0 * ps4 * (F)gs[k].sx4;
      A[7][k] = p0 * ps4 * (F)gs[k].sx2y2;
      A[8][k] = ps4 * ps2 * (F)gs[k].sx6;
      A[9][k] = ps4 * ps2 * (F)gs[k].sx4y2;
      A[10][k] = ps4 * ps2 * (F)gs[k].sx2y2z2;
    }
  }
  return true;
}

// Gaussian elimination with partial pivoting; false if singular or NaN.
template <typename F, int K>
static bool solve_k(F A[K][K], const F* b, F* x) {
  F M[K][K + 1];
  for (int r = 0; r < K; ++r) {
    for (int c = 0; c < K; ++c) M[r][c] = A[r][c];
    M[r][K] = b[r];
  }
  for (int c = 0; c < K; ++c) {
    int piv = c;
    for (int r = c + 1; r < K; ++r)
      if ((M[r][c] < 0 ? -M[r][c] : M[r][c]) > (M[piv][c] < 0 ? -M[piv][c] : M[piv][c])) piv = r;
    if (M[piv][c] == 0) return false;
    if (piv != c)
      for (int k = 0; k <= K; ++k) std::swap(M[c][k], M[piv][k]);
    for (int r = c + 1; r < K; ++r) {
      const F f = M[r][c] / M[c][c];
      for (int k = c; k <= K; ++k) M[r][k] -= f * M[c][k];
    }
  }
  for (int r = K - 1; r >= 0; --r) {
    F s = M[r][K];
    for (int k = r + 1; k < K; ++k) s -= M[r][k] * x[k];
    x[r] = s / M[r][r];
  }
  for (int r = 0; r < K; ++r)
    if (!(x[r] == x[r])) return false;
  return true;
}

static bool valid_groups(const int* groups, int ngroups) {
  if ((ngroups != 6 && ngroups != 11) || !groups) return false;
  for (int k = 0; k < ngroups; ++k) {
    if (groups[k] < 1 || groups[k] > 84) return false;
    for (int j = 0; j < k; ++j)
      if (groups[j] == groups[k]) return false;
  }
  return true;
}

template <int K>
static bool weights_q(const int* groups, double m, double v0, qf* x) {
  qf A[K][K], b[K];
  GroupSums gs[K];
  for (int k = 0; k < K; ++k) gs[k] = group_sums(groups[k]);
  rest_moments_q((qf)m, b, K);
  if (!build_system<qf, K>(gs, (qf)m, (qf)v0, A)) return false;
  return solve_k<qf, K>(A, b, x);
}

bool quadrature_weights(const int* groups, int ngroups, double m, double v0, double* w) {
  qf x[kMom];
  bool ok = false;
  if (ngroups == 6) ok = weights_q<6>(groups, m, v0, x);
  else if (ngroups == 11) ok = weights_q<11>(groups, m, v0, x);
  if (!ok) return false;
  for (int k = 0; k < ngroups; ++k) w[k] = (double)x[k];
  return true;
}

// Positive-weight windows (Sec. III D).  Each weight w_k(v0) is scanned on a
// uniform grid; every sign change is refined by bisection; the sorted set of
// crossings splits (0, v_max) into intervals of constant sign pattern, and
// those whose midpoint has all weights positive are the windows.
template <int K>
static int window_k(const int* groups, double m, double* lo, double* hi) {
  double vmax = 1e300;
  for (int k = 0; k < K; ++k) {
    const int l2 = group_len2(groups[k]);
    if (l2 > 0) vmax = std::min(vmax, 1.0 / std::sqrt((double)l2));
  }
  if (vmax > 1.0) vmax = 1.0;
  qf bq[K];
  rest_moments_q((qf)m, bq, K);
  double b[K];
  for (int k = 0; k < K; ++k) b[k] = (double)bq[k];
  GroupSums gs[K];
  for (int k = 0; k < K; ++k) gs[k] = group_sums(groups[k]);
  auto weights_d = [&](double v, double* w) -> bool {
    double A[K][K];
    if (!build_system<double, K>(gs, m, v, A)) return false;
    return solve_k<double, K>(A, b, w);
  };
  const int N = 20000;
  const double v_a = vmax * 1e-4, v_b = vmax * (1 - 1e-9);
  std::vector<double> cross;
  double wprev[K];
  bool okprev = weights_d(v_a, wprev);
  double vprev = v_a;
  for (int i = 1; i <= N; ++i) {
    const double v = v_a + (v_b - v_a) * i / N;
    double w[K];
    const bool ok = weights_d(v, w);
    if (ok && okprev) {
      for (int k = 0; k < K; ++k) {
        if ((w[k] > 0) != (wprev[k] > 0)) {
          double a = vprev, c = v;
          const bool sa = wprev[k] > 0;
          for (int it = 0; it < 80; ++it) {
            const double mid = 0.5 * (a + c);
            double wm[K];
            if (!weights_d(mid, wm)) break;
            if ((wm[k] > 0) == sa) a = mid;
            else c = mid;
          }
          cross.push_back(0.5 * (a + c));
        }
      }
    } else if (ok != okprev) {
      cross.push_back(ok ? v : vprev);
    }
    std::memcpy(wprev, w, sizeof w);
    okprev = ok;
    vprev = v;
  }
  cross.push_back(v_a);
  cross.push_back(v_b);
  std::sort(cross.begin(), cross.end());
  int count = 0;
  double best = -1;
  for (size_t i = 0; i + 1 < cross.size(); ++i) {
    const double a = cross[i], c = cross[i + 1];
    if (!(c > a)) continue;
    double w[K];
    if (!quadrature_weights(groups, K, m, 0.5 * (a + c), w)) continue;
    bool pos = true;
    for (int k = 0; k < K; ++k) pos = pos && (w[k] > 0);
    if (!pos) continue;
    ++count;
    if (c - a > best) {
      best = c - a;
      *lo = a;
      *hi = c;
    }
  }
  return count;
}

int quadrature_window(const int* groups, int ngroups, double m, double* lo, double* hi) {
  if (ngroups == 6) return window_k<6>(groups, m, lo, hi);
  if (ngroups == 11) return window_k<11>(groups, m, lo, hi);
  return 0;
}
// ------------------------------------------------------- App. A constants
static SiteConsts site_consts(double mbar, qf* cJ00_1, qf* cJ00_0, qf* Aq, qf* Bq, qf* Cq,
                              qf* Dq, qf* Eq, qf* k21q, qf* k32q) {
  const qf m = (qf)mbar;
  qf k1, k2, k3;
  bessel_k123_scaled(m, &k1, &k2, &k3);   // common factor e^m cancels below
  const qf den = m * k1 * k1 + 3 * k2 * k1 - m * k2 * k2;
  const qf A = q_sqrt(m * (m + k2 * (3 * k1 - m * k2) / (k1 * k1)));
  const qf B = q_sqrt(m * k2 / k1);
  const qf C = q_sqrt(2 * m * m + 5 * m * k2 / k1 - 3 * k1 * (m * k1 + 3 * k2) / den + 3);
  const qf D = q_sqrt(m * m * (m * k2 * k2 + 5 * k3 * k2 - m * k3 * k3) / (k1 * k2));
  const qf E = q_sqrt(m * m * k3 / k1);
  const qf X = -m * k1 / k2 + m * k2 / k1 - 3;
  const qf Y = (-m * m * k1 * k1 + (m * m + 3) * k2 * k2 - 3 * m * k2 * k1) / den;
  const qf s3 = q_sqrt((qf)3);
  *cJ00_1 = 3 / X - 3;
  *cJ00_0 = 3 * k1 * (m * k1 + 3 * k2) / den - m * m - 3;
  *Aq = A, *Bq = B, *Cq = C, *Dq = D, *Eq = E;
  *k21q = k2 / k1;
  *k32q = k3 / k2;
  SiteConsts sc;
  sc.mbar = mbar;
  sc.inv_m = (double)(1 / m);
  sc.k21 = (double)(k2 / k1);
  sc.k32 = (double)(k3 / k2);
  sc.Rr = (double)(k1 / k2);
  sc.A = (double)A, sc.B = (double)B, sc.C = (double)C, sc.D = (double)D, sc.E = (double)E;
  sc.iA = (double)(1 / A), sc.iB = (double)(1 / B), sc.i3C = (double)(1 / (s3 * C));
  sc.iD = (double)(1 / D), sc.i2E = (double)(1 / (2 * E)), sc.i23E = (double)(1 / (2 * s3 * E));
  sc.iE = (double)(1 / E);
  sc.cb00_1 = (double)(3 * (1 / X - 1));
  sc.Y = (double)Y;
  sc.mY = (double)(m + Y);
  sc.mk32 = (double)(m * k3 / k2);
  return sc;
}

struct PopConstsQ {
  qf p0, px, py, pz2, w;
  qf J[NJ];
};

rlbm_status build_stencil(const rlbm_stencil* st, double m, StencilBuild* out, std::string* err) {
  if (!st || !valid_groups(st->groups, st->ngroups) || st->ngroups != 6) {
    *err = "stencil must list 6 distinct group ids in 1..84 (second order, Sec. III D)";
    return RLBM_EINVAL;
  }
  if (!(m > 0) || !std::isfinite(m)) {
    *err = "m must be positive and finite";
    return RLBM_EINVAL;
  }
  // canonical order: ascending group ids (the weights follow the groups)
  int sorted[6];
  for (int k = 0; k < 6; ++k) sorted[k] = st->groups[k];
  std::sort(sorted, sorted + 6);
  for (int k = 0; k < 6; ++k) out->groups[k] = sorted[k];
  out->mbar = m;
  double v0 = st->v0;
  if (!(v0 >= 0) || !std::isfinite(v0)) {
    *err = "v0 must be >= 0";
    return RLBM_EINVAL;
  }
  if (v0 == 0) {
    double lo, hi;
    if (quadrature_window(sorted, 6, m, &lo, &hi) == 0) {
      *err = "no v0 gives positive weights for these groups at this m";
      return RLBM_ENOQUAD;
    }
    v0 = 0.5 * (lo + hi);
  }
  out->v0 = v0;
  for (int k = 0; k < 6; ++k) {
    if (!(v0 * v0 * group_len2(sorted[k]) < 1)) {
      *err = "v0 ||n_k|| must stay below the speed of light (Sec. III C)";
      return RLBM_EINVAL;
    }
  }
  if (!quadrature_weights(sorted, 6, m, v0, out->w_group)) {
    *err = "singular quadrature system at this v0";
    return RLBM_ENOQUAD;
  }
  for (int k = 0; k < 6; ++k) {
    if (!(out->w_group[k] > 0)) {
      *err = "a quadrature weight is not positive at this v0 (Sec. III D requires w > 0)";
      return RLBM_ENOQUAD;
    }
  }
  // weights again in binary128 for the per-population constants
  qf wq[6];
  weights_q<6>(sorted, m, v0, wq);
  qf cJ1, cJ0, Aq, Bq, Cq, Dq, Eq, k21q, k32q;
  out->sc = site_consts(m, &cJ1, &cJ0, &Aq, &Bq, &Cq, &Dq, &Eq, &k21q, &k32q);
  const qf s3 = q_sqrt((qf)3);
  const qf b0r = 1 / (k21q * (qf)m);          // K1/K2(mbar)/mbar
  out->b0ref1 = (double)b0r;
  {
    const qf Rr = 1 / k21q, z = (qf)m;
    out->cv_r = (double)(3 - z * z * (Rr * Rr + 3 * Rr / z - 1));
  }
  qf mref[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  qf kref = 0;
  // fold: merge (nx, ny, +nz) with (nx, ny, -nz) inside each group
  out->pops.clear();
  out->popc.clear();
  out->halo = 0;
  for (int k = 0; k < 6; ++k) {
    const qf len2 = (qf)group_len2(sorted[k]);
    const qf gam = 1 / q_sqrt(1 - (qf)v0 * (qf)v0 * len2);
    const qf p0 = (qf)m * gam, ps = (qf)m * gam * (qf)v0;
    {
      const qf w = wq[k], P0 = p0, Pv = ps, Pv2 = ps * ps;
      const qf mq = (qf)m;
      const qf gm[5] = {P0, P0 * P0, Pv, P0 * Pv, Pv2};
      const qf gf[10] = {w / mq,
                         w * (P0 - mq * k21q) / (Aq * Aq),
                         w * (P0 * P0 + cJ1 * P0 + cJ0) / (3 * Cq * Cq),
                         -w * Pv2 * len2 / (4 * Eq * Eq),
                         w * Pv2 * len2 / (12 * Eq * Eq),
                         w * Pv / (Bq * Bq),
                         w * Pv * (P0 - mq * k32q) / (Dq * Dq),
                         w * Pv2 / (4 * Eq * Eq),
                         w * Pv2 / (2 * Eq * Eq),
                         w * Pv2 / (Eq * Eq)};
      for (int q = 0; q < 5; ++q) out->gm[k][q] = (double)gm[q];
      for (int q = 0; q < 10; ++q) out->gf[k][q] = (double)gf[q];
      out->gk[k][0] = (double)(P0 * (P0 - mq));
      out->gk[k][1] = (double)(Pv * (P0 - mq));
      out->rmax1[k] = 0;
    }
    std::vector<std::array<int, 3>> seen;
    std::vector<int> mult;
    for (const auto& v : group_orbit(sorted[k])) {
      std::array<int, 3> key{v[0], v[1], std::abs(v[2])};
      auto it = std::find(seen.begin(), seen.end(), key);
      if (it == seen.end()) {
        seen.push_back(key);
        mult.push_back(1);
      } else {
        mult[it - seen.begin()] += 1;
      }
    }
    for (size_t a = 0; a < seen.size(); ++a) {
      FoldedPop fp{k, seen[a][0], seen[a][1], seen[a][2] * seen[a][2], mult[a]};
      out->pops.push_back(fp);
      out->halo = std::max(out->halo, std::max(std::abs(fp.nx), std::abs(fp.ny)));
      PopConstsQ pc;
      pc.p0 = p0;
      pc.px = ps * fp.nx;
      pc.py = ps * fp.ny;
      pc.pz2 = ps * ps * fp.nz2;
      pc.w = wq[k] * (qf)fp.mult;
      pc.J[0] = 1;
      pc.J[1] = (p0 - (qf)m * k21q) / Aq;
      pc.J[2] = pc.px / Bq;
      pc.J[3] = pc.py / Bq;
      pc.J[4] = (p0 * p0 + cJ1 * p0 + cJ0) / (s3 * Cq);
      pc.J[5] = pc.px * (p0 - (qf)m * k32q) / Dq;
      pc.J[6] = pc.py * (p0 - (qf)m * k32q) / Dq;
      pc.J[7] = (pc.py * pc.py - pc.pz2) / (2 * Eq);
      pc.J[8] = (-2 * pc.px * pc.px + pc.py * pc.py + pc.pz2) / (2 * s3 * Eq);
      pc.J[9] = pc.px * pc.py / Eq;
      const qf mom[9] = {pc.p0, pc.px, pc.py, pc.p0 * pc.p0, pc.p0 * pc.px, pc.p0 * pc.py,
                         pc.px * pc.px, pc.px * pc.py, pc.py * pc.py};
      std::array<double, 21> row;
      for (int q = 0; q < 9; ++q) {
        row[q] = (double)mom[q];
        mref[q] += pc.w * b0r * mom[q];
      }
      kref += pc.w * b0r * pc.p0 * (pc.p0 - (qf)m);
      out->rmax1[k] = std::max(out->rmax1[k], (double)(pc.w * b0r));
      for (int q = 0; q < NJ; ++q) row[9 + q] = (double)(pc.w * pc.J[q]);
      row[19] = (double)(pc.px / pc.p0);
      row[20] = (double)(pc.py / pc.p0);
      out->popc.push_back(row);
    }
  }
  for (int q = 0; q < 9; ++q) out->mref1[q] = (double)mref[q];
  out->kref1 = (double)kref;
  out->ykr1 = (double)(kref / mref[0]);
  if ((int)out->pops.size() > QMAX) {
    *err = "folded stencil has more populations than the compiled maximum (96)";
    return RLBM_ENOTSUP;
  }
  return RLBM_OK;
}

// ------------------------------------------------------- third order
// Inverse of a K x K binary128 matrix by Gauss-Jordan elimination with
// partial pivoting (K = 20: the Gram matrix of the centred monomials).
static bool invert_q(std::vector<qf>& M, int K) {
  std::vector<qf> I((size_t)K * K, (qf)0);
  for (int i = 0; i < K; ++i) I[(size_t)i * K + i] = 1;
  for (int c = 0; c < K; ++c) {
    int piv = c;
    for (int r = c + 1; r < K; ++r)
      if (q_abs(M[(size_t)r * K + c]) > q_abs(M[(size_t)piv * K + c])) piv = r;
    if (M[(size_t)piv * K + c] == 0) return false;
    if (piv != c)
      for (int k = 0; k < K; ++k) {
        std::swap(M[(size_t)c * K + k], M[(size_t)piv * K + k]);
        std::swap(I[(size_t)c * K + k], I[(size_t)piv * K + k]);
      }
    const qf d = 1 / M[(size_t)c * K + c];
    for (int k = 0; k < K; ++k) {
      M[(size_t)c * K + k] *= d;
      I[(size_t)c * K + k] *= d;
    }
    for (int r = 0; r < K; ++r) {
      if (r == c) continue;
      const qf f = M[(size_t)r * K + c];
      if (f == 0) continue;
      for (int k = 0; k < K; ++k) {
        M[(size_t)r * K + k] -= f * M[(size_t)c * K + k];
        I[(size_t)r * K + k] -= f * I[(size_t)c * K + k];
      }
    }
  }
  M.swap(I);
  return true;
}

// The twenty centred monomials (kO3Mono order) at one folded population.
static void o3_monomials(qf t, qf px, qf py, qf pz2, qf* phi) {
  phi[0] = 1;
  phi[1] = t;
  phi[2] = px;
  phi[3] = py;
  phi[4] = t * px;
  phi[5] = t * py;
  phi[6] = px * px;
  phi[7] = py * py;
  phi[8] = px * py;
  phi[9] = pz2;
  phi[10] = t * px * px;
  phi[11] = t * py * py;
  phi[12] = t * px * py;
  phi[13] = px * px * px;
  phi[14] = px * px * py;
  phi[15] = px * py * py;
  phi[16] = py * py * py;
  phi[17] = t * pz2;
  phi[18] = px * pz2;
  phi[19] = py * pz2;
}

rlbm_status build_stencil_o3(const rlbm_stencil* st, double m, StencilBuildO3* out, std::string* err) {
  if (!st || !valid_groups(st->groups, st->ngroups) || st->ngroups != 11) {
    *err = "a third-order stencil lists 11 distinct group ids in 1..84 (Sec. III D)";
    return RLBM_EINVAL;
  }
  if (!(m > 0) || !std::isfinite(m)) {
    *err = "m must be positive and finite";
    return RLBM_EINVAL;
  }
  int sorted[11];
  for (int k = 0; k < 11; ++k) sorted[k] = st->groups[k];
  std::sort(sorted, sorted + 11);
  for (int k = 0; k < 11; ++k) out->groups[k] = sorted[k];
  out->mbar = m;
  double v0 = st->v0;
  if (!(v0 >= 0) || !std::isfinite(v0)) {
    *err = "v0 must be >= 0";
    return RLBM_EINVAL;
  }
  if (v0 == 0) {
    double lo, hi;
    if (quadrature_window(sorted, 11, m, &lo, &hi) == 0) {
      *err = "no v0 gives positive weights for these groups at this m";
      return RLBM_ENOQUAD;
    }
    v0 = 0.5 * (lo + hi);
  }
  out->v0 = v0;
  for (int k = 0; k < 11; ++k)
    if (!(v0 * v0 * group_len2(sorted[k]) < 1)) {
      *err = "v0 ||n_k|| must stay below the speed of light (Sec. III C)";
      return RLBM_EINVAL;
    }
  qf wq[11];
  if (!weights_q<11>(sorted, m, v0, wq)) {
    *err = "singular quadrature system at this v0";
    return RLBM_ENOQUAD;
  }
  for (int k = 0; k < 11; ++k) {
    out->w_group[k] = (double)wq[k];
    if (!(wq[k] > 0)) {
      *err = "a quadrature weight is not positive at this v0 (Sec. III D requires w > 0)";
      return RLBM_ENOQUAD;
    }
  }
  qf cJ1, cJ0, Aq, Bq, Cq, Dq, Eq, k21q, k32q;
  out->sc = site_consts(m, &cJ1, &cJ0, &Aq, &Bq, &Cq, &Dq, &Eq, &k21q, &k32q);
  const qf mq = (qf)m;
  const qf c = mq * k21q;                  // <p0>_omega = mbar K2/K1(mbar)
  const qf wr1 = 1 / (k21q * mq);          // K1/K2(mbar)/mbar
  out->c = (double)c;
  {
    const qf Rr = 1 / k21q;
    out->cv_r = (double)(3 - mq * mq * (Rr * Rr + 3 * Rr / mq - 1));
  }
  // fold (as build_stencil): per group, the orbit with +-n_z merged
  struct PopQ {
    qf p0, px, py, pz2, w;
  };
  std::vector<PopQ> pq;
  out->pops.clear();
  out->halo = 0;
  for (int k = 0; k < 11; ++k) {
    const qf len2 = (qf)group_len2(sorted[k]);
    const qf gam = 1 / q_sqrt(1 - (qf)v0 * (qf)v0 * len2);
    const qf p0 = mq * gam, ps = mq * gam * (qf)v0;
    const qf gm[5] = {p0, p0 * p0, ps, p0 * ps, ps * ps};
    for (int q = 0; q < 5; ++q) out->gm[k][q] = (double)gm[q];
    std::vector<std::array<int, 3>> seen;
    std::vector<int> mult;
    for (const auto& v : group_orbit(sorted[k])) {
      std::array<int, 3> key{v[0], v[1], std::abs(v[2])};
      auto it = std::find(seen.begin(), seen.end(), key);
      if (it == seen.end()) {
        seen.push_back(key);
        mult.push_back(1);
      } else {
        mult[it - seen.begin()] += 1;
      }
    }
    for (size_t a = 0; a < seen.size(); ++a) {
      FoldedPop fp{k, seen[a][0], seen[a][1], seen[a][2] * seen[a][2], mult[a]};
      out->pops.push_back(fp);
      out->halo = std::max(out->halo, std::max(std::abs(fp.nx), std::abs(fp.ny)));
      pq.push_back(PopQ{p0, ps * fp.nx, ps * fp.ny, ps * ps * fp.nz2, wq[k] * (qf)fp.mult});
    }
  }
  const int Q = (int)pq.size();
  if (Q > kMaxPopO3) {
    *err = "folded stencil has more populations than the compiled maximum (256)";
    return RLBM_ENOTSUP;
  }
  // Gram matrix of the centred monomials under the stencil's weights; the
  // quadrature is exact for their products, so this is the continuum one
  const int K = kO3Mono;
  std::vector<qf> phi((size_t)Q * K), G((size_t)K * K, (qf)0);
  for (int i = 0; i < Q; ++i) {
    o3_monomials(pq[i].p0 - c, pq[i].px, pq[i].py, pq[i].pz2, &phi[(size_t)i * K]);
    for (int a = 0; a < K; ++a)
      for (int b = 0; b < K; ++b) G[(size_t)a * K + b] += pq[i].w * phi[(size_t)i * K + a] * phi[(size_t)i * K + b];
  }
  if (!invert_q(G, K)) {
    *err = "singular third-order Gram matrix (the stencil is not third order)";
    return RLBM_ENOQUAD;
  }
  qf mref[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  out->rows.assign(Q, {});
  for (int i = 0; i < Q; ++i) {
    const PopQ& P = pq[i];
    const qf mom[9] = {P.p0, P.px, P.py, P.p0 * P.p0, P.p0 * P.px, P.p0 * P.py,
                       P.px * P.px, P.px * P.py, P.py * P.py};
    auto& row = out->rows[i];
    for (int q = 0; q < 9; ++q) {
      row[q] = (double)mom[q];
      mref[q] += P.w * wr1 * mom[q];
    }
    row[9] = (double)(P.w * wr1);
    for (int l = 0; l < K; ++l) {
      qf acc = 0;
      for (int b = 0; b < K; ++b) acc += G[(size_t)l * K + b] * phi[(size_t)i * K + b];
      row[10 + l] = (double)(P.w * acc);
    }
    row[30] = (double)(P.px / P.p0);
    row[31] = (double)(P.py / P.p0);
  }
  for (int q = 0; q < 9; ++q) out->mref1[q] = (double)mref[q];
  return RLBM_OK;
}

rlbm_status build_stencil3d_o3(const rlbm_stencil* st, double m, StencilBuild3O3* out, std::string* err) {
  // weights, v0 and site constants as for the folded third-order build
  StencilBuildO3 f;
  rlbm_status s = build_stencil_o3(st, m, &f, err);
  if (s != RLBM_OK) return s;
  for (int k = 0; k < 11; ++k) {
    out->groups[k] = f.groups[k];
    out->w_group[k] = f.w_group[k];
  }
  out->c = f.c;
  StencilBuild& sb = out->base.sb;
  sb.mbar = m;
  sb.v0 = f.v0;
  sb.sc = f.sc;
  sb.cv_r = f.cv_r;
  sb.halo = 0;
  const double v0 = f.v0;
  qf wq[11];
  weights_q<11>(f.groups, m, v0, wq);
  const qf mq = (qf)m;
  qf k1, k2, k3;
  bessel_k123_scaled(mq, &k1, &k2, &k3);
  const qf c = mq * k2 / k1;
  const qf wr1 = k1 / (k2 * mq);           // K1/K2(mbar)/mbar
  struct PopQ {
    qf p0, px, py, pz, w;
  };
  std::vector<PopQ> pq;
  out->base.pops.clear();
  out->base.halo = 0;
  for (int k = 0; k < 11; ++k) {
    const qf len2 = (qf)group_len2(f.groups[k]);
    const qf gam = 1 / q_sqrt(1 - (qf)v0 * (qf)v0 * len2);
    const qf p0 = mq * gam, ps = mq * gam * (qf)v0;
    for (const auto& v : group_orbit(f.groups[k])) {   // lexicographic (n_x, n_y, n_z)
      Pop3 q{};
      q.group = k;
      q.nx = v[0];
      q.ny = v[1];
      q.nz = v[2];
      out->base.pops.push_back(q);
      for (int a = 0; a < 3; ++a) out->base.halo = std::max(out->base.halo, std::abs(v[a]));
      pq.push_back(PopQ{p0, ps * v[0], ps * v[1], ps * v[2], wq[k]});
    }
  }
  const int Q = (int)pq.size();
  if (Q > kMaxPop3) {
    *err = "unfolded stencil has more populations than the compiled maximum (160)";
    return RLBM_ENOTSUP;
  }
  const int K = kO3Mono3;
  auto pw = [](qf x, int e) {
    qf r = 1;
    for (int j = 0; j < e; ++j) r *= x;
    return r;
  };
  std::vector<qf> phi((size_t)Q * K), G((size_t)K * K, (qf)0);
  for (int i = 0; i < Q; ++i) {
    const qf t = pq[i].p0 - c;
    for (int l = 0; l < K; ++l) {
      const int* e = kO3Exp3.e[l];
      phi[(size_t)i * K + l] = pw(t, e[0]) * pw(pq[i].px, e[1]) * pw(pq[i].py, e[2]) * pw(pq[i].pz, e[3]);
    }
    for (int a = 0; a < K; ++a)
      for (int b = 0; b < K; ++b) G[(size_t)a * K + b] += pq[i].w * phi[(size_t)i * K + a] * phi[(size_t)i * K + b];
  }
  if (!invert_q(G, K)) {
    *err = "singular third-order Gram matrix (the stencil is not third order)";
    return RLBM_ENOQUAD;
  }
  qf mref[14] = {};
  out->wrows.assign(Q, {});
  for (int i = 0; i < Q; ++i) {
    const PopQ& P = pq[i];
    const qf mom[14] = {P.p0, P.px, P.py, P.pz, P.p0 * P.p0, P.p0 * P.px, P.p0 * P.py, P.p0 * P.pz,
                        P.px * P.px, P.px * P.py, P.px * P.pz, P.py * P.py, P.py * P.pz, P.pz * P.pz};
    Pop3& q = out->base.pops[i];
    for (int k = 0; k < 14; ++k) {
      q.c[k] = (double)mom[k];
      mref[k] += P.w * wr1 * mom[k];
    }
    q.c[14] = (double)(P.w * wr1);
    q.c[28] = (double)(P.px / P.p0);
    q.c[29] = (double)(P.py / P.p0);
    q.c[30] = (double)(P.pz / P.p0);
    for (int l = 0; l < K; ++l) {
      qf acc = 0;
      for (int b = 0; b < K; ++b) acc += G[(size_t)l * K + b] * phi[(size_t)i * K + b];
      out->wrows[i][l] = (double)(P.w * acc);
    }
  }
  for (int k = 0; k < 14; ++k) out->base.mref1[k] = (double)mref[k];
  return RLBM_OK;
}

rlbm_status build_stencil3d(const rlbm_stencil* st, double m, StencilBuild3* out, std::string* err) {
  rlbm_status s = build_stencil(st, m, &out->sb, err);
  if (s != RLBM_OK) return s;
  const int* g6 = out->sb.groups;        // ascending, as the weights
  const double v0 = out->sb.v0;
  qf wq[6];
  weights_q<6>(g6, m, v0, wq);
  qf cJ1, cJ0, Aq, Bq, Cq, Dq, Eq, k21q, k32q;
  site_consts(m, &cJ1, &cJ0, &Aq, &Bq, &Cq, &Dq, &Eq, &k21q, &k32q);
  const qf s3 = q_sqrt((qf)3);
  const qf mq = (qf)m;
  const qf b0r = 1 / (k21q * mq);          // K1/K2(mbar)/mbar: J^(0) coefficient of r_i
  qf mref[14] = {};
  out->pops.clear();
  out->halo = 0;
  for (int k = 0; k < 6; ++k) {
    const qf len2 = (qf)group_len2(g6[k]);
    const qf gam = 1 / q_sqrt(1 - (qf)v0 * (qf)v0 * len2);
    const qf p0 = mq * gam, ps = mq * gam * (qf)v0;
    {
      const qf w = wq[k], Pv2 = ps * ps;
      const qf K9 = w * Pv2 / (4 * Eq * Eq), K10 = w * Pv2 / (12 * Eq * Eq), K13 = w * Pv2 / (Eq * Eq);
      const qf gf[10] = {w / mq,
                         w * (p0 - mq * k21q) / (Aq * Aq),
                         w * (p0 * p0 + cJ1 * p0 + cJ0) / (3 * Cq * Cq),
                         -len2 * K9,
                         len2 * K10,
                         w * ps / (Bq * Bq),
                         w * ps * (p0 - mq * k32q) / (Dq * Dq),
                         K9,
                         K10,
                         K13};
      for (int q = 0; q < 10; ++q) out->gf3[k][q] = (double)gf[q];
    }
    // lexicographic (n_x, n_y, n_z) inside a group: the order the compiled 3D
    // stencils use (rlbm_stencils.h, unfold_stencil)
    std::vector<std::array<int, 3>> orb = group_orbit(g6[k]);
    std::sort(orb.begin(), orb.end());
    for (const auto& v : orb) {
      Pop3 q;
      q.group = k;
      q.nx = v[0];
      q.ny = v[1];
      q.nz = v[2];
      out->halo = std::max(out->halo, std::max(std::abs(v[0]), std::max(std::abs(v[1]), std::abs(v[2]))));
      const qf px = ps * v[0], py = ps * v[1], pz = ps * v[2];
      const qf mom[14] = {p0,      px,      py,      pz,      p0 * p0, p0 * px, p0 * py,
                          p0 * pz, px * px, px * py, px * pz, py * py, py * pz, pz * pz};
      const qf sh21 = p0 - mq * k21q, sh32 = p0 - mq * k32q;
      const qf J[14] = {1,
                        sh21 / Aq,
                        px / Bq,
                        py / Bq,
                        pz / Bq,
                        (p0 * p0 + cJ1 * p0 + cJ0) / (s3 * Cq),
                        px * sh32 / Dq,
                        py * sh32 / Dq,
                        pz * sh32 / Dq,
                        (py * py - pz * pz) / (2 * Eq),
                        (-2 * px * px + py * py + pz * pz) / (2 * s3 * Eq),
                        px * pz / Eq,
                        py * pz / Eq,
                        px * py / Eq};
      for (int a = 0; a < 14; ++a) {
        q.c[a] = (double)mom[a];
        q.c[14 + a] = (double)(wq[k] * J[a]);
        mref[a] += wq[k] * b0r * mom[a];
      }
      q.c[28] = (double)(px / p0);
      q.c[29] = (double)(py / p0);
      q.c[30] = (double)(pz / p0);
      out->pops.push_back(q);
    }
  }
  for (int a = 0; a < 14; ++a) out->mref1[a] = (double)mref[a];
  if ((int)out->pops.size() > kMaxPop3) {
    *err = "stencil has more populations than the 3D kernels support (160)";
    return RLBM_ENOTSUP;
  }
  return RLBM_OK;
}

template <typename CT>
void fill_pop_table(const StencilBuild& sb, int Nx, int Ny, PopTable<CT>* pt) {
  std::memset(pt, 0, sizeof(*pt));
  for (size_t i = 0; i < sb.pops.size(); ++i) {
    const FoldedPop& fp = sb.pops[i];
    const std::array<double, 21>& r = sb.popc[i];
    pt->dxm[i] = ((fp.nx % Nx) + Nx) % Nx;
    pt->dym[i] = ((fp.ny % Ny) + Ny) % Ny;
    for (int k = 0; k < 9; ++k) pt->mom[k][i] = (CT)r[k];
    for (int k = 0; k < NJ; ++k) pt->cj[k][i] = (CT)r[9 + k];
    pt->vx[i] = (CT)r[19];
    pt->vy[i] = (CT)r[20];
  }
}

template void fill_pop_table<double>(const StencilBuild&, int, int, PopTable<double>*);
template void fill_pop_table<float>(const StencilBuild&, int, int, PopTable<float>*);

// --------------------------------------------------------- R(zeta) tables
// For every slice [2^e (1 + j/8), 2^e (1 + (j+1)/8)) the Chebyshev series of
// R in the local variable x in [-1, 1] (zeta = 2^e (1 + (j + 1/2 + x/2)/8)) is
// computed from 16 Chebyshev nodes in binary128, truncated to the table
// degree and converted to monomial coefficients (kernels use Horner).
static void fit_slice(int e, int j, int ncoef, qf* mono) {
  const int N = 16;
  qf f[N], xs[N];
  const qf scale = (qf)std::ldexp(1.0, e);
  for (int k = 0; k < N; ++k) {
    // nodes in binary128: FP64 nodes break the discrete orthogonality at the
    // 1e-16 level, which leaks the O(1) leading coefficient into the small ones
    xs[k] = q_cos(q_pi * ((qf)k + (qf)0.5) / (qf)N);
    const qf z = scale * (1 + ((qf)j + (qf)0.5 + xs[k] / 2) / 8);
    f[k] = bessel_ratio_q(z, 24.0);   // 24 digits: ample for FP64 coefficients
  }
  // Chebyshev coefficients c_n = (2/N) sum_k f_k T_n(x_k)
  qf c[N];
  for (int n = 0; n < ncoef; ++n) {
    qf s = 0;
    for (int k = 0; k < N; ++k) {
      qf t0 = 1, t1 = xs[k], tn = (n == 0) ? t0 : t1;
      for (int q = 2; q <= n; ++q) {
        tn = 2 * xs[k] * t1 - t0;
        t0 = t1;
        t1 = tn;
      }
      s += f[k] * tn;
    }
    c[n] = s * 2 / N;
  }
  c[0] /= 2;
  // monomial form: accumulate c_n T_n(x) with T_n built as coefficient arrays
  std::vector<qf> Tm2(ncoef, 0), Tm1(ncoef, 0), Tn(ncoef, 0);
  for (int q = 0; q < ncoef; ++q) mono[q] = 0;
  Tm2[0] = 1;                                       // T_0
  mono[0] += c[0];
  if (ncoef > 1) {
    Tm1[1] = 1;                                     // T_1
    mono[1] += c[1];
  }
  for (int n = 2; n < ncoef; ++n) {
    for (int q = 0; q < ncoef; ++q) Tn[q] = -Tm2[q] + ((q > 0) ? 2 * Tm1[q - 1] : (qf)0);
    for (int q = 0; q < ncoef; ++q) mono[q] += c[n] * Tn[q];
    Tm2 = Tm1;
    Tm1 = Tn;
  }
}

struct RatioTables {
  std::vector<double> t64;
  std::vector<float> t32;
  RatioTables() : t64((size_t)RT_NSEG * RT_NC64), t32((size_t)RT_NSEG * RT_NC32) {
    qf mono[RT_NC64];
    for (int e = RT_EMIN; e < RT_EMAX; ++e) {
      for (int j = 0; j < RT_SEG; ++j) {
        const int seg = (e - RT_EMIN) * RT_SEG + j;
        fit_slice(e, j, RT_NC64, mono);
        for (int q = 0; q < RT_NC64; ++q) t64[(size_t)seg * RT_NC64 + q] = (double)mono[q];
        fit_slice(e, j, RT_NC32, mono);
        for (int q = 0; q < RT_NC32; ++q) t32[(size_t)seg * RT_NC32 + q] = (float)(double)mono[q];
      }
    }
  }
};

static const RatioTables& tables() {
  static const RatioTables t;   // thread-safe one-time construction
  return t;
}

const std::vector<double>& ratio_table64() { return tables().t64; }
const std::vector<float>& ratio_table32() { return tables().t32; }

// Host mirror of ratio64 / ratio32 in rlbm_kernels.cuh (same formulas).
template <typename R_t>
static R_t ratio_outside_host(R_t z) {
  if (z < R_t(1)) {
    const R_t ge = R_t(0.57721566490153286061);
    const R_t z2 = z * z;
    return R_t(0.5) * z * (R_t(1) + R_t(0.25) * z2 + R_t(0.5) * z2 * (std::log(R_t(0.5) * z) + ge - R_t(0.5)));
  }
  const R_t u = R_t(1) / z;
  const R_t p1 = R_t(1) + u * (R_t(0.375) + u * (R_t(-0.1171875) + u * R_t(0.1025390625)));
  const R_t p2 = R_t(1) + u * (R_t(1.875) + u * (R_t(0.8203125) + u * R_t(-0.3076171875)));
  return p1 / p2;
}

double ratio_eval_host(double z, int precision) {
  if (!(z > 0) || !std::isfinite(z)) return std::nan("");
  if (precision == 32) {
    const float zf = (float)z;
    int bits;
    std::memcpy(&bits, &zf, 4);
    const int e = ((bits >> 23) & 0xff) - 127;
    if (e < RT_EMIN || e >= RT_EMAX) return ratio_outside_host<float>(zf);
    const int j = (bits >> 20) & 7;
    const int db = ((bits & 0xFFFFF) << 3) | 0x3F800000;
    float d;
    std::memcpy(&d, &db, 4);
    const float x = 2.0f * d - 3.0f;
    const float* c = ratio_table32().data() + ((e - RT_EMIN) * RT_SEG + j) * RT_NC32;
    float r = c[RT_NC32 - 1];
    for (int k = RT_NC32 - 2; k >= 0; --k) r = std::fma(r, x, c[k]);
    return r;
  }
  long long bits;
  std::memcpy(&bits, &z, 8);
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;
  if (e < RT_EMIN || e >= RT_EMAX) return ratio_outside_host<double>(z);
  const int j = (int)((bits >> 49) & 7);
  const long long db = ((bits & ((1LL << 49) - 1)) << 3) | 0x3FF0000000000000LL;
  double d;
  std::memcpy(&d, &db, 8);
  const double x = 2.0 * d - 3.0;
  const double* c = ratio_table64().data() + ((e - RT_EMIN) * RT_SEG + j) * RT_NC64;
  double r = c[RT_NC64 - 1];
  for (int k = RT_NC64 - 2; k >= 0; --k) r = std::fma(r, x, c[k]);
  return r;
}

// dR(Td) per slice: Chebyshev interpolation at 16 nodes of the slice (R from
// the FP64 table, differences in extended precision), truncated to degree
// DR_NC - 1 and rewritten as monomials in the kernels' local variable x.
std::vector<double> dr_table(double mbar) {
  using ld = long double;
  std::vector<double> tab((size_t)DR_NSEG * DR_NC, 0.0);
  const ld Rm = (ld)ratio_eval_host(mbar, 64);
  const int N = 16;
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int seg = 0; seg < DR_NSEG; ++seg) {
    // slice [a, a + 1/64) in Td, x = 64 (Td - c) with c the end nearest 0
    const bool pos = seg >= DR_NNEG;
    const int k = pos ? seg - DR_NNEG : -(DR_NNEG - 1 - seg);   // c = k/64 (k <= 0 below)
    const ld c = (ld)k / 64;
    // t in [-1, 1] -> x = (t + 1)/2 (pos) or (t - 1)/2 (neg)
    ld f[N], ts[N];
    for (int q = 0; q < N; ++q) {
      ts[q] = std::cos(pi * ((ld)q + 0.5L) / N);
      const ld x = pos ? (ts[q] + 1) / 2 : (ts[q] - 1) / 2;
      const ld T = 1 + c + x / 64;
      f[q] = (ld)ratio_eval_host((double)((ld)mbar / T), 64) - Rm;
    }
    ld ch[DR_NC];
    for (int n = 0; n < DR_NC; ++n) {
      ld acc = 0;
      for (int q = 0; q < N; ++q) acc += f[q] * std::cos((ld)n * pi * ((ld)q + 0.5L) / N);
      ch[n] = acc * 2 / N;
    }
    ch[0] /= 2;
    // Chebyshev -> monomials in t
    ld mt[DR_NC] = {}, Tm2[DR_NC] = {}, Tm1[DR_NC] = {}, Tn[DR_NC] = {};
    Tm2[0] = 1;
    mt[0] += ch[0];
    Tm1[1] = 1;
    mt[1] += ch[1];
    for (int n = 2; n < DR_NC; ++n) {
      for (int q = 0; q < DR_NC; ++q) Tn[q] = -Tm2[q] + (q > 0 ? 2 * Tm1[q - 1] : 0);
      for (int q = 0; q < DR_NC; ++q) mt[q] += ch[n] * Tn[q];
      for (int q = 0; q < DR_NC; ++q) {
        Tm2[q] = Tm1[q];
        Tm1[q] = Tn[q];
      }
    }
    // t = 2x - 1 (pos) or 2x + 1 (neg): expand sum mt[n] t^n in x
    const ld b = pos ? -1 : 1;
    ld mx[DR_NC] = {};
    ld pw[DR_NC] = {};   // coefficients of (2x + b)^n
    pw[0] = 1;
    for (int n = 0; n < DR_NC; ++n) {
      for (int q = 0; q <= n; ++q) mx[q] += mt[n] * pw[q];
      ld nx[DR_NC] = {};
      for (int q = 0; q <= n && q + 1 < DR_NC; ++q) {
        nx[q + 1] += 2 * pw[q];
        nx[q] += b * pw[q];
      }
      for (int q = 0; q < DR_NC; ++q) pw[q] = nx[q];
    }
    for (int q = 0; q < DR_NC; ++q) tab[(size_t)seg * DR_NC + q] = (double)mx[q];
  }
  return tab;
}

}  // namespace rlbm
