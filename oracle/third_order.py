"""Third-order discrete equilibrium (Sec. III A-B at order N = 3, Eq. 14-16).

The paper lists the third-order polynomials and projections only in its
supplemental material, which is not available here, so this module builds
them from their definitions:

* J^(k): the polynomials of degree <= 3 in p^mu, orthonormal under the weight
  omega of Eq. 36 (Sec. III A).  They are the Gram-Schmidt (Cholesky)
  orthonormalisation of a monomial basis under the discrete inner product
  <f, g> = sum_i w_i f(p_i) g(p_i), in 60-digit decimal arithmetic.  On a
  third-order stencil this inner product equals the continuum one for every
  product of degree <= 6 (Eq. 47), so the J^(k) are the paper's polynomials up
  to the choice of basis inside each degree.  The monomials are
  t^a p_x^i p_y^j p_z^l with t = p0 - c, a in {0, 1}, a + i + j + l <= 3:
  p0^2 = mbar^2 + |p|^2 at every node reduces all higher powers of p0.  That
  gives 30 of them for the unfolded stencil (Sec. III A: 30 polynomials at
  third order) and 20 for the folded one (even in p_z).  The shift
  c = <p0>_omega = mbar K2/K1(mbar) only conditions the basis; the span is
  the same for any c.
* a^(k)(U, T) = int f^eq J^(k) d^3p/p0 (Eq. 15) per unit density, from the
  closed-form moments (Eq. 4-6) of the Maxwell-Juttner distribution
  normalised to N^a = n U^a (Eq. 43-44), with h = (e + P)/n = mbar R + 4T and
  R = K1/K2(mbar/T) (Eq. 28-29):
     rank 0:  K1(zeta)/(mbar K2(zeta))
     rank 1:  U^a
     rank 2:  h U^a U^b - T eta^ab
     rank 3:  A3 U^a U^b U^c + B3 (eta^ab U^c + eta^ac U^b + eta^bc U^a),
              A3 = mbar^2 + 6 T h,  B3 = -T h.
  Rank 3 (a reading; the paper only says that higher moments follow from
  differentiating with respect to m/T, Sec. III A): Lorentz covariance leaves
  the two scalars A3, B3.  The trace eta_bc T^abc = mbar^2 N^a gives
  A3 + 6 B3 = mbar^2.  Two derivatives of the normalisation
  4 pi m^2 T K2(m/T) with respect to 1/T give, in the rest frame,
  <E^3> = A3 + 3 B3 = mbar^2 + 3 mbar T R + 12 T^2 (the Bessel recurrences
  of Eq. 38-39 reduce K4 and K3 to K1 and K2).
* f_i^eq = n w_i sum_k a^(k) J^(k)(p_i) (Eq. 16).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from decimal import Decimal

import numpy as np

from . import groups as G
from . import quadrature as QD
from . import special as S

ETA = np.diag([1.0, -1.0, -1.0, -1.0])


def monomial_exponents(two_d):
    """(a, i, j, l) of the basis t^a p_x^i p_y^j p_z^l, lowest degree first."""
    out = []
    for deg in range(4):
        for a in (0, 1):
            r = deg - a
            if r < 0:
                continue
            for i in range(r, -1, -1):
                for j in range(r - i, -1, -1):
                    l = r - i - j
                    if two_d and l % 2:
                        continue
                    out.append((a, i, j, l))
    return out


def mj_moment(idx, U, T, mbar):
    """int f p^idx[0] p^idx[1] ... d^3p/p0 per unit density (rank <= 3), for
    contravariant U[..., 4] and T (see the module docstring)."""
    T = np.asarray(T, dtype=np.float64)
    R = S.bessel_ratio_k1k2(mbar / T)
    r = len(idx)
    if r == 0:
        return R / mbar
    if r == 1:
        return U[..., idx[0]]
    h = mbar * R + 4.0 * T
    if r == 2:
        a, b = idx
        return h * U[..., a] * U[..., b] - T * ETA[a, b]
    if r == 3:
        a, b, c = idx
        A3 = mbar * mbar + 6.0 * T * h
        B3 = -T * h
        return (A3 * U[..., a] * U[..., b] * U[..., c]
                + B3 * (ETA[a, b] * U[..., c] + ETA[a, c] * U[..., b] + ETA[b, c] * U[..., a]))
    raise ValueError("rank <= 3 only")


def _pw(x, k):
    """x^k for decimals with 0^0 = 1."""
    return x ** k if k else Decimal(1)


def _cholesky_inverse_dec(Gm):
    """C = L^{-1} for G = L L^T (decimal, lower triangular)."""
    K = len(Gm)
    L = [[Decimal(0)] * K for _ in range(K)]
    for i in range(K):
        for j in range(i + 1):
            s = Gm[i][j] - sum(L[i][k] * L[j][k] for k in range(j))
            if i == j:
                if s <= 0:
                    raise ValueError("Gram matrix not positive definite: the stencil is not third order")
                L[i][i] = s.sqrt()
            else:
                L[i][j] = s / L[j][j]
    C = [[Decimal(0)] * K for _ in range(K)]
    for i in range(K):
        C[i][i] = Decimal(1) / L[i][i]
        for j in range(i):
            C[i][j] = -sum(L[i][k] * C[k][j] for k in range(j, i)) / L[i][i]
    return C


class ThirdOrder:
    """J^(k) tables and projection matrix of one third-order stencil, folded
    (``two_d``) or unfolded; see the module docstring."""

    def __init__(self, stencil, two_d):
        # Eq. 46-47: orthonormality under the stencil's own weights
        if stencil.order != 3:
            raise ValueError("third-order equilibrium needs an 11-group stencil")
        self.two_d = two_d
        self.mbar = stencil.mbar
        self.expo = monomial_exponents(two_d)
        m = S._dec(stencil.mbar)
        v0 = S._dec(stencil.v0)
        self.c_dec = m * S.kv_dec(2, m) / S.kv_dec(1, m)
        self.c = float(self.c_dec)
        rows = stencil.population_vectors(two_d)
        phis = []
        wd = []
        for k, nx, ny, nz, mult in rows:
            gam = QD._gamma_dec(v0, G.length2(stencil.group_ids[k]))
            s = m * gam * v0
            t = m * gam - self.c_dec
            px, py, pz = s * nx, s * ny, s * nz
            phis.append([_pw(t, a) * _pw(px, i) * _pw(py, j) * _pw(pz, l) for a, i, j, l in self.expo])
            wd.append(S._dec(float(stencil.w_group[k])) * mult)
        K = len(self.expo)
        Gm = [[sum(wd[q] * phis[q][a] * phis[q][b] for q in range(len(rows))) for b in range(K)]
              for a in range(K)]
        C = _cholesky_inverse_dec(Gm)
        self.C = np.array([[float(x) for x in r] for r in C])
        self.J = np.array([[float(sum(C[k][l] * ph[l] for l in range(k + 1))) for k in range(K)]
                           for ph in phis])                       # [Q, K]
        self.K = K

    def monomial_moments(self, U, T):
        """mu_l(U, T) per unit density for the basis monomials; [..., K]."""
        cols = []
        for a, i, j, l in self.expo:
            idx = (1,) * i + (2,) * j + (3,) * l
            mom = mj_moment(idx, U, T, self.mbar)
            if a == 1:
                mom = mj_moment((0,) + idx, U, T, self.mbar) - self.c * mom
            cols.append(np.broadcast_to(mom, np.shape(T)))
        return np.stack(cols, axis=-1)

    def projections(self, U, T):
        """a^(k)(U, T) of Eq. 15 per unit density; [..., K]."""
        return self.monomial_moments(U, T) @ self.C.T

    def feq(self, w, n, U, T):
        """f_i^eq = n w_i sum_k a^(k) J^(k)(p_i) (Eq. 16); f[Q, ...]."""
        a = self.projections(U, T)
        n = np.asarray(n)
        return n[None] * w.reshape((-1,) + (1,) * n.ndim) * np.tensordot(self.J, a, axes=([1], [-1]))
