"""Discrete equilibrium f_i^eq (Eq. 16), by two independent routes.

Route (i), the paper's: f_i^eq = n w_i sum_k b^(k)(U, T) J^(k)(p_i) with the
App. A polynomials and the (corrected) App. B projections.

Route (ii), basis free: the discrete equilibrium is the unique
w_i * (polynomial of degree <= 2 in p_i) whose discrete moments against every
monomial phi_j of degree <= 2 equal the continuum Maxwell-Juttner moments
(that is what a second-order truncation recovers, Sec. II A item 2 and
Sec. III C).  With G_jl = sum_i w_i phi_j(p_i) phi_l(p_i) and the closed-form
moments mu_j per unit density

    int f phi d^3p/p0:  1 -> K1(zeta)/(m K2(zeta))            (Eq. 38, 44)
                        p^a -> U^a                            (Eq. 7)
                        p^a p^b -> (e+P) U^a U^b - P eta^ab   (Eq. 8, 28-29)

f_i^eq = n w_i sum_j c_j phi_j(p_i) with G c = mu.

TEST INFRASTRUCTURE ONLY (see the package docstring)."""
import numpy as np

from . import polynomials as P
from . import special as S

ETA = np.diag([1.0, -1.0, -1.0, -1.0])


def feq_route_i(w, p, n, U, T, consts):
    """w[Q], p[Q,4]; n[...], U[...,4], T[...] -> f[Q, ...] (route (i))."""
    Jp = P.J(p, consts)                       # [Q, 14]
    bk = P.b(U, T, consts)                    # [..., 14]
    return np.asarray(n)[None] * w.reshape((-1,) + (1,) * np.ndim(n)) * np.tensordot(Jp, bk, axes=([1], [-1]))


def _monomials(p, two_d):
    p0, px, py, pz = p[..., 0], p[..., 1], p[..., 2], p[..., 3]
    if two_d:
        cols = [np.ones_like(p0), p0, px, py, p0 * px, p0 * py, px * px, py * py, px * py, pz * pz]
    else:
        cols = [np.ones_like(p0), p0, px, py, pz, p0 * px, p0 * py, p0 * pz,
                px * px, py * py, pz * pz, px * py, px * pz, py * pz]
    return np.stack(cols, axis=-1)


def continuum_moments(U, T, mbar, two_d):
    """Closed-form moments mu_j per unit density of the Maxwell-Juttner
    distribution for the monomials of ``_monomials`` (see module doc)."""
    T = np.asarray(T, dtype=np.float64)
    zeta = mbar / T
    r12 = S.bessel_ratio_k1k2(zeta)
    e_over_n = 3.0 * T + mbar * r12          # Eq. 28
    p_over_n = T                             # Eq. 29
    h = e_over_n + p_over_n

    def Tab(a, bb):
        return h * U[..., a] * U[..., bb] - p_over_n * ETA[a, bb]

    s0 = r12 / mbar
    if two_d:
        cols = [s0, U[..., 0], U[..., 1], U[..., 2], Tab(0, 1), Tab(0, 2),
                Tab(1, 1), Tab(2, 2), Tab(1, 2), Tab(3, 3)]
    else:
        cols = [s0, U[..., 0], U[..., 1], U[..., 2], U[..., 3], Tab(0, 1), Tab(0, 2), Tab(0, 3),
                Tab(1, 1), Tab(2, 2), Tab(3, 3), Tab(1, 2), Tab(1, 3), Tab(2, 3)]
    return np.stack(cols, axis=-1)


def feq_route_ii(w, p, n, U, T, mbar, two_d):
    """Basis-free discrete equilibrium (route (ii)); f[Q, ...]."""
    phi = _monomials(p, two_d)                # [Q, J]
    scale = np.sqrt(np.einsum("i,ij->j", w, phi * phi))   # column equilibration only
    phi = phi / scale
    G = np.einsum("i,ij,ik->jk", w, phi, phi)
    mu = continuum_moments(U, T, mbar, two_d) / scale   # [..., J]
    c = np.linalg.solve(G, mu.reshape(-1, mu.shape[-1]).T).T.reshape(mu.shape)
    return np.asarray(n)[None] * w.reshape((-1,) + (1,) * np.ndim(n)) * np.tensordot(phi, c, axes=([1], [-1]))
