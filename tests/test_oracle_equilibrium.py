"""Pins of the oracle's polynomials (App. A), projections (App. B, corrected)
and discrete equilibrium (Eq. 16) against closed forms and an independent
projection."""
import math

import numpy as np
import pytest

from oracle import equilibrium as EQ
from oracle import polynomials as P
from oracle import quadrature as QD
from oracle import special as S

G1_6 = [1, 2, 3, 4, 5, 6]
M1 = ([5, 12, 14, 17, 21, 26], 1.0, 0.23342)


@pytest.fixture(scope="module")
def st5():
    return QD.Stencil(G1_6, 5, 0.398)


@pytest.fixture(scope="module")
def st1():
    return QD.Stencil(*M1)


def _fields(shape, seed, umax=0.4):
    rng = np.random.default_rng(seed)
    n = 0.5 + rng.random(shape)
    T = 0.5 + 1.5 * rng.random(shape)
    ang = 2 * math.pi * rng.random(shape)
    sp = umax * rng.random(shape)
    ux, uy = sp * np.cos(ang), sp * np.sin(ang)
    g = 1 / np.sqrt(1 - ux ** 2 - uy ** 2)
    U = np.stack([g, g * ux, g * uy, np.zeros(shape)], -1)
    return n, U, T


@pytest.mark.parametrize("which", ["st5", "st1"])
def test_app_a_orthonormal_on_quadrature(which, request):
    # T5: sum_i w_i J^(l)(p_i) J^(k)(p_i) = delta_lk (Eq. 46-47) with the
    # printed App. A polynomials on a quadrature whose weights are pinned.
    st = request.getfixturevalue(which)
    w, p, _, _ = st.populations3d()
    c = P.Constants(st.mbar)
    Jp = P.J(p, c)
    G = np.einsum("i,ij,ik->jk", w, Jp, Jp)
    assert np.max(np.abs(G - np.eye(P.NPOLY))) < 5e-12


def test_app_a_constants_closed_forms():
    # B^2 = <p_x^2> = mbar K2/K1, E^2 = <p_x^2 p_y^2> = mbar^2 K3/K1 (rest frame).
    for m in (0.36, 1.0, 5.0):
        c = P.Constants(m)
        assert abs(c.B ** 2 / float(S.rest_moment_dec("px2", m)) - 1) < 1e-14
        assert abs(c.E ** 2 / float(S.rest_moment_dec("px2py2", m)) - 1) < 1e-14


@pytest.mark.parametrize("which", ["st5", "st1"])
def test_app_b_projections_match_discrete_projection(which, request):
    # T6: the (corrected) App. B coefficients equal the projections of the
    # route-(ii) equilibrium on the App. A polynomials, sum_i f_i J^(k)(p_i)/n.
    st = request.getfixturevalue(which)
    w, p, _, _ = st.populations3d()
    c = P.Constants(st.mbar)
    n, U, T = _fields((40,), 7)
    U[:, 3] = 0.1 * U[:, 1]                    # a z component too (3D stencil)
    U[:, 0] = np.sqrt(1 + U[:, 1] ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2)
    f2 = EQ.feq_route_ii(w, p, n, U, T, st.mbar, two_d=False)   # [Q, 40]
    proj = np.einsum("is,ik->sk", f2, P.J(p, c)) / n[:, None]
    bk = P.b(U, T, c)
    scale = np.max(np.abs(bk), axis=0)
    assert np.max(np.abs(proj - bk) / scale) < 1e-11


def test_app_b_as_printed_fails_the_projection(st5):
    # Planted mistake: the printed b_00 (U_0 coefficient 1/X - 1, +T) and the
    # printed b_xx/b_yy, b_xy/b_yz labels fail the same check.
    w, p, _, _ = st5.populations3d()
    c = P.Constants(5.0)
    n, U, T = _fields((10,), 3)
    U[:, 3] = 0.2 * U[:, 2]
    U[:, 0] = np.sqrt(1 + U[:, 1] ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2)
    f2 = EQ.feq_route_ii(w, p, n, U, T, 5.0, two_d=False)
    proj = np.einsum("is,ik->sk", f2, P.J(p, c)) / n[:, None]
    bk = P.b(U, T, c)
    printed = bk.copy()
    r32 = S.bessel_ratio_k1k2(5.0 / T) + 4 * T / 5.0
    printed[:, 5] = (5 * r32 * U[:, 0] ** 2 + (1 / c.X - 1) * U[:, 0]
                     + S.bessel_ratio_k1k2(5.0 / T) * c.Y + T) / (math.sqrt(3) * c.C)
    printed[:, [9, 10]] = bk[:, [10, 9]]
    printed[:, [12, 13]] = bk[:, [13, 12]]
    for k in (5, 9, 10, 12, 13):
        assert np.max(np.abs(proj[:, k] - printed[:, k])) > 1e-3


@pytest.mark.parametrize("which", ["st5", "st1"])
def test_discrete_equilibrium_moments_closed_form(which, request):
    # T7: sum_i f_i^eq p_i^a = n U^a (Eq. 7), sum_i f_i^eq p^a p^b = (e+P)U^aU^b - P eta^ab
    # (Eq. 8) with e = 3nT + nm K1/K2 and P = nT (Eq. 28-29), Bessel values
    # from the library routine.
    st = request.getfixturevalue(which)
    w, p, _, _, _ = st.populations2d()
    c = P.Constants(st.mbar)
    n, U, T = _fields((64,), 11)
    f = EQ.feq_route_i(w, p, n, U, T, c)
    m = st.mbar
    z = m / T
    e = n * (3 * T + m * S.kv(1, z) / S.kv(2, z))
    Pn = n * T
    eta = np.diag([1.0, -1.0, -1.0])
    Nd = np.einsum("ia,is->sa", p[:, :3], f)
    Td = np.einsum("ia,ib,is->sab", p[:, :3], p[:, :3], f)
    Ne = n[:, None] * U[:, :3]
    Te = (e + Pn)[:, None, None] * U[:, :3, None] * U[:, None, :3] - Pn[:, None, None] * eta
    assert np.max(np.abs(Nd - Ne) / np.abs(Ne).max(axis=1, keepdims=True)) < 1e-13
    assert np.max(np.abs(Td - Te) / np.abs(Te).max(axis=(1, 2), keepdims=True)) < 1e-13


@pytest.mark.parametrize("which", ["st5", "st1"])
def test_route_i_equals_route_ii_folded(which, request):
    st = request.getfixturevalue(which)
    w, p, _, _, _ = st.populations2d()
    c = P.Constants(st.mbar)
    n, U, T = _fields((5, 9), 5)
    f1 = EQ.feq_route_i(w, p, n, U, T, c)
    f2 = EQ.feq_route_ii(w, p, n, U, T, st.mbar, two_d=True)
    # route (ii) solves a monomial Gram system whose conditioning at mbar = 5
    # limits it to ~5e-13 of max f (its moments still match to ~2e-14)
    assert np.max(np.abs(f1 - f2)) < 1e-12 * np.max(np.abs(f2))


def test_second_order_expansion_tracks_maxwell_juttner():
    # Sec. III B, Fig. 4: the second-order expansion omega(p0) sum_k a_k J_k
    # approximates the MJ distribution; at m = 5, T = 1, u = 0.3 the relative
    # L2 error along p = (p_x, 0, 0) is a few percent at most, while the
    # first-order one is clearly worse.
    m, T, u = 5.0, 1.0, 0.3
    c = P.Constants(m)
    g = 1 / math.sqrt(1 - u * u)
    U = np.array([[g, g * u, 0.0, 0.0]])
    px = np.linspace(-4, 8, 241)
    pv = np.stack([np.sqrt(m * m + px ** 2), px, 0 * px, 0 * px], -1)
    NR = 4 * math.pi * m * S.kv(1, m)
    omega = np.exp(-pv[:, 0]) / NR
    Nmj = 4 * math.pi * m * m * T ** 3 * S.kv(2, m / T)     # Eq. 44, n = 1
    mj = np.exp(-(pv[:, 0] * g - px * g * u) / T) / Nmj
    bk = P.b(U, np.array([T]), c)[0]
    Jv = P.J(pv, c)
    second = omega * (Jv @ bk)
    first = omega * (Jv[:, :5] @ bk[:5])
    err2 = np.linalg.norm(second - mj) / np.linalg.norm(mj)
    err1 = np.linalg.norm(first - mj) / np.linalg.norm(mj)
    assert err2 < 0.1 and err1 > 2 * err2
