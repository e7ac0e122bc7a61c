"""Pins of the oracle's lattice step (Eq. 19-20, 28-29, 49) against
invariants, limits, special cases and brute force."""
import math

import numpy as np
import pytest
import scipy.optimize as so

from oracle import lattice as L
from oracle import quadrature as QD
from oracle import special as S

M1 = ([5, 12, 14, 17, 21, 26], 1.0, 0.23342)
G1_6 = ([1, 2, 3, 4, 5, 6], 5.0, 0.398)


def _smooth_state(lat, seed, du=0.1, dT=0.2):
    rng = np.random.default_rng(seed)
    shp = lat.shape
    n = 1 + 0.2 * (rng.random(shp) - 0.5)
    T = 1 + dT * (rng.random(shp) - 0.5)
    ux = du * (rng.random(shp) - 0.5)
    uy = du * (rng.random(shp) - 0.5)
    lat.init(n, ux, uy, T)
    return n, ux, uy, T


# ---------------------------------------------------------------- EOS (Sec. II B)
def test_eos_limits():
    # T8: zeta K1/K2 -> 0 as zeta -> 0 (e -> 3nT, Eq. 27); zeta K1/K2 - zeta -> -3/2
    # as zeta -> inf (e_c -> 3/2 nT, Eq. 30).
    z = np.array([1e-3, 1e-2])
    assert np.all(z * S.bessel_ratio_k1k2(z) < 2 * z * z)
    zl = np.array([1e3, 1e4])
    assert np.all(np.abs(zl * S.bessel_ratio_k1k2(zl) - zl + 1.5) < 2.0 / zl)


def test_eos_ratio_eq31():
    # Eq. 31: e/(3nT) = 1 + (1/3)(m/T) K1/K2 from Eq. 28; monotone in T for fixed m.
    T = np.linspace(0.05, 20, 400)
    ratio = 1 + (1 / 3) * (1.0 / T) * S.kv(1, 1.0 / T) / S.kv(2, 1.0 / T)
    assert np.all(np.diff(ratio) < 0) and ratio[-1] < 1.01 and ratio[0] > 1.3


@pytest.mark.parametrize("m", [0.01, 0.36, 1.0, 5.0])
def test_temperature_inversion(m):
    # The bracketed Newton inverts Eq. 28 to round-off over zeta in [1e-3, 1e3];
    # checked against an independent library root finder (brentq).
    T = m / np.logspace(-3, 3, 25)
    e_over_n = 3 * T + m * S.bessel_ratio_k1k2(m / T)
    Tn = L.temperature(e_over_n, m)
    # e/n ~ m + 1.5 T at large zeta: rounding of e/n alone moves T by ~eps zeta
    cond = np.maximum(1.0, m / T)
    assert np.max(np.abs(Tn / T - 1) / cond) < 5e-15
    for y, t in zip(e_over_n[::6], T[::6]):
        tb = so.brentq(lambda x: 3 * x + m * S.bessel_ratio_k1k2(m / x) - y, (y - m) / 3, (y - m) / 1.5,
                       xtol=1e-300, rtol=1e-15)
        assert abs(tb / t - 1) < 1e-14 * max(1.0, m / t)


# --------------------------------------------------------- Landau (Eq. 19-20)
def _power_landau(Tmn):
    """Independent Landau solve: power iteration on T^a_b (dominant eigenvalue
    is the energy density because e > P >= 0)."""
    eta = np.diag([1.0, -1.0, -1.0])
    M = Tmn @ eta
    U = np.array([1.0, 0.0, 0.0])
    for _ in range(400):
        U = M @ U
        U = U / math.sqrt(U[0] ** 2 - U[1] ** 2 - U[2] ** 2)
    e = (U @ eta) @ Tmn @ (eta @ U)
    return e, U


def test_landau_matches_power_iteration():
    lat = L.make_lattice(*M1, 0.8, (4, 5))
    _smooth_state(lat, 3, du=0.6)
    lat.f = lat.f * (1 + 0.05 * np.random.default_rng(4).standard_normal(lat.f.shape))
    N, Tmn = lat.moments()
    e, U = L.landau(Tmn, 3)
    for j in range(4):
        for i in range(5):
            e2, U2 = _power_landau(Tmn[j, i])
            assert abs(e2 / e[j, i] - 1) < 1e-13
            assert np.max(np.abs(U2 - U[j, i])) < 1e-13


# ------------------------------------------------------- macros round trip
@pytest.mark.parametrize("st", [M1, G1_6])
def test_equilibrium_round_trip(st):
    # Init f = f^eq(n, U, T); the macros of f^eq give back (n, u, T).
    lat = L.make_lattice(*st, 0.8, (6, 7))
    n, ux, uy, T = _smooth_state(lat, 1, du=0.6, dT=0.8)
    mac = lat.macros()
    assert np.max(np.abs(mac["n"] / n - 1)) < 1e-13
    assert np.max(np.abs(mac["T"] / T - 1)) < 1e-13
    assert np.max(np.abs(mac["ux"] - ux)) < 1e-13 and np.max(np.abs(mac["uy"] - uy)) < 1e-13


# ------------------------------------------------- collision invariants (T9)
@pytest.mark.parametrize("st", [M1, G1_6])
def test_collision_conserves_N0_T0nu(st):
    # Sec. II A: the collision conserves U.N and U.T; with the Landau frame this
    # fixes N^0 and T^{0 nu} per site (not N^x, T^xx: the non-equilibrium parts
    # are only orthogonal to U).
    lat = L.make_lattice(*st, 0.7, (5, 6))
    _smooth_state(lat, 2, du=0.5)
    lat.f = lat.f * (1 + 0.1 * np.random.default_rng(5).standard_normal(lat.f.shape))
    N0, T0 = lat.moments()
    fs = lat.collide()
    N1, T1 = lat.moments(fs)
    assert np.max(np.abs(N1[..., 0] / N0[..., 0] - 1)) < 1e-13
    rel = np.abs(T1[..., 0, :] - T0[..., 0, :]) / np.abs(T0[..., 0, 0])[..., None]
    assert np.max(rel) < 1e-13
    # the spatial flux N^x does relax
    assert np.max(np.abs(N1[..., 1] - N0[..., 1])) > 1e-6


def test_planted_sign_error_breaks_conservation():
    # Planted mistake: weight (p0 U0 + p.U)/(p0 tau) instead of p.U/(p0 tau).
    lat = L.make_lattice(*M1, 0.7, (4, 4))
    _smooth_state(lat, 2, du=0.5)
    lat.f = lat.f * (1 + 0.1 * np.random.default_rng(5).standard_normal(lat.f.shape))
    mac = lat.macros()
    feq = lat.equilibrium(mac["n"], mac["U"], mac["T"])
    U = mac["U"].reshape(-1, 4)
    pU = lat.p[:, 0, None] * U[:, 0] + lat.p[:, 1, None] * U[:, 1] + lat.p[:, 2, None] * U[:, 2]
    omega = (pU / (lat.p[:, 0, None] * lat.tau)).reshape(lat.f.shape)
    bad = lat.f - omega * (lat.f - feq)
    N0, _ = lat.moments()
    N1, _ = lat.moments(bad)
    assert np.max(np.abs(N1[..., 0] / N0[..., 0] - 1)) > 1e-6


@pytest.mark.parametrize("st", [M1, G1_6])
def test_global_conservation_over_steps(st):
    lat = L.make_lattice(*st, 0.75, (12, 10))
    _smooth_state(lat, 6, du=0.3)
    N, Tm = lat.moments()
    tot0 = (N[..., 0].sum(), Tm[..., 0, 0].sum(), Tm[..., 0, 1].sum(), Tm[..., 0, 2].sum())
    lat.step(5)
    N, Tm = lat.moments()
    tot1 = (N[..., 0].sum(), Tm[..., 0, 0].sum(), Tm[..., 0, 1].sum(), Tm[..., 0, 2].sum())
    scale = abs(tot0[1])
    assert all(abs(a - b) < 1e-12 * scale for a, b in zip(tot0, tot1))


# ------------------------------------------------------ stationarity (T13)
def test_uniform_state_is_stationary():
    lat = L.make_lattice(*M1, 0.9, (5, 8))
    lat.init(np.full((5, 8), 0.7), np.full((5, 8), 0.2), np.full((5, 8), -0.1), np.full((5, 8), 1.3))
    f0 = lat.f.copy()
    lat.step(4)
    assert np.max(np.abs(lat.f - f0) / np.abs(f0)) < 1e-13


# ------------------------------------------------------ streaming (brute force)
def test_stream_brute_force_8x8():
    # Eq. 49: f_i(x + n_i, t + 1) = f*_i(x, t), written as explicit site loops.
    lat = L.make_lattice(*M1, 0.8, (8, 8))
    _smooth_state(lat, 8)
    fs = lat.collide()
    out = lat.stream(fs)
    Ny, Nx = 8, 8
    for i in range(lat.Q):
        dx, dy = int(lat.d[i][0]), int(lat.d[i][1])
        for y in range(Ny):
            for x in range(Nx):
                assert out[i, (y + dy) % Ny, (x + dx) % Nx] == fs[i, y, x]


def test_planted_reversed_stream_detected():
    lat = L.make_lattice(*M1, 0.8, (8, 8))
    _smooth_state(lat, 8)
    fs = lat.collide()
    wrong = np.stack([np.roll(fs[i], shift=(-int(lat.d[i][1]), -int(lat.d[i][0])), axis=(0, 1))
                      for i in range(lat.Q)])
    assert np.max(np.abs(wrong - lat.stream(fs))) > 1e-6


# --------------------------------------------------- fold and 1D == 2D (T10)
def test_fold_equals_unfolded_3d_on_nz1():
    # The folded 2D lattice reproduces the 3D model on an Nx x Ny x 1 lattice.
    st = QD.Stencil(*M1)
    l2 = L.Lattice(st, 0.8, (8, 8), two_d=True)
    l3 = L.Lattice(st, 0.8, (1, 8, 8), two_d=False)
    rng = np.random.default_rng(9)
    n = 1 + 0.1 * rng.random((8, 8))
    T = 1 + 0.2 * rng.random((8, 8))
    ux = 0.2 * (rng.random((8, 8)) - 0.5)
    uy = 0.2 * (rng.random((8, 8)) - 0.5)
    l2.init(n, ux, uy, T)
    l3.init(n[None], ux[None], uy[None], T[None])
    l2.step(3)
    l3.step(3)
    m2, m3 = l2.macros(), l3.macros()
    for k in ("n", "T", "ux", "uy"):
        assert np.max(np.abs(m2[k] - m3[k][0])) < 1e-13, k
    assert np.max(np.abs(m3["uz"])) < 1e-15


def test_quasi_1d_equals_2d():
    # Sec. IV, Fig. 6: a y-uniform 2D run equals the 1D run to machine precision.
    a = L.make_lattice(*M1, 0.7, (1, 40))
    b = L.make_lattice(*M1, 0.7, (6, 40))
    x = np.arange(40)
    n = np.where(x < 20, 1.0, 0.5)
    T = np.where(x < 20, 1.0, 0.8)
    a.init(n[None], 0 * n[None], 0 * n[None], T[None])
    b.init(np.tile(n, (6, 1)), np.zeros((6, 40)), np.zeros((6, 40)), np.tile(T, (6, 1)))
    a.step(10)
    b.step(10)
    ma, mb = a.macros(), b.macros()
    for k in ("n", "T", "ux"):
        assert np.max(np.abs(mb[k] - ma[k])) < 1e-13, k
    assert np.max(np.abs(mb["uy"])) < 1e-14
