"""Taylor-Green decay of the oracle against the viscosity predicted from tau.

Sec. IV relates tau to the shear viscosity by Grad's eta = (2/3) P (tau - dt/2)
and warns that the link is approximate.  The test checks two predictions:

1. Prefactor free: the decay rate is proportional to (tau - 1/2) (lattice
   units, dt = 1 step), so rates at tau = 0.6 and 0.9 are in the ratio 1 : 4.
2. Absolute: the Chapman-Enskog shear stress of the lattice equation itself.
   With populations moving n_i = p_i/(p0_i v0) cells per step and the
   relaxation weight p.U/(p0 tau) = 1/tau at rest, the non-equilibrium stress
   is -(tau - 1/2) sum_i p^a p^b (n_i . grad) f_i^eq, and with
   d f_i^eq / d u_x = n w_i p_i^x / B^2 at rest (App. A/B) the momentum
   equation of the Taylor-Green mode u_x = u0 sin(kx) cos(ky) gives the
   velocity decay rate per step
       lambda = (tau - 1/2) n (S4 - S22) k^2 / (B^2 v0^2 (e + P)),
   S4 = sum_i w_i p_x^4 / p0,  S22 = sum_i w_i p_x^2 p_y^2 / p0.
   (For an isotropic stencil S4 = 3 S22 and lambda = (tau-1/2) n S22 |k|^2 / ...;
   the 1/p0 factor makes the second-order quadratures slightly anisotropic.)
   The kinetic energy decays at 2 lambda.  Grad's value replaces
   n (S4 - S22)/(2 B^2) by (2/3) P; at m/T = 1 it is about 25 % low.
"""
import numpy as np
import pytest

from oracle import lattice as L
from oracle import polynomials as P
from oracle import quadrature as QD

M1 = ([5, 12, 14, 17, 21, 26], 1.0, 0.23342)


def _decay_rate(tau, N=48, steps=160, u0=0.01):
    lat = L.make_lattice(*M1, tau, (N, N))
    k = 2 * np.pi / N
    x = np.arange(N)
    X, Y = np.meshgrid(x, x)
    lat.init(np.ones((N, N)), u0 * np.sin(k * X) * np.cos(k * Y), -u0 * np.cos(k * X) * np.sin(k * Y),
             np.ones((N, N)))
    ts, E = [], []
    for s in range(steps + 1):
        if s % 8 == 0 and s >= steps // 4:
            mac = lat.macros()
            ts.append(s)
            E.append(0.5 * np.sum(mac["ux"] ** 2 + mac["uy"] ** 2))
        if s < steps:
            lat.step(1)
    rate = -np.polyfit(np.array(ts), np.log(np.array(E)), 1)[0]
    return rate, k, lat


@pytest.fixture(scope="module")
def rates():
    return {tau: _decay_rate(tau) for tau in (0.6, 0.9)}


def test_rate_scales_with_tau_minus_half(rates):
    r6, r9 = rates[0.6][0], rates[0.9][0]
    assert abs((r9 / r6) / 4.0 - 1) < 0.02


def test_rate_matches_lattice_chapman_enskog(rates):
    st = QD.Stencil(*M1)
    w, p, _, _ = st.populations3d()
    c = P.Constants(st.mbar)
    S4 = np.sum(w * p[:, 1] ** 4 / p[:, 0])
    S22 = np.sum(w * (p[:, 1] * p[:, 2]) ** 2 / p[:, 0])
    for tau, (rate, k, lat) in rates.items():
        e = float(np.mean(lat.macros()["e"]))
        n, Pr = 1.0, 1.0
        lam = (tau - 0.5) * n * (S4 - S22) * k * k / (c.B ** 2 * st.v0 ** 2 * (e + Pr))
        assert abs(rate / (2 * lam) - 1) < 0.03, (tau, rate, 2 * lam)
        grad = (tau - 0.5) * (2.0 / 3.0) * Pr * 2 * k * k / (st.v0 ** 2 * (e + Pr))
        assert 1.15 < rate / (2 * grad) < 1.5
