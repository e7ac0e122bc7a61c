"""Exact solution of the planar Riemann problem of an ideal (inviscid)
Maxwell-Juttner fluid, used as an outside reference for the shock-tube
workload: a left state of higher pressure at rest, a right state at rest, a
rarefaction running left and a shock running right, joined by a contact at
pressure P* and velocity v* (relativistic Riemann problem; Marti and Muller's
review of numerical relativistic hydrodynamics gives the textbook form).

Units: c = 1, temperatures in units of the reference temperature, m = m/T_R.
Equation of state of the massive Maxwell-Juttner gas (Eq. 28-29 of the
paper): P = n T, e/n = m R + 3 T, enthalpy per particle H = (e + P)/n =
m R + 4 T, R = K1/K2(m/T).  Sound speed c_s^2 = (c_p/c_v) T/H with
c_v = 3 - z^2 R'(z), R' = R^2 + 3 R/z - 1, c_p = c_v + 1 (z = m/T).  Entropy
per particle (up to a constant) s/n = H/T + ln(T K2(z)) - ln n, from
n ~ m^2 T K2(z) exp(mu/T) and s/n = (H - mu)/T.

Across the rarefaction the Riemann invariant atanh(v) + int c_s dn/n is
constant along the isentrope through the left state; across the shock the
three conservation laws [N^x] = V [N^0], [T^0x] = V [T^00], [T^xx] = V [T^0x]
(V the shock speed) hold, solved here in the rest frame of the right state.
This module holds no step of the lattice Boltzmann method; it is test
infrastructure like the oracle, and shares no code with either path."""
import math

from scipy import integrate, optimize, special


def ratio(z):
    """R(z) = K1(z)/K2(z)."""
    return special.kve(1, z) / special.kve(2, z)


def enthalpy(T, m):
    return m * ratio(m / T) + 4.0 * T


def energy(n, T, m):
    return n * (m * ratio(m / T) + 3.0 * T)


def sound_speed(T, m):
    z = m / T
    R = ratio(z)
    cv = 3.0 - z * z * (R * R + 3.0 * R / z - 1.0)
    return math.sqrt((cv + 1.0) / cv * T / enthalpy(T, m))


def entropy_per_particle(n, T, m):
    z = m / T
    return enthalpy(T, m) / T + math.log(T) + math.log(special.kve(2, z)) - z - math.log(n)


def isentrope_T(n, s, m, T_hint):
    """Temperature at density n on the isentrope s/n = s (increasing in T)."""
    f = lambda T: entropy_per_particle(n, T, m) - s
    lo, hi = T_hint, T_hint
    while f(lo) > 0:
        lo *= 0.5
    while f(hi) < 0:
        hi *= 2.0
    return optimize.brentq(f, lo, hi, xtol=1e-15, rtol=1e-14, maxiter=200)


def rarefaction(P, nL, TL, m):
    """(n, T, v) behind a left-running rarefaction from the left state at
    rest down to pressure P < nL TL."""
    s = entropy_per_particle(nL, TL, m)
    T_of_n = lambda n: isentrope_T(n, s, m, TL)
    n = optimize.brentq(lambda n: n * T_of_n(n) - P, 1e-6 * nL, nL, xtol=1e-15, rtol=1e-14)
    rap, _ = integrate.quad(lambda q: sound_speed(T_of_n(q), m) / q, n, nL, epsabs=1e-13, epsrel=1e-12)
    return n, T_of_n(n), math.tanh(rap)


def shock(P, nR, TR, m):
    """(n, T, v, V) behind a right-running shock into the right state at rest
    raised to pressure P > nR TR: post-shock density, temperature, fluid
    velocity and shock speed.  The Taub adiabat H_b^2 - H_a^2 =
    (H_b/n_b + H_a/n_a)(P_b - P_a) fixes n_b; the other laws give
    gamma_b = n_b (e_a + P_b)/(n_a w_b), V = (P_b - P_a)/(v_b (e_a + P_b))."""
    Pa, Ha, ea = nR * TR, enthalpy(TR, m), energy(nR, TR, m)
    taub = lambda nb: enthalpy(P / nb, m) ** 2 - Ha ** 2 - (enthalpy(P / nb, m) / nb + Ha / nR) * (P - Pa)
    # at n_b = n_a the residual is (H_b + H_a)(H_b - H_a - (T_b - T_a)) > 0
    # (dH/dT = c_p > 1); it turns negative at large compression
    nb = optimize.brentq(taub, nR, _bracket_upper(taub, nR), xtol=1e-15, rtol=1e-14, maxiter=400)
    Tb = P / nb
    wb = nb * enthalpy(Tb, m)
    gb = nb * (ea + P) / (nR * wb)
    vb = math.sqrt(max(0.0, 1.0 - 1.0 / (gb * gb)))
    if vb == 0.0:                # vanishing shock: an acoustic wave
        return nb, Tb, 0.0, sound_speed(TR, m)
    V = (P - Pa) / (vb * (ea + P))
    return nb, Tb, vb, float(V)


def _bracket_upper(f, na):
    """A density above the shock's, where the Taub residual is negative."""
    x = na * 1.01
    for _ in range(200):
        if f(x) < 0:
            return x
        x *= 1.2
    raise RuntimeError("no shock density found")


def jump_residuals(a, b, V, m):
    """Relative residuals of the three jump conditions between states
    a = (n, T, v) and b = (n, T, v) across a discontinuity moving at V."""
    def fluxes(n, T, v):
        g2 = 1.0 / (1.0 - v * v)
        g = math.sqrt(g2)
        w = energy(n, T, m) + n * T
        N0, Nx = n * g, n * g * v
        T00, T0x, Txx = w * g2 - n * T, w * g2 * v, w * g2 * v * v + n * T
        return (Nx - V * N0, T0x - V * T00, Txx - V * T0x), (N0, T00, T0x)
    fa, sa = fluxes(*a)
    fb, sb = fluxes(*b)
    return [abs(x - y) / max(abs(s), abs(t), 1e-300) for x, y, s, t in zip(fa, fb, sa, sb)]


def solve(nL, TL, nR, TR, m):
    """Intermediate states of the Riemann problem with both sides at rest
    and nL TL > nR TR: dict with P*, v*, the rarefaction side (nL*, TL*),
    the shock side (nR*, TR*) and the shock speed V."""
    PL, PR = nL * TL, nR * TR
    assert PL > PR
    g = lambda P: rarefaction(P, nL, TL, m)[2] - shock(P, nR, TR, m)[2]
    P = optimize.brentq(g, PR * (1.0 + 1e-9), PL * (1.0 - 1e-9), xtol=1e-15, rtol=1e-13, maxiter=200)
    nl, tl, v = rarefaction(P, nL, TL, m)
    nr, tr, vs, V = shock(P, nR, TR, m)
    return dict(P=P, v=v, v_shock_side=vs, nL=nl, TL=tl, nR=nr, TR=tr, V=V)
