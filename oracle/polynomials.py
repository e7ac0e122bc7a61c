"""Second-order orthonormal polynomials (App. A) and projections (App. B).

All quantities are adimensional, momenta in units of T_R (T_R = 1 here, so
mbar = m).  The fourteen polynomials are ordered

    0: J^(0)      1: J_0    2: J_x    3: J_y    4: J_z
    5: J_00       6: J_0x   7: J_0y   8: J_0z
    9: J_xx      10: J_yy  11: J_xz  12: J_yz  13: J_xy

with the App. A definitions as printed (spatial components are the
contravariant p^x, p^y, p^z of Eq. 48).

App. B is used with three corrections (each derived by carrying out the
projection integral Eq. 15 against the App. A polynomial with the closed-form
equilibrium moments Eq. 7-8, 28-29; the tests check every b^(k) against an
independent projection):

1. The expressions printed for b_xx and b_yy are exchanged: the one printed
   as b_yy, mbar K3/K2(zeta) (U_y^2 - U_z^2)/(2E), is the projection on
   J_xx = (p_y^2 - p_z^2)/(2E), and vice versa.
2. The expressions printed for b_yz and b_xy are exchanged: mbar K3/K2 U_x U_y/E
   is the projection on J_xy, mbar K3/K2 U_y U_z/E the one on J_yz.
3. b_00: the U_0 coefficient is 3(1/X - 1), where X is the denominator that
   appears in J_00 (J_00 has p0 (3/X - 3)), and the last term is -T/T_R:
   b_00 = [mbar K3/K2(zeta) U_0^2 + 3(1/X - 1) U_0 + K1/K2(zeta) Y - T/T_R]/(sqrt3 C)
   with Y the mbar-fraction printed in b_00.

TEST INFRASTRUCTURE ONLY (see the package docstring)."""
import math

import numpy as np

from . import special as S

NPOLY = 14


class Constants:
    """The mbar-only constants of App. A: A, B, C, D, E and the Bessel values.

    They are evaluated in 60-digit decimal arithmetic (``special.kv_dec``) and
    rounded to FP64 once: X, Y and the J_00 constant are differences of
    nearly equal Bessel products (at mbar = 5 they lose more than a decade),
    and FP64 evaluation would leave ~1e-13 errors in the equilibrium moments."""

    def __init__(self, mbar):
        m = S._dec(mbar)
        self.mbar = float(m)
        k1, k2, k3 = (S.kv_dec(n, m) for n in (1, 2, 3))
        self.k1, self.k2, self.k3 = float(k1), float(k2), float(k3)
        self.k21 = float(k2 / k1)          # K2/K1 (mbar)
        self.k32 = float(k3 / k2)          # K3/K2 (mbar)
        self.A = float((m * (m + k2 * (3 * k1 - m * k2) / k1 ** 2)).sqrt())
        self.B = float((m * k2 / k1).sqrt())
        den = m * k1 ** 2 + 3 * k2 * k1 - m * k2 ** 2
        self.C = float((2 * m ** 2 + 5 * m * k2 / k1 - 3 * k1 * (m * k1 + 3 * k2) / den + 3).sqrt())
        self.D = float((m ** 2 * (m * k2 ** 2 + 5 * k3 * k2 - m * k3 ** 2) / (k1 * k2)).sqrt())
        self.E = float((m ** 2 * k3 / k1).sqrt())
        # J_00 = (p0^2 + cJ00_1 p0 + cJ00_0)/(sqrt3 C), cJ00_1 = 3/X - 3
        X = -m * k1 / k2 + m * k2 / k1 - 3
        self.X = float(X)
        self.cJ00_1 = float(3 / X - 3)                         # p0 coefficient of J_00
        self.cJ00_0 = float(3 * k1 * (m * k1 + 3 * k2) / den - m ** 2 - 3)   # constant of J_00
        self.cb00_1 = float(3 * (1 / X - 1))                   # U_0 coefficient of b_00
        # b_00 mbar fraction
        self.Y = float((-m ** 2 * k1 ** 2 + (m ** 2 + 3) * k2 ** 2 - 3 * m * k2 * k1) / den)


def J(p, c):
    """The 14 polynomials of App. A at momenta p[..., 4] = (p0, px, py, pz); returns [..., 14]."""
    p0, px, py, pz = p[..., 0], p[..., 1], p[..., 2], p[..., 3]
    m = c.mbar
    s3 = math.sqrt(3.0)
    out = np.empty(p.shape[:-1] + (NPOLY,))
    out[..., 0] = 1.0
    out[..., 1] = (p0 - m * c.k21) / c.A
    out[..., 2] = px / c.B
    out[..., 3] = py / c.B
    out[..., 4] = pz / c.B
    out[..., 5] = (p0 ** 2 + p0 * c.cJ00_1 + c.cJ00_0) / (s3 * c.C)
    shift = m * c.k32
    out[..., 6] = px * (p0 - shift) / c.D
    out[..., 7] = py * (p0 - shift) / c.D
    out[..., 8] = pz * (p0 - shift) / c.D
    out[..., 9] = (py ** 2 / 2.0 - pz ** 2 / 2.0) / c.E
    out[..., 10] = (-2.0 * px ** 2 + py ** 2 + pz ** 2) / (2.0 * s3 * c.E)
    out[..., 11] = px * pz / c.E
    out[..., 12] = py * pz / c.E
    out[..., 13] = px * py / c.E
    return out


def b(U, T, c):
    """Projections b^(k) of App. B (corrected, see module doc) per unit density,
    for contravariant four-velocity U[..., 4] and temperature T (T_R = 1).
    Returns [..., 14] in the order of ``J``."""
    U0, Ux, Uy, Uz = U[..., 0], U[..., 1], U[..., 2], U[..., 3]
    T = np.asarray(T, dtype=np.float64)
    m = c.mbar
    zeta = m / T
    r12 = S.bessel_ratio_k1k2(zeta)          # K1/K2 (zeta)
    r32 = r12 + 4.0 / zeta                   # K3/K2 (zeta) = K1/K2 + 4/zeta
    s3 = math.sqrt(3.0)
    out = np.empty(U.shape[:-1] + (NPOLY,))
    out[..., 0] = r12 / m
    out[..., 1] = (U0 - c.k21 * r12) / c.A
    out[..., 2] = Ux / c.B
    out[..., 3] = Uy / c.B
    out[..., 4] = Uz / c.B
    out[..., 5] = (m * r32 * U0 ** 2 + c.cb00_1 * U0 + r12 * c.Y - T) / (s3 * c.C)
    k32m = c.k32
    out[..., 6] = (m * r32 * U0 * Ux - m * k32m * Ux) / c.D
    out[..., 7] = (m * r32 * U0 * Uy - m * k32m * Uy) / c.D
    out[..., 8] = (m * r32 * U0 * Uz - m * k32m * Uz) / c.D
    out[..., 9] = m * r32 * (Uy ** 2 - Uz ** 2) / (2.0 * c.E)
    out[..., 10] = m * r32 * (-2.0 * Ux ** 2 + Uy ** 2 + Uz ** 2) / (2.0 * s3 * c.E)
    out[..., 11] = m * r32 * Ux * Uz / c.E
    out[..., 12] = m * r32 * Uy * Uz / c.E
    out[..., 13] = m * r32 * Ux * Uy / c.E
    return out
