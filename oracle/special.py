"""Special functions and rest-frame moments for the oracle.

Extended precision (python ``decimal``, 60 significant digits):

* ``kv_dec(nu, x)``: modified Bessel function of the second kind from its
  integral representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt,
  integrated with the trapezoidal rule, which converges geometrically for
  this entire, even integrand (Trefethen & Weideman, SIAM Rev. 56 (2014)).
* ``rest_moment_dec(name, mbar)``: <phi> = int omega(p0) phi d^3p / p0 with the
  weight omega = exp(-p0/T_R)/N_R of Eq. 36 (T_R = 1) and N_R of Eq. 41, for
  the six monomials phi that fix a second-order quadrature and the eleven
  that fix a third-order one (Sec. III D).

FP64: ``kv`` (scipy's Bessel K, a library routine) and the ratio
R(zeta) = K1(zeta)/K2(zeta) used by the equation of state, Eq. 28.

TEST INFRASTRUCTURE ONLY (see the package docstring)."""
from decimal import Decimal, getcontext

import numpy as np
import scipy.special as sps

PREC = 60
getcontext().prec = PREC

_ONE = Decimal(1)
_TWO = Decimal(2)
_TINY = Decimal(10) ** (-(PREC + 8))


def _dec(x):
    """Decimal value of x; a float enters through its shortest decimal repr
    (0.398 -> Decimal('0.398')), as the paper prints its parameters."""
    if isinstance(x, Decimal):
        return x
    if isinstance(x, int):
        return Decimal(x)
    return Decimal(repr(float(x)))


def _trapezoid_even(fun, h):
    """(h/2) f(0) + h sum_{j>=1} f(j h): the trapezoidal rule for int_0^inf of an
    even integrand that decays double-exponentially; stops once terms are
    negligible and decreasing."""
    total = fun(Decimal(0)) / _TWO
    j = 1
    prev = None
    while True:
        term = fun(h * j)
        total += term
        if prev is not None and abs(term) <= _TINY * abs(total) and abs(term) <= abs(prev):
            break
        prev = term
        j += 1
        if j > 200000:
            raise RuntimeError("trapezoid did not converge")
    return total * h


def _step_for(x, precision_digits=PREC):
    """Trapezoid step for integrands exp(-x cosh t) * (powers of cosh, sinh).

    Analytic in the strip |Im t| < a with |integrand| <= exp(-x cosh(t) cos a),
    the error is about exp(x (1 - cos a) - 2 pi a / h).  For x of order one,
    a = pi/4 gives exp(-pi^2/(2h)); for large x the best a ~ 2 pi/(h x) gives
    exp(-2 pi^2/(h^2 x)).  The step satisfies both for the working precision."""
    import math
    digits = (precision_digits + 10) * math.log(10.0)
    h_small = math.pi ** 2 / (2.0 * digits)
    h_large = math.sqrt(2.0 * math.pi ** 2 / (digits * max(float(x), 1e-300)))
    return Decimal(repr(min(h_small, h_large)))


def kv_dec(nu, x):
    """K_nu(x) in 60-digit decimal arithmetic (integral representation, trapezoid)."""
    x = _dec(x)
    nu = _dec(nu)
    h = _step_for(x)

    def f(t):
        et = t.exp()
        cosh_t = (et + _ONE / et) / _TWO
        enu = (nu * t).exp()
        cosh_nu = (enu + _ONE / enu) / _TWO
        return (-x * cosh_t).exp() * cosh_nu

    return _trapezoid_even(f, h)


# The six monomials of a second-order quadrature (Sec. III D: "6 linearly
# independent components").  For each: (power of p0, power of |p|, angular mean
# of the direction factor over the unit sphere).
#   1, p0, p_x^2, p0 p_x^2, p_x^4, p_x^2 p_y^2
# <n_x^2> = 1/3, <n_x^4> = 1/5, <n_x^2 n_y^2> = 1/15 over the unit sphere.
MONOMIALS6 = ("1", "p0", "px2", "p0px2", "px4", "px2py2")
# Third order (Sec. III D: eleven independent conditions): exactness for every
# product of two polynomials of degree <= 3, i.e. every on-shell monomial of
# degree <= 6.  With p0^2 = mbar^2 + |p|^2 at every node and odd monomials
# vanishing on both sides, five more conditions join the six:
#   p0 p_x^4, p0 p_x^2 p_y^2, p_x^6, p_x^4 p_y^2, p_x^2 p_y^2 p_z^2
# (<n_x^6> = 1/7, <n_x^4 n_y^2> = 1/35, <n_x^2 n_y^2 n_z^2> = 1/105).
MONOMIALS11 = MONOMIALS6 + ("p0px4", "p0px2py2", "px6", "px4py2", "px2py2pz2")
_MONO_SPEC = {
    "1": (0, 0, Decimal(1)),
    "p0": (1, 0, Decimal(1)),
    "px2": (0, 2, Decimal(1) / Decimal(3)),
    "p0px2": (1, 2, Decimal(1) / Decimal(3)),
    "px4": (0, 4, Decimal(1) / Decimal(5)),
    "px2py2": (0, 4, Decimal(1) / Decimal(15)),
    "p0px4": (1, 4, Decimal(1) / Decimal(5)),
    "p0px2py2": (1, 4, Decimal(1) / Decimal(15)),
    "px6": (0, 6, Decimal(1) / Decimal(7)),
    "px4py2": (0, 6, Decimal(1) / Decimal(35)),
    "px2py2pz2": (0, 6, Decimal(1) / Decimal(105)),
}


def rest_moment_dec(name, mbar):
    """int omega(p0) phi(p) d^3p/p0 for omega of Eq. 36 normalised by Eq. 40-41 (T_R = 1).

    In rapidity chi (p0 = m cosh chi, |p| = m sinh chi) the measure d^3p/p0 is
    m^2 sinh^2(chi) dchi dOmega, so with N_R = 4 pi mbar K1(mbar):
      <phi> = <angular> int_0^inf e^{-m cosh} (m cosh)^a (m sinh)^(b+2) dchi / (m K1(m)).
    """
    m = _dec(mbar)
    a, b, ang = _MONO_SPEC[name]
    h = _step_for(m)

    def f(c):
        ec = c.exp()
        ch = (ec + _ONE / ec) / _TWO
        sh = (ec - _ONE / ec) / _TWO
        return (-m * ch).exp() * (m * ch) ** a * (m * sh) ** (b + 2)

    integral = _trapezoid_even(f, h)
    return ang * integral / (m * kv_dec(1, m))


def kv(nu, x):
    """FP64 K_nu(x) (scipy library routine)."""
    return sps.kv(nu, x)


def bessel_ratio_k1k2(zeta):
    """R(zeta) = K1(zeta)/K2(zeta) in FP64, via exponentially scaled Bessel
    functions so that large zeta does not underflow."""
    zeta = np.asarray(zeta, dtype=np.float64)
    return sps.kve(1, zeta) / sps.kve(2, zeta)
