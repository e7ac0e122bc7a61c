"""Pins of the oracle's special functions and rest-frame moments."""
from decimal import Decimal

import numpy as np
import pytest
import scipy.special as sps

from oracle import special as S


@pytest.mark.parametrize("nu", [0, 1, 2, 3])
@pytest.mark.parametrize("x", [0.01, 0.36, 1.0, 5.0, 30.0])
def test_decimal_bessel_matches_library(nu, x):
    # Two independent evaluations: the trapezoidal integral vs scipy's kv.
    assert abs(float(S.kv_dec(nu, x)) / sps.kv(nu, x) - 1) < 1e-15


def test_decimal_bessel_recurrence():
    # K_{nu+1}(x) = K_{nu-1}(x) + (2 nu / x) K_nu(x), checked to 45 digits.
    for x in ("0.2", "1", "7.5"):
        x = Decimal(x)
        k1, k2, k3 = (S.kv_dec(n, x) for n in (1, 2, 3))
        assert abs(k3 - (k1 + 4 / x * k2)) < Decimal("1e-45") * k3


@pytest.mark.parametrize("m", [0.36, 1.0, 5.0])
def test_rest_moments_closed_forms(m):
    # Eq. 40: <1> = 1.  Eq. 39 with Eq. 41: <p0> = mbar K2/K1; the rest-frame
    # pressure (Eq. 8, 29) gives <p_x^2> = n T = mbar K2/K1 as well.
    k21 = S.kv_dec(2, m) / S.kv_dec(1, m)
    md = S._dec(m)
    assert abs(S.rest_moment_dec("1", m) - 1) < Decimal("1e-45")
    assert abs(S.rest_moment_dec("p0", m) - md * k21) < Decimal("1e-44")
    assert abs(S.rest_moment_dec("px2", m) - md * k21) < Decimal("1e-44")


@pytest.mark.parametrize("m", [0.36, 1.0, 5.0])
def test_rest_moments_fourth_order_closed_forms(m):
    # Textbook identity int_0^inf e^{-z cosh t} sinh^{2nu} t dt
    #   = Gamma(nu + 1/2)/sqrt(pi) (2/z)^nu K_nu(z), and d/dz of it for one power
    # of cosh, give (T_R = 1):
    #   <p_x^2 p_y^2> = m^2 K3/K1,  <p_x^4> = 3 m^2 K3/K1,  <p0 p_x^2> = m^2 + 4 m K2/K1.
    md = S._dec(m)
    k1, k2, k3 = (S.kv_dec(n, m) for n in (1, 2, 3))
    tol = Decimal("1e-40")
    assert abs(S.rest_moment_dec("px2py2", m) / (md * md * k3 / k1) - 1) < tol
    assert abs(S.rest_moment_dec("px4", m) / (3 * md * md * k3 / k1) - 1) < tol
    assert abs(S.rest_moment_dec("p0px2", m) / (md * md + 4 * md * k2 / k1) - 1) < tol


def test_bessel_ratio_fp64():
    z = np.array([1e-3, 0.01, 0.36, 1.0, 5.0, 100.0, 700.0])
    r = S.bessel_ratio_k1k2(z)
    ref = np.array([float(S.kv_dec(1, x) / S.kv_dec(2, x)) for x in z])
    assert np.max(np.abs(r / ref - 1)) < 1e-14
