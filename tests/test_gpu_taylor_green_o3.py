"""Shear viscosity of the third-order scheme on the GPU: Taylor-Green decay
on 256^2 at m/T_R = 5 (u0 = 0.02, k = 2 pi/256), FP64.

* the fitted kinetic-energy decay rate equals 2 lambda with
  lambda = (tau - 1/2) k^2 (C4 - C22)/(e + P), the lattice Chapman-Enskog
  coefficient of the scheme's own equilibrium (computed from the oracle's),
  for the third-order stencil at tau = 0.6, 0.9, 1.2 and for a second-order
  one (G1-G6) at tau = 0.9, and scales as tau - 1/2;
* against the Anderson-Witting value (Chapman-Enskog, (2/15) <|p|^4/E^2>),
  the third-order decay is within 3 %, the second-order one more than 8 %
  slow (Sec. IV: second order does not recover the viscosity moments)."""
import math

import numpy as np
import pytest

from test_oracle_third_order import _continuum_shear, _lattice_shear
from oracle import quadrature as QD
from paper_1703_04605_gb300 import workloads as W

pytestmark = pytest.mark.gpu
N = 256
STEPS = 2000
EVERY = 200
K = 2 * math.pi / N
G16 = dict(groups=[1, 2, 3, 4, 5, 6], m=5.0, v0=0.398)


def _rate(st, tau):
    from paper_1703_04605_gb300 import Lattice
    f = W.taylor_green(N, u0=0.02)
    with Lattice(st["groups"], st["m"], tau, N, N, dtype="f64", v0=st["v0"]) as lat:
        lat.init(f["n"], f["ux"], f["uy"], f["T"])
        ts, E = [], []
        for t in range(0, STEPS + 1, EVERY):
            if t:
                lat.step(EVERY)
            if t >= 200:
                m = lat.moments()
                ts.append(t)
                E.append(0.5 * np.sum(m["ux"] ** 2 + m["uy"] ** 2))
    return -np.polyfit(np.array(ts), np.log(np.array(E)), 1)[0]


@pytest.fixture(scope="module")
def coefs():
    from paper_1703_04605_gb300 import build
    build.build()
    o3 = W.STENCIL_O3
    s3 = QD.Stencil(o3["groups"], o3["m"], o3["v0"])
    s2 = QD.Stencil(G16["groups"], G16["m"], G16["v0"])
    return dict(o3=_lattice_shear(s3), g16=_lattice_shear(s2), cont=_continuum_shear(5.0))


def test_third_order_decay(coefs):
    st = W.STENCIL_O3
    rates = {tau: _rate(st, tau) for tau in (0.6, 0.9, 1.2)}
    for tau, r in rates.items():
        lam = (tau - 0.5) * K * K * coefs["o3"]
        assert abs(r / (2 * lam) - 1) < 0.03, (tau, r, 2 * lam)
        lam_cont = (tau - 0.5) * K * K * coefs["cont"] / st["v0"] ** 2
        assert abs(r / (2 * lam_cont) - 1) < 0.03, (tau, r, 2 * lam_cont)
    for tau in (0.9, 1.2):
        assert abs((rates[tau] / rates[0.6]) / ((tau - 0.5) / 0.1) - 1) < 0.02, rates


def test_second_order_decay_is_slower_than_kinetic(coefs):
    r = _rate(G16, 0.9)
    lam = 0.4 * K * K * coefs["g16"]
    assert abs(r / (2 * lam) - 1) < 0.03, (r, 2 * lam)
    lam_cont = 0.4 * K * K * coefs["cont"] / G16["v0"] ** 2
    assert r / (2 * lam_cont) - 1 < -0.08, (r, 2 * lam_cont)
