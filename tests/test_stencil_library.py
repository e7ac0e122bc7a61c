"""Coverage of the stencil library: every mbar in [0.36, 10] maps to a compiled
group set that has a positive-weight v0 window there (Sec. III D)."""
import numpy as np
import pytest

A = pytest.importorskip("paper_1703_04605_gb300._abi")
from paper_1703_04605_gb300 import stencils


@pytest.fixture(scope="module")
def lib():
    from paper_1703_04605_gb300 import build
    build.build()
    return A.load()


def test_every_mass_has_a_window(lib):
    for m in np.exp(np.linspace(np.log(0.3), np.log(12.0), 60)):
        groups, mu = stencils.choose(m)
        lo, hi, n = A.quadrature_window(groups, mu)
        assert n >= 1 and hi > lo, (m, groups)
        w = A.quadrature_weights(groups, mu, 0.5 * (lo + hi))
        assert min(w) > 0, (m, groups, w)


def test_clamps():
    assert stencils.choose(0.1)[1] == 0.36
    assert stencils.choose(0.60)[1] == 0.58
    assert stencils.choose(0.63)[1] == 0.65
    assert stencils.choose(5.0)[0] == list(stencils.S2)


def test_third_order_every_mass_has_a_window(lib):
    # eleven-group stencils over [1.875, 14]: every chosen set is positive
    for m in np.exp(np.linspace(np.log(1.6), np.log(15.0), 24)):
        groups, mu = stencils.choose(m, order=3)
        assert len(groups) == 11
        lo, hi, n = A.quadrature_window(groups, mu)
        assert n >= 1 and hi > lo, (m, groups)
        w = A.quadrature_weights(groups, mu, 0.5 * (lo + hi))
        assert min(w) > 0, (m, groups, w)


def test_third_order_choices():
    assert stencils.choose(1.0, order=3)[1] == 1.875
    assert stencils.choose(5.0, order=3)[0] == list(stencils.O3_M5)
    assert stencils.choose(5.2, order=3)[0] == list(stencils.O3_D)
    assert stencils.choose(20.0, order=3)[0] == list(stencils.O3_E)
    with pytest.raises(ValueError):
        stencils.choose(1.0, order=4)
