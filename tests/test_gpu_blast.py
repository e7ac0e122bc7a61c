"""Near-massless blast on a 1024 x 1024 copy of the 8192 x 8192 workload (disc
of radius 64 at T = 2 in a T = 1 background, n = 1, u = 0, tau = 0.7; the
temperatures in units of their mean, T_R = 1.5, so 4/3 and 2/3).  The
requested m/T = 0.01 has no positive second-order quadrature (Sec. III D), so
the lattice runs at the smallest covered mass, m/T_R = 0.36, on the paper's
133-velocity stencil G1, G14, G49, G51, G60, G70 (Sec. IV).

* BF16-deviation and FP32 storage against the FP64 path after 500 steps;
* FP64 path against the oracle on windows across the disc edge (2 steps);
* equation of state of the read-out, e/(3nT) - 1 = (zeta/3) K1(zeta)/K2(zeta)
  (Eq. 28), against SciPy's Bessel functions, and its distance from the
  massless e = 3nT."""
import numpy as np
import pytest
from scipy import special as sp

from gpu_common import errors, oracle_lattice
from paper_1703_04605_gb300 import workloads as W

pytestmark = pytest.mark.gpu
N, R, TAU, STEPS = 1024, 64, 0.7, 500
ST = W.STENCIL_E5


@pytest.fixture(scope="module")
def fields():
    from paper_1703_04605_gb300 import build
    build.build()
    return W.blast(N, R)


@pytest.fixture(scope="module")
def runs(fields):
    from paper_1703_04605_gb300 import Lattice
    out = {}
    for dtype in ("f64", "f32", "bf16dev"):
        with Lattice(ST["groups"], ST["m"], TAU, N, N, dtype=dtype, v0=ST["v0"]) as lat:
            lat.init(fields["n"], fields["ux"], fields["uy"], fields["T"])
            lat.step(STEPS)
            out[dtype] = lat.moments()
    return out


def test_bf16dev_against_f64(runs):
    eb = errors(runs["bf16dev"], runs["f64"])
    assert max(eb.values()) < 2e-3, eb


def test_f32_against_f64(runs):
    # Not the storage of this workload, and outside what FP32 storage holds to
    # 1e-5: the FP32 path stores deviations from the state (n_ref, T_R), and
    # here both the disc (4/3 T_R) and the background (2/3 T_R) are far from
    # it, so each uniform region rounds the same way at every site and step
    # (measured after 500 steps: n 2.9e-5, T 3.5e-5, u 7.8e-5).
    e32 = errors(runs["f32"], runs["f64"])
    assert e32["n"] < 1e-4 and e32["T"] < 1e-4 and e32["u"] < 2e-4, e32


def test_blast_has_developed(runs):
    m = runs["f64"]
    assert np.abs(m["ux"]).max() > 0.01          # an outgoing wave
    assert m["T"].max() < 4 / 3 and m["T"].min() < 2 / 3


def test_equation_of_state(runs):
    for dtype in ("f64", "bf16dev"):
        m = runs[dtype]
        z = ST["m"] / m["T"]
        ratio = sp.kve(1, z) / sp.kve(2, z)
        dev = m["e"] / (3 * m["n"] * m["T"]) - 1
        assert np.max(np.abs(dev - z * ratio / 3)) < 1e-12, dtype
        # finite mass: e exceeds 3nT by about zeta^2/6 (1-5 % here)
        assert 0.005 < dev.min() and dev.max() < 0.08


def test_f64_against_oracle_across_the_edge(fields):
    from paper_1703_04605_gb300 import Lattice
    with Lattice(ST["groups"], ST["m"], TAU, N, N, dtype="f64", v0=ST["v0"]) as lat:
        lat.init(fields["n"], fields["ux"], fields["uy"], fields["T"])
        lat.step(2)
        got = lat.moments()
        h = lat.info()["halo"]
    r = 2 * h + 1
    c = N // 2
    sites = [(c, c + R), (c + R, c), (c - R, c - 1), (c + 45, c + 45), (c, c), (0, 0)]
    worst = 0.0
    for (y, x) in sites:
        iy = (np.arange(y - r, y + r + 1) % N)[:, None]
        ix = (np.arange(x - r, x + r + 1) % N)[None, :]
        win = {k: v[iy, ix] for k, v in fields.items()}
        o = oracle_lattice(ST, TAU, (2 * r + 1, 2 * r + 1))
        o.init(win["n"], win["ux"], win["uy"], win["T"])
        o.step(2)
        mac = o.macros()
        for k in ("n", "T"):
            worst = max(worst, abs(got[k][y, x] / mac[k][r, r] - 1))
        for k in ("ux", "uy"):
            worst = max(worst, abs(got[k][y, x] - mac[k][r, r]))   # u is O(1e-3) after 2 steps
    assert worst < 1e-12, worst
