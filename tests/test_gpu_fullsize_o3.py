"""Full-size checks of the third-order workload (4096^2 random flow at
m/T_R = 5, the stencil G1,G2,G5,G6,G7,G9,G10,G11,G12,G13,G15) in the
launch configuration the benchmark times (the compiled FP32 kernel, the
generic FP64 kernel).

* sampled parity: after two steps a site depends only on sites within twice
  the halo (3), so the oracle's third-order lattice advances a periodic
  window of side 4 halo + 3 around each sampled site and its centre must
  match the CUDA path;
* global conservation of N^0 and T^{0 nu} (a property at any size);
* FP32 against the FP64 path after 205 steps (the benchmark's warm-up plus
  timed steps)."""
import numpy as np
import pytest

from gpu_common import errors, oracle_lattice
from paper_1703_04605_gb300 import workloads as W

pytestmark = pytest.mark.gpu
N = 4096
TAU = 0.8
ST = W.STENCIL_O3


@pytest.fixture(scope="module")
def fields():
    from paper_1703_04605_gb300 import build
    build.build()
    return W.random_flow(N)


def _run(fields, dtype, steps, mask=None):
    from paper_1703_04605_gb300 import Lattice, _abi as A
    with Lattice(ST["groups"], ST["m"], TAU, N, N, dtype=dtype, v0=ST["v0"]) as lat:
        lat.init(fields["n"], fields["ux"], fields["uy"], fields["T"])
        lat.step(steps)
        return lat.moments(mask if mask is not None else (A.M_N | A.M_UX | A.M_UY | A.M_T)), lat.info()


@pytest.mark.parametrize("dtype,tol,kernel", [("f32", 1e-5, 5), ("f64", 1e-12, 0)])
def test_sampled_sites_two_steps(fields, dtype, tol, kernel):
    got, info = _run(fields, dtype, 2)
    assert info["kernel"] == kernel and info["order"] == 3
    h = info["halo"]
    r = 2 * h + 1
    side = 2 * r + 1
    rng = np.random.default_rng(43)
    sites = [(0, 0), (N - 1, N - 1), (0, N // 2), (N - 2, 3)] + [tuple(rng.integers(0, N, 2)) for _ in range(6)]
    worst = {"n": 0.0, "T": 0.0, "u": 0.0}
    for (y, x) in sites:
        iy = (np.arange(y - r, y + r + 1) % N)[:, None]
        ix = (np.arange(x - r, x + r + 1) % N)[None, :]
        win = {k: v[iy, ix] for k, v in fields.items()}
        o = oracle_lattice(ST, TAU, (side, side))
        o.init(win["n"], win["ux"], win["uy"], win["T"])
        o.step(2)
        mac = o.macros()
        ref = {k: np.array([[mac[k][r, r]]]) for k in ("n", "T", "ux", "uy")}
        g = {k: np.array([[got[k][y, x]]]) for k in ("n", "T", "ux", "uy")}
        e = errors(g, ref)
        # velocity relative to the workload's velocity scale (0.05)
        e["u"] = max(abs(g["ux"][0, 0] - ref["ux"][0, 0]), abs(g["uy"][0, 0] - ref["uy"][0, 0])) / 0.05
        for k in worst:
            worst[k] = max(worst[k], e[k])
    assert max(worst.values()) < tol, worst


def test_global_conservation_f64(fields):
    from paper_1703_04605_gb300 import _abi as A
    m0, _ = _run(fields, "f64", 0, A.M_NVEC | A.M_TMN)
    m1, _ = _run(fields, "f64", 6, A.M_NVEC | A.M_TMN)
    for k in ("N0", "T00", "T0x", "T0y"):
        a, b = m0[k].sum(), m1[k].sum()
        assert abs(a - b) < 1e-12 * abs(m0["T00"].sum()), k


def test_f32_vs_f64_after_205_steps(fields):
    g32, _ = _run(fields, "f32", 205)
    g64, _ = _run(fields, "f64", 205)
    e = errors(g32, g64)
    assert max(e.values()) < 1e-5, e
