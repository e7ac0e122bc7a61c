"""The paper's demonstrations (Sec. IV-V) on the CUDA path against the oracle,
element by element: small crops of each input recipe (the Riemann problem on
each stencil of the m/T_R sweep, the acoustic pulse, the Taylor-dispersion
disc and the colliding discs), FP64 within 1e-12 and FP32 (plain and
extended moment sums) within 1e-5 of the oracle in n, T and u.  The tubes
are y-invariant and run on eight identical rows, which puts them on the
compiled stencil kernels."""
import numpy as np
import pytest

from gpu_common import errors, run_oracle
from paper_1703_04605_gb300 import stencils, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1703_04605_gb300 import build
    build.build()


def _stencil(m):
    from paper_1703_04605_gb300 import quadrature_window
    groups, mb = stencils.choose(m)
    lo, hi, _ = quadrature_window(groups, mb)
    return dict(groups=groups, m=mb, v0=0.5 * (lo + hi))


def _gpu(st, tau, f, steps, dtype, ext=False):
    from paper_1703_04605_gb300 import Lattice
    Ny, Nx = f["n"].shape
    with Lattice(st["groups"], st["m"], tau, Nx, Ny, dtype=dtype, v0=st["v0"]) as lat:
        if ext:
            lat.set_extended_sums(True)
        lat.init(f["n"], f["ux"], f["uy"], f["T"])
        lat.step(steps)
        out = lat.moments()
        kernel = lat.info()["kernel"]
    return out, kernel


def _check(st, tau, f, steps, u_scale=None):
    ref = run_oracle(st, tau, f, steps)
    res = {}
    for dtype, ext, tol in (("f64", False, 1e-12), ("f32", False, 1e-5), ("f32", True, 1e-5)):
        got, kernel = _gpu(st, tau, f, steps, dtype, ext)
        e = errors(got, ref)
        if u_scale is not None:         # flows that start at rest: u against a stated scale too
            du = max(np.abs(got["ux"] - ref["ux"]).max(), np.abs(got["uy"] - ref["uy"]).max())
            e["u"] = du / max(u_scale, np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
        assert max(e.values()) < tol, (dtype, ext, e)
        if dtype == "f32":
            assert kernel in (1, 2, 3, 4)        # the compiled stencil kernel ran
        res[(dtype, ext)] = e
    return res


@pytest.mark.parametrize("m", W.RIEMANN_SWEEP_M)
def test_riemann_crop_against_oracle(m):
    """Sec. IV-V: the strong Riemann problem (n 1 : 0.124, T 1 : 0.5) on a
    periodic 160-cell tube, 16 steps, at each m/T_R of the sweep."""
    st = _stencil(m)
    f = W.riemann(160, 8)
    _check(st, W.sod_tau(0.1, v0=st["v0"]), f, 16, u_scale=0.05)


def test_sound_pulse_crop_against_oracle():
    """A 5 % density pulse (velocities up to ~3 % of c): the FP64 round-off of
    u stays well below 1e-12 of the flow's velocity scale."""
    st = _stencil(1.0)
    f = W.sound_pulse(128, 8, amp=5e-2, sigma=8.0)
    _check(st, 0.55, f, 20, u_scale=1e-2)


def test_taylor_dispersion_crop_against_oracle():
    """One disc at v = c/2 (density 1 -> 0.1 background), 64^2, 15 steps."""
    st = _stencil(1.0)
    f = W.taylor_dispersion(64, R=12, v=0.5)
    _check(st, W.DISC_TAU, f, 15)


def test_colliding_discs_crop_against_oracle():
    """Two discs at -+c/2, 64^2, 15 steps."""
    st = _stencil(1.0)
    f = W.colliding_discs(64, R=12, v=0.5)
    _check(st, W.DISC_TAU, f, 15)
