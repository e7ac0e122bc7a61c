"""Native 3D lattices (rlbm3_*): the unfolded stencil on Nx x Ny x Nz periodic
lattices against the oracle's 3D lattice (same stencil, same v0), and
properties that hold at any size.

* FP64 parity with the oracle (1e-12) on ragged lattices, three stencils;
* FP32 storage against the oracle: the compiled kernels (1e-5) and the
  generic one;
* Nz = 1 with u_z = 0 equals the folded 2D lattice of the same stencil
  (the fold of the 3D stencil is exact while U^z = 0);
* rotation: a flow along z equals the same flow along x, transposed (the
  stencil's full symmetry);
* global conservation of N^0 and T^{0 nu}; the moments at t = 0 are the
  input fields."""
from decimal import Decimal

import numpy as np
import pytest

from gpu_common import errors
from oracle import lattice as OL
from oracle import quadrature as QD
from paper_1703_04605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1703_04605_gb300 import build
    build.build()


def smooth3(Nx, Ny, Nz, seed, dn=0.1, dT=0.1, du=0.08, modes=3):
    """Periodic smooth random fields on [Nz, Ny, Nx]: a few Fourier modes."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")

    def field():
        f = np.zeros((Nz, Ny, Nx))
        for _ in range(modes):
            k = [rng.integers(0, 3) * 2 * np.pi / N for N in (Nx, Ny, Nz)]
            f += rng.uniform(-1, 1) * np.cos(k[0] * x + k[1] * y + k[2] * z + rng.uniform(0, 2 * np.pi))
        return f / modes

    return dict(n=1 + dn * field(), T=1 + dT * field(), ux=du * field(), uy=du * field(), uz=du * field())


def oracle3(st, tau, fields, steps):
    Nz, Ny, Nx = fields["n"].shape
    s = QD.Stencil(st["groups"], st["m"], st["v0"], w=QD.weights(st["groups"], st["m"], Decimal(st["v0"])))
    lat = OL.Lattice(s, tau, (Nz, Ny, Nx), two_d=False)
    lat.init(fields["n"], fields["ux"], fields["uy"], fields["T"], uz=fields["uz"])
    lat.step(steps)
    return lat.macros()


def gpu3(st, tau, fields, steps, dtype="f64", mask=None):
    from paper_1703_04605_gb300 import Lattice3D
    Nz, Ny, Nx = fields["n"].shape
    with Lattice3D(st["groups"], st["m"], tau, Nx, Ny, Nz, dtype=dtype, v0=st["v0"]) as lat:
        lat.init(fields["n"], fields["ux"], fields["uy"], fields["uz"], fields["T"])
        lat.step(steps)
        out = lat.moments() if mask is None else lat.moments(mask)
        info = lat.info()
    return out, info


def errors3(got, ref):
    e = errors(got, ref)
    umax = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max(), np.abs(ref["uz"]).max())
    e["u"] = max(np.abs(got[k] - ref[k]).max() for k in ("ux", "uy", "uz")) / umax
    return e


@pytest.mark.parametrize("name,shape,steps", [("G16", (7, 8, 9), 4), ("M1", (5, 6, 9), 3), ("E5", (4, 5, 13), 2)])
def test_f64_against_oracle(name, shape, steps):
    st = {"G16": W.STENCIL_G16, "M1": W.STENCIL_M1, "E5": W.STENCIL_E5}[name]
    f = smooth3(shape[2], shape[1], shape[0], seed=31)
    got, info = gpu3(st, 0.8, f, steps)
    assert info["Q"] == {"G16": 57, "M1": 96, "E5": 133}[name]
    ref = oracle3(st, 0.8, f, steps)
    e = errors3(got, ref)
    assert max(e.values()) < 1e-12, e


@pytest.mark.parametrize("name,kernel", [("G16", 2), ("M1", 1), ("E5", 3), ("S2", 4)])
def test_f32_compiled_against_oracle(name, kernel):
    st = {"G16": W.STENCIL_G16, "M1": W.STENCIL_M1, "E5": W.STENCIL_E5, "S2": W.STENCIL_S2}[name]
    f = smooth3(13, 13, 13, seed=32) if name == "E5" else smooth3(11, 9, 8, seed=32)
    got, info = gpu3(st, 0.8, f, 10, dtype="f32")
    assert info["kernel"] == kernel
    assert info["bytes_per_site"] == 2 * info["Q"] * 4
    ref = oracle3(st, 0.8, f, 10)
    e = errors3(got, ref)
    assert max(e.values()) < 1e-5, e


def test_f32_generic_against_oracle():
    # narrower than the M1 halo (4) in x: the generic FP32 kernel
    st = W.STENCIL_M1
    f = smooth3(3, 9, 8, seed=36)
    got, info = gpu3(st, 0.8, f, 10, dtype="f32")
    assert info["kernel"] == 0
    ref = oracle3(st, 0.8, f, 10)
    e = errors3(got, ref)
    # per-population FP32 constants (as the generic 2D FP32 kernel)
    assert e["n"] < 1e-5 and e["T"] < 1e-5 and e["u"] < 1e-4, e


def test_nz1_equals_folded_2d():
    from paper_1703_04605_gb300 import Lattice
    st = W.STENCIL_M1
    f = smooth3(24, 20, 1, seed=33)
    f["uz"] = np.zeros_like(f["uz"])
    got, _ = gpu3(st, 0.9, f, 12)
    with Lattice(st["groups"], st["m"], 0.9, 24, 20, dtype="f64", v0=st["v0"]) as lat:
        lat.init(f["n"][0], f["ux"][0], f["uy"][0], f["T"][0])
        lat.step(12)
        ref2 = lat.moments()
    for k in ("n", "T"):
        assert np.max(np.abs(got[k][0] / ref2[k] - 1)) < 1e-12, k
    for k in ("ux", "uy"):
        assert np.max(np.abs(got[k][0] - ref2[k])) < 1e-13, k
    assert np.max(np.abs(got["uz"])) < 1e-15


def test_rotation_z_equals_x():
    st = W.STENCIL_G16
    N = 8
    f = smooth3(N, N, N, seed=34)
    # the same fields with the roles of x and z exchanged
    g = {k: np.ascontiguousarray(np.transpose(v, (2, 1, 0))) for k, v in f.items()}
    g["ux"], g["uz"] = g["uz"].copy(), g["ux"].copy()
    a, _ = gpu3(st, 0.8, f, 6)
    b, _ = gpu3(st, 0.8, g, 6)
    for k in ("n", "T"):
        assert np.max(np.abs(np.transpose(b[k], (2, 1, 0)) / a[k] - 1)) < 1e-12, k
    assert np.max(np.abs(np.transpose(b["uz"], (2, 1, 0)) - a["ux"])) < 1e-13
    assert np.max(np.abs(np.transpose(b["ux"], (2, 1, 0)) - a["uz"])) < 1e-13


def test_conservation_and_t0():
    from paper_1703_04605_gb300 import _abi as A
    st = W.STENCIL_G16
    f = smooth3(10, 9, 8, seed=35)
    m0, _ = gpu3(st, 0.7, f, 0, mask=A.M_N | A.M_UX | A.M_UY | A.M_UZ | A.M_T | A.M_NVEC | A.M_TMN)
    for k in ("n", "T"):
        assert np.max(np.abs(m0[k] / f[k] - 1)) < 1e-12, k
    for k in ("ux", "uy", "uz"):
        assert np.max(np.abs(m0[k] - f[k])) < 1e-13, k
    m1, _ = gpu3(st, 0.7, f, 7, mask=A.M_NVEC | A.M_TMN)
    scale = abs(m0["T00"].sum())
    for k in ("N0", "T00", "T0x", "T0y", "T0z"):
        assert abs(m1[k].sum() - m0[k].sum()) < 1e-12 * scale, k


# ---------------------------------------------------------------- third order
def test_third_order_f64_against_oracle():
    # eleven groups unfolded (159 populations), the thirty-monomial equilibrium
    st = W.STENCIL_O3
    f = smooth3(7, 6, 5, seed=37, dn=0.05, dT=0.05, du=0.06)
    got, info = gpu3(st, 0.8, f, 3)
    assert info["Q"] == 159 and info["order"] == 3 and info["kernel"] == 0
    ref = oracle3(st, 0.8, f, 3)
    e = errors3(got, ref)
    assert max(e.values()) < 1e-12, e


def test_third_order_f32_against_oracle():
    st = W.STENCIL_O3
    f = smooth3(8, 7, 6, seed=38, dn=0.05, dT=0.05, du=0.06)
    got, info = gpu3(st, 0.8, f, 8, dtype="f32")
    assert info["order"] == 3
    ref = oracle3(st, 0.8, f, 8)
    e = errors3(got, ref)
    # per-population FP32 constants (as the generic FP32 kernels)
    assert e["n"] < 1e-5 and e["T"] < 1e-5 and e["u"] < 1e-4, e


def test_third_order_nz1_equals_folded_2d():
    from paper_1703_04605_gb300 import Lattice
    st = W.STENCIL_O3
    f = smooth3(20, 18, 1, seed=39, dn=0.05, dT=0.05, du=0.06)
    f["uz"] = np.zeros_like(f["uz"])
    got, _ = gpu3(st, 0.9, f, 6)
    with Lattice(st["groups"], st["m"], 0.9, 20, 18, dtype="f64", v0=st["v0"]) as lat:
        lat.init(f["n"][0], f["ux"][0], f["uy"][0], f["T"][0])
        lat.step(6)
        ref2 = lat.moments()
    for k in ("n", "T"):
        assert np.max(np.abs(got[k][0] / ref2[k] - 1)) < 1e-12, k
    for k in ("ux", "uy"):
        assert np.max(np.abs(got[k][0] - ref2[k])) < 1e-13, k
    assert np.max(np.abs(got["uz"])) < 1e-15


def test_third_order_conservation():
    from paper_1703_04605_gb300 import _abi as A
    st = W.STENCIL_O3
    f = smooth3(9, 8, 7, seed=40, dn=0.08, dT=0.08, du=0.06)
    m0, _ = gpu3(st, 0.7, f, 0, mask=A.M_NVEC | A.M_TMN)
    m1, _ = gpu3(st, 0.7, f, 10, mask=A.M_NVEC | A.M_TMN)
    scale = abs(m0["T00"].sum())
    for k in ("N0", "T00", "T0x", "T0y", "T0z"):
        assert abs(m1[k].sum() - m0[k].sum()) < 1e-12 * scale, k
