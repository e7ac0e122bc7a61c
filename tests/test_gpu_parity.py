"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances: FP64 storage 1e-12, FP32 storage 1e-5 (relative for n
and T; max |du| / max |u| for the velocity)."""
import numpy as np
import pytest

from gpu_common import errors, run_gpu, run_oracle, smooth_fields
from paper_1703_04605_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STENCILS = {"M1": W.STENCIL_M1, "G16": W.STENCIL_G16, "E5": W.STENCIL_E5, "S2": W.STENCIL_S2}
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16dev": 2e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1703_04605_gb300 import build
    build.build()


@pytest.mark.parametrize("name", ["M1", "G16", "E5", "S2"])
def test_f64_small_ragged(name):
    # 37 x 29 = 1073 sites: nine blocks of 128 sites and a ragged tail;
    # Q = 58, 39, 73 exercise three population buckets.
    st = STENCILS[name]
    f = smooth_fields(37, 29, seed=11)
    got, info = run_gpu(st, 0.8, f, "f64", 20)
    ref = run_oracle(st, 0.8, f, 20)
    assert info["t"] == 20
    e = errors(got, ref)
    assert max(e.values()) < TOL["f64"], e


def test_f64_moments_at_t0_roundtrip():
    st = W.STENCIL_M1
    f = smooth_fields(19, 23, seed=5, du=0.3)
    got, _ = run_gpu(st, 0.8, f, "f64", 0)
    assert np.max(np.abs(got["n"] / f["n"] - 1)) < 1e-13
    assert np.max(np.abs(got["T"] / f["T"] - 1)) < 1e-13
    assert np.max(np.abs(got["ux"] - f["ux"])) < 1e-13
    assert np.max(np.abs(got["uy"] - f["uy"])) < 1e-13


def test_f64_full_moment_planes():
    from paper_1703_04605_gb300 import Lattice, _abi as A
    from gpu_common import oracle_lattice
    st = W.STENCIL_G16
    f = smooth_fields(16, 12, seed=3)
    with Lattice(st["groups"], st["m"], 0.9, 16, 12, dtype="f64", v0=st["v0"]) as lat:
        lat.init(f["n"], f["ux"], f["uy"], f["T"])
        lat.step(3)
        got = lat.moments(A.M_NVEC | A.M_TMN | A.M_E)
    o = oracle_lattice(st, 0.9, (12, 16))
    o.init(f["n"], f["ux"], f["uy"], f["T"])
    o.step(3)
    mac = o.macros()
    N, Tm = mac["N"], mac["Tmn"]
    names = {"N0": N[..., 0], "Nx": N[..., 1], "Ny": N[..., 2], "T00": Tm[..., 0, 0], "T0x": Tm[..., 0, 1],
             "T0y": Tm[..., 0, 2], "Txx": Tm[..., 1, 1], "Txy": Tm[..., 1, 2], "Tyy": Tm[..., 2, 2], "e": mac["e"]}
    for k, ref in names.items():
        assert np.max(np.abs(got[k] - ref)) < 1e-12 * np.max(np.abs(Tm[..., 0, 0])), k


def test_f64_sod_full_config():
    # 800 x 1 shock tube, 500 steps, tau for eta/s = 0.1 (the small workload
    # the oracle runs at full size).
    st = W.STENCIL_M1
    f = W.sod(800, 1)
    tau = W.sod_tau()
    got, _ = run_gpu(st, tau, f, "f64", 500)
    ref = run_oracle(st, tau, f, 500)
    e = errors(got, ref)
    assert max(e.values()) < TOL["f64"], e
    assert np.max(np.abs(got["uy"])) < 1e-14


@pytest.mark.parametrize("shape", [(1, 1), (1, 50), (50, 1), (3, 200)])
def test_f64_degenerate_shapes(shape):
    # lattices smaller than the stencil: every displacement wraps several times
    Ny, Nx = shape
    st = W.STENCIL_M1
    f = smooth_fields(Nx, Ny, seed=2)
    got, _ = run_gpu(st, 0.7, f, "f64", 12)
    ref = run_oracle(st, 0.7, f, 12)
    e = errors(got, ref)
    assert e["n"] < 1e-12 and e["T"] < 1e-12
    umax = max(np.max(np.abs(ref["ux"])), np.max(np.abs(ref["uy"])))
    assert np.max(np.abs(got["ux"] - ref["ux"])) < 1e-12 * max(umax, 1.0)


@pytest.mark.parametrize("name", ["M1", "G16", "E5", "S2"])
def test_f32_small_ragged(name):
    st = STENCILS[name]
    f = smooth_fields(45, 31, seed=17)
    got, info = run_gpu(st, 0.8, f, "f32", 50)
    assert info["kernel"] == {"M1": 1, "G16": 2, "E5": 3, "S2": 4}[name]
    ref = run_oracle(st, 0.8, f, 50)
    e = errors(got, ref)
    assert max(e.values()) < TOL["f32"], e


def test_f32_taylor_green_crop():
    # 64 x 64 Taylor-Green at u0 = 0.05, 200 steps, FP32 vs the FP64 oracle
    st = W.STENCIL_M1
    f = W.taylor_green(64, u0=0.05)
    got, _ = run_gpu(st, 0.9, f, "f32", 200)
    ref = run_oracle(st, 0.9, f, 200)
    e = errors(got, ref)
    assert max(e.values()) < TOL["f32"], e


def test_uniform_state_stationary_f32():
    st = W.STENCIL_M1
    f = dict(n=np.full((9, 40), 0.7), T=np.full((9, 40), 1.3), ux=np.full((9, 40), 0.2),
             uy=np.full((9, 40), -0.1))
    got, _ = run_gpu(st, 0.9, f, "f32", 30)
    assert np.max(np.abs(got["n"] / 0.7 - 1)) < 3e-6
    assert np.max(np.abs(got["T"] / 1.3 - 1)) < 3e-6
    assert np.max(np.abs(got["ux"] - 0.2)) < 1e-6


def test_f32_generic_kernel_tiny_lattice():
    # lattices narrower than the stencil halo use the generic kernel
    st = W.STENCIL_M1
    f = smooth_fields(3, 40, seed=4)
    got, info = run_gpu(st, 0.8, f, "f32", 20)
    assert info["kernel"] == 0
    ref = run_oracle(st, 0.8, f, 20)
    e = errors(got, ref)
    assert max(e.values()) < TOL["f32"], e


@pytest.mark.parametrize("name", ["M1", "G16", "E5", "S2"])
def test_bf16dev_small_ragged(name):
    st = STENCILS[name]
    f = smooth_fields(45, 31, seed=19)
    got, info = run_gpu(st, 0.8, f, "bf16dev", 50)
    assert info["kernel"] == {"M1": 1, "G16": 2, "E5": 3, "S2": 4}[name]
    assert info["bytes_per_site"] == 2 * info["Q"] * 2
    ref = run_oracle(st, 0.8, f, 50)
    e = errors(got, ref)
    assert max(e.values()) < TOL["bf16dev"], e


def test_bf16dev_moments_at_t0():
    # the stored deviations decode back to the equilibrium of the fields
    st = W.STENCIL_M1
    f = smooth_fields(24, 20, seed=6, du=0.3, dT=0.5)
    got, _ = run_gpu(st, 0.8, f, "bf16dev", 0)
    assert np.max(np.abs(got["n"] / f["n"] - 1)) < 1e-3
    assert np.max(np.abs(got["T"] / f["T"] - 1)) < 1e-3
    assert np.max(np.abs(got["ux"] - f["ux"])) < 1e-3


def test_bf16dev_blast_crop():
    # the near-massless blast (disc at T = 2 in T = 1) on the E5 stencil,
    # 64 x 64 with a radius-8 disc, 60 steps, against the FP64 oracle
    st = W.STENCIL_E5
    f = W.blast(64, 8)
    got, _ = run_gpu(st, 0.7, f, "bf16dev", 60)
    ref = run_oracle(st, 0.7, f, 60)
    e = errors(got, ref)
    assert max(e.values()) < TOL["bf16dev"], e


def test_bf16dev_unsupported_stencil_is_an_error():
    from paper_1703_04605_gb300 import Lattice, RLBMError
    with pytest.raises(RLBMError):
        Lattice([1, 2, 25, 29, 32, 57], 1.0, 0.8, 32, 32, dtype="bf16dev", v0=0.164844)
