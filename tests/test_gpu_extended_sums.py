"""FP32 storage with extended moment sums (rlbm_set_extended_sums): the same
step (Eq. 49) as the plain FP32 kernel, with the conserved and kinetic
moments (Eq. 4-5, 18) accumulated to about 2^-40 relative.  Checked against
the oracle on every compiled stencil, for bit-identical results between a
batch and single lattices, and for the API's refusals."""
import numpy as np
import pytest

from gpu_common import errors, run_oracle, smooth_fields
from paper_1703_04605_gb300 import stencils, workloads as W

pytestmark = pytest.mark.gpu

STENCILS = [W.STENCIL_M1, W.STENCIL_G16, W.STENCIL_E5, W.STENCIL_S2]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1703_04605_gb300 import build
    build.build()


@pytest.mark.parametrize("st", STENCILS, ids=["M1", "G16", "E5", "S2"])
def test_extended_sums_match_oracle(st):
    """Ragged lattice (not a multiple of the 128-thread block or the 32-wide
    row pitch), strong flow: after 12 steps within the FP32 bound of the
    oracle, and closer to it than plain FP32 sums in n and T."""
    from paper_1703_04605_gb300 import Lattice
    Nx, Ny, tau, steps = 45, 29, 0.7, 12
    f = smooth_fields(Nx, Ny, seed=61, dn=0.3, dT=0.2, du=0.15)
    ref = run_oracle(st, tau, f, steps)
    got = {}
    for level in (0, 1, 2):
        with Lattice(st["groups"], st["m"], tau, Nx, Ny, dtype="f32", v0=st["v0"]) as lat:
            lat.set_extended_sums(level)
            assert lat.info()["extended_sums"] == level
            assert lat.info()["kernel"] in (1, 2, 3, 4)
            lat.init(f["n"], f["ux"], f["uy"], f["T"])
            lat.step(steps)
            got[level] = errors(lat.moments(), ref)
    for level in (1, 2):
        e = got[level]
        assert max(e.values()) < 1e-5, (level, e)
        assert max(e["n"], e["T"]) <= 1.5 * max(got[0]["n"], got[0]["T"]), (level, got)


def test_extended_sums_batch_equals_single():
    """A batch mixing lattices with and without extended sums gives what each
    lattice gives alone (the graph nodes run each context's own kernel)."""
    from paper_1703_04605_gb300 import Lattice, batch_step
    specs = [(1.0, 0.8, 40, 37, True), (5.0, 0.9, 31, 45, True), (0.4, 0.75, 48, 48, False),
             (2.5, 0.7, 50, 33, True), (3.0, 1.2, 36, 36, False)]

    def make(i, s):
        m, tau, Nx, Ny, ext = s
        groups, mu = stencils.choose(m)
        lat = Lattice(groups, mu, tau, Nx, Ny, dtype="f32", v0=0.0)
        lat.set_extended_sums(ext)
        f = smooth_fields(Nx, Ny, seed=300 + i, du=0.08)
        lat.init(f["n"], f["ux"], f["uy"], f["T"])
        return lat

    batch = [make(i, s) for i, s in enumerate(specs)]
    alone = [make(i, s) for i, s in enumerate(specs)]
    batch_step(batch, 21)
    for lat in alone:
        lat.step(21)
    for b, a in zip(batch, alone):
        e = errors(b.moments(), a.moments())
        assert max(e.values()) < 1e-12, e
    # switching a member's variant drops the cached graph: still identical
    batch[1].set_extended_sums(False)
    alone[1].set_extended_sums(False)
    batch_step(batch, 4)
    for lat in alone:
        lat.step(4)
    for b, a in zip(batch, alone):
        e = errors(b.moments(), a.moments())
        assert max(e.values()) < 1e-12, e
    for lat in batch + alone:
        lat.close()


def test_extended_sums_refused_where_no_compiled_fp32_kernel():
    from paper_1703_04605_gb300 import Lattice, _abi as A
    st = W.STENCIL_M1
    for dtype in ("f64", "bf16dev"):
        with Lattice(st["groups"], st["m"], 0.8, 16, 16, dtype=dtype, v0=st["v0"]) as lat:
            with pytest.raises(A.RLBMError) as ei:
                lat.set_extended_sums(True)
            assert ei.value.status == A.RLBM_ENOTSUP
    with Lattice(st["groups"], st["m"], 0.8, 16, 16, dtype="f32", v0=st["v0"]) as lat:
        with pytest.raises(A.RLBMError) as ei:
            lat.set_extended_sums(3)
        assert ei.value.status == A.RLBM_EINVAL
    o3 = W.STENCIL_O3
    with Lattice(o3["groups"], o3["m"], 0.8, 16, 16, dtype="f32", v0=o3["v0"]) as lat:
        with pytest.raises(A.RLBMError) as ei:
            lat.set_extended_sums(True)
        assert ei.value.status == A.RLBM_ENOTSUP
