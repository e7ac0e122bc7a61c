"""rlbm_batch_step: many independent lattices of different stencils, sizes,
masses and relaxation times advanced together must give what each lattice
gives when advanced alone (same arithmetic; the batched and single-lattice
kernels are separate compilations of the same site update)."""
import numpy as np
import pytest

from gpu_common import errors, run_oracle, smooth_fields
from paper_1703_04605_gb300 import stencils, workloads as W

pytestmark = pytest.mark.gpu

SPECS = [  # (mbar, tau, Nx, Ny)
    (1.0, 0.8, 40, 37), (0.9, 1.1, 64, 64), (2.5, 0.7, 50, 33), (8.0, 0.9, 31, 45),
    (0.45, 0.75, 48, 48), (4.0, 1.4, 100, 20), (0.62, 0.95, 24, 24),
]


def _make(spec, seed, dtype="f32"):
    from paper_1703_04605_gb300 import Lattice
    m, tau, Nx, Ny = spec
    groups, mu = stencils.choose(m)
    lat = Lattice(groups, mu, tau, Nx, Ny, dtype=dtype, v0=0.0)
    f = smooth_fields(Nx, Ny, seed=seed, du=0.08)
    lat.init(f["n"], f["ux"], f["uy"], f["T"])
    return lat


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1703_04605_gb300 import build
    build.build()


def test_batch_equals_single_lattices():
    from paper_1703_04605_gb300 import batch_step
    batch = [_make(s, 100 + i) for i, s in enumerate(SPECS)]
    alone = [_make(s, 100 + i) for i, s in enumerate(SPECS)]
    assert sorted({b.info()["kernel"] for b in batch}) == [1, 2, 3, 4]
    batch_step(batch, 20)        # first call: autotune, graph, odd remainder handling
    batch_step(batch, 5)         # cached choice, one graph pair and one single step
    for lat in alone:
        lat.step(25)
    for b, a in zip(batch, alone):
        assert b.info()["t"] == 25
        mb, ma = b.moments(), a.moments()
        e = errors(mb, ma)
        assert max(e.values()) < 2e-6, e
    for lat in batch + alone:
        lat.close()


def test_batch_matches_oracle():
    from paper_1703_04605_gb300 import batch_step
    st = W.STENCIL_M1
    from paper_1703_04605_gb300 import Lattice
    f = smooth_fields(36, 28, seed=9)
    lat = Lattice(st["groups"], st["m"], 0.8, 36, 28, dtype="f32", v0=st["v0"])
    other = Lattice(st["groups"], st["m"], 0.8, 20, 20, dtype="f32", v0=st["v0"])
    lat.init(f["n"], f["ux"], f["uy"], f["T"])
    g = smooth_fields(20, 20, seed=10)
    other.init(g["n"], g["ux"], g["uy"], g["T"])
    batch_step([lat, other], 30)
    ref = run_oracle(st, 0.8, f, 30)
    e = errors(lat.moments(), ref)
    assert max(e.values()) < 1e-5, e


def test_batch_rejections():
    from paper_1703_04605_gb300 import RLBMError, batch_step
    a = _make(SPECS[0], 1)
    b = _make(SPECS[0], 2, dtype="f64")
    with pytest.raises(RLBMError):
        batch_step([a, b], 2)
    with pytest.raises(RLBMError):
        batch_step([a, a], 2)
    a.close()
    b.close()


def test_batch_workload_sample():
    # 12 lattices of the batch workload generator (sides 64..256 here)
    from paper_1703_04605_gb300 import Lattice, batch_step
    specs = W.batch_specs(12, Lmin=64, Lmax=256)
    batch, alone = [], []
    for s in specs:
        groups, mu = stencils.choose(s["m"])
        f = W.batch_fields(s)
        for group in (batch, alone):
            lat = Lattice(groups, mu, s["tau"], s["L"], s["L"], dtype="f32", v0=0.0)
            lat.init(f["n"], f["ux"], f["uy"], f["T"])
            group.append(lat)
    batch_step(batch, 40)
    from paper_1703_04605_gb300 import batch_tuning
    tune = batch_tuning(batch)
    assert tune["minb"] in (4, 5) and tune["per_launch"] in (8, 16, 30)
    kinds = {}
    for lat in batch:
        kinds[lat.info()["kernel"]] = kinds.get(lat.info()["kernel"], 0) + 1
    assert tune["launches"] == sum(-(-c // tune["per_launch"]) for c in kinds.values())
    for lat in alone:
        lat.step(40)
    for b, a in zip(batch, alone):
        e = errors(b.moments(), a.moments())
        assert max(e.values()) < 2e-6, e
