"""The persistent batch engine (rlbm_batch_step): one cooperative launch per
stencil and storage variant covers all steps; its blocks wait, with a bounded
poll, for the previous step of a tile's lattice.  It must give bit for bit
what each lattice gives alone, at any sites-per-thread, for every variant;
a wait that cannot be met must end the launch and surface as RLBM_ETIMEOUT
on the lattices' next synchronising call, leaving the contexts usable."""
import pytest

from gpu_common import errors, smooth_fields
from paper_1703_04605_gb300 import stencils

pytestmark = pytest.mark.gpu

SPECS = [  # (mbar, tau, Nx, Ny, storage, extended-sum level)
    (1.0, 0.8, 40, 37, "f32", 0), (0.9, 1.1, 64, 64, "f32", 1), (2.5, 0.7, 50, 33, "f32", 0),
    (8.0, 0.9, 31, 45, "f32", 2), (0.45, 0.75, 48, 48, "f32", 0), (4.0, 1.4, 100, 20, "bf16dev", 0),
    (0.62, 0.95, 24, 24, "f32", 1), (6.0, 0.8, 130, 7, "f32", 0),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1703_04605_gb300 import build
    build.build()


@pytest.fixture(autouse=True)
def _default_options():
    from paper_1703_04605_gb300 import set_batch_options
    set_batch_options("auto")
    yield
    set_batch_options("auto")


def _make(spec, seed):
    from paper_1703_04605_gb300 import Lattice
    m, tau, Nx, Ny, dtype, ext = spec
    groups, mu = stencils.choose(m)
    lat = Lattice(groups, mu, tau, Nx, Ny, dtype=dtype, v0=0.0)
    if ext:
        lat.set_extended_sums(ext)
    f = smooth_fields(Nx, Ny, seed=seed, du=0.08)
    lat.init(f["n"], f["ux"], f["uy"], f["T"])
    return lat


def _same(batch, alone):
    for b, a in zip(batch, alone):
        assert b.info()["t"] == a.info()["t"]
        e = errors(b.moments(), a.moments())
        assert max(e.values()) < 1e-12, e


def test_persistent_engine_equals_single_lattices():
    from paper_1703_04605_gb300 import batch_engine, batch_step, set_batch_options
    set_batch_options("persistent")
    batch = [_make(s, 400 + i) for i, s in enumerate(SPECS)]
    alone = [_make(s, 400 + i) for i, s in enumerate(SPECS)]
    assert sorted({b.info()["kernel"] for b in batch}) == [1, 2, 3, 4]
    batch_step(batch, 13)              # odd: parities flip
    batch_step(batch, 6)
    for lat in alone:
        lat.step(19)
    _same(batch, alone)
    eng = batch_engine(batch)
    assert eng["engine"] == "persistent" and eng["param"] >= 1 and eng["launches"] >= 4
    for lat in batch + alone:
        lat.close()


def test_autotuner_tries_both_engines_and_results_do_not_depend_on_the_choice():
    from paper_1703_04605_gb300 import batch_engine, batch_step
    batch = [_make(s, 500 + i) for i, s in enumerate(SPECS)]
    alone = [_make(s, 500 + i) for i, s in enumerate(SPECS)]
    batch_step(batch, 71)              # 42 graph + 24 persistent tuning steps, then the winner
    for lat in alone:
        lat.step(71)
    _same(batch, alone)
    eng = batch_engine(batch)
    assert eng["engine"] in ("graph", "persistent")
    for lat in batch + alone:
        lat.close()


def test_unmeetable_wait_times_out_and_contexts_stay_usable():
    from paper_1703_04605_gb300 import RLBMError, _abi as A, batch_step, set_batch_options
    batch = [_make(s, 600 + i) for i, s in enumerate(SPECS[:3])]
    # every wait target is one unit beyond reach: each block gives up after
    # 2000 polls, the launch ends and the lattices report the timeout
    set_batch_options("persistent", spin_limit=2000, wait_offset=1)
    batch_step(batch, 4)
    for lat in batch:
        with pytest.raises(RLBMError) as ei:
            lat.sync()
        assert ei.value.status == A.RLBM_ETIMEOUT
        lat.sync()                     # the error word was cleared: no further error
    # the contexts still work: re-initialise and run on the default engine
    set_batch_options("auto")
    alone = [_make(s, 600 + i) for i, s in enumerate(SPECS[:3])]
    for i, (lat, s) in enumerate(zip(batch, SPECS[:3])):
        f = smooth_fields(s[2], s[3], seed=600 + i, du=0.08)
        lat.init(f["n"], f["ux"], f["uy"], f["T"])
    batch_step(batch, 5)
    for lat in alone:
        lat.step(5)
    _same(batch, alone)
    for lat in batch + alone:
        lat.close()
