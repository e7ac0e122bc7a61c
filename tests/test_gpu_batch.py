"""rlbm_batch_step: many independent lattices of different stencils, sizes,
masses and relaxation times (second and third order) advanced together must
give what each lattice gives when advanced alone (the graph nodes run the single-lattice kernel, so
the results are identical), and what the oracle gives."""
import numpy as np
import pytest

from gpu_common import errors, run_oracle, smooth_fields
from paper_1703_04605_gb300 import stencils, workloads as W

pytestmark = pytest.mark.gpu

SPECS = [  # (mbar, tau, Nx, Ny)
    (1.0, 0.8, 40, 37), (0.9, 1.1, 64, 64), (2.5, 0.7, 50, 33), (8.0, 0.9, 31, 45),
    (0.45, 0.75, 48, 48), (4.0, 1.4, 100, 20), (0.62, 0.95, 24, 24),
]


def _make(spec, seed, dtype="f32", order=2):
    from paper_1703_04605_gb300 import Lattice
    m, tau, Nx, Ny = spec
    groups, mu = stencils.choose(m, order=order)
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
    batch_step(batch, 20)        # too few steps to tune: graphs of 8 and 2 steps
    batch_step(batch, 5)         # graph of 2 steps and one single step (parity flips)
    batch_step(batch, 45)        # below the 66 tuning steps: graphs of 8 and 2, one single step
    for lat in alone:
        lat.step(70)
    for b, a in zip(batch, alone):
        assert b.info()["t"] == 70
        mb, ma = b.moments(), a.moments()
        e = errors(mb, ma)
        assert max(e.values()) < 1e-12, e
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


def test_batch_bf16_equals_single_lattices():
    from paper_1703_04605_gb300 import batch_step
    specs = [(1.0, 0.8, 40, 37), (5.0, 0.9, 31, 45), (0.4, 0.75, 48, 48), (2.5, 0.7, 50, 33)]
    batch = [_make(s, 200 + i, dtype="bf16dev") for i, s in enumerate(specs)]
    alone = [_make(s, 200 + i, dtype="bf16dev") for i, s in enumerate(specs)]
    batch_step(batch, 9)
    for lat in alone:
        lat.step(9)
    for b, a in zip(batch, alone):
        e = errors(b.moments(), a.moments())
        assert max(e.values()) < 1e-12, e      # same kernel, same inputs: identical
    for lat in batch + alone:
        lat.close()


def test_batch_third_order_equals_single_lattices():
    # compiled third-order kernels of five library sets (halo 3-5) beside a
    # second-order lattice, in one graph: identical to stepping each alone
    from paper_1703_04605_gb300 import batch_step
    specs = [(2.0, 0.8, 33, 29, 3), (2.5, 1.1, 40, 21, 3), (5.0, 0.9, 27, 36, 3), (6.0, 0.7, 24, 24, 3),
             (8.0, 1.3, 45, 18, 3), (1.0, 0.8, 40, 37, 2)]
    batch = [_make(s[:4], 300 + i, order=s[4]) for i, s in enumerate(specs)]
    alone = [_make(s[:4], 300 + i, order=s[4]) for i, s in enumerate(specs)]
    assert [b.info()["kernel"] for b in batch[:5]] == [8, 9, 5, 6, 7]
    batch_step(batch, 9)         # graph of 8 steps and one single step
    batch_step(batch, 45)        # below the 66 tuning steps: graphs of 8 and 2, one single step
    for lat in alone:
        lat.step(54)
    for b, a in zip(batch, alone):
        assert b.info()["t"] == 54
        e = errors(b.moments(), a.moments())
        assert max(e.values()) < 1e-12, e      # same kernel, same inputs: identical
    for lat in batch + alone:
        lat.close()


def test_batch_rejections():
    from paper_1703_04605_gb300 import RLBMError, batch_step
    a = _make(SPECS[0], 1)
    b = _make(SPECS[0], 2, dtype="f64")
    with pytest.raises(RLBMError):
        batch_step([a, b], 2)
    with pytest.raises(RLBMError):
        batch_step([a, a], 2)
    # third order: FP64 storage, or FP32 on the generic kernel (narrower than the halo)
    c = _make((5.0, 0.8, 16, 16), 3, dtype="f64", order=3)
    d = _make((5.0, 0.8, 2, 16), 4, order=3)
    assert d.info()["kernel"] == 0
    for other in (c, d):
        with pytest.raises(RLBMError, match="ENOTSUP"):
            batch_step([a, other], 2)
    for lat in (a, b, c, d):
        lat.close()


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
    batch_step(batch, 72)        # >= 66: the autotuner times both engines
    from paper_1703_04605_gb300 import batch_engine, batch_tuning
    eng = batch_engine(batch)
    tune = batch_tuning(batch)
    if eng["engine"] == "graph":
        assert eng["param"] in (2, 8, 32) and eng["launches"] == len(batch)
        assert tune["steps_per_graph"] == eng["param"] and tune["launches_per_step"] == len(batch)
    else:
        assert eng["engine"] == "persistent" and eng["param"] in (1, 2, 4) and 1 <= eng["launches"] <= 4
        assert tune["steps_per_graph"] == 0 and tune["launches_per_step"] == 0
    for lat in alone:
        lat.step(72)
    for b, a in zip(batch, alone):
        e = errors(b.moments(), a.moments())
        assert max(e.values()) < 1e-12, e


def test_batch_workload_lattices_against_oracle():
    """16 lattices of the 256-lattice workload (the 8 smallest and 8 drawn at
    random) advanced together: the 8 smallest against the oracle on the whole
    lattice after 2 and 10 steps, the others on periodic windows around
    sampled sites after 2 steps (a site depends only on sites within twice the
    halo)."""
    from gpu_common import oracle_lattice
    from paper_1703_04605_gb300 import Lattice, batch_step
    specs = W.batch_specs(256)
    order = sorted(range(256), key=lambda i: specs[i]["L"])
    small = order[:8]
    rng = np.random.default_rng(77)
    others = [int(i) for i in rng.choice(order[8:], 8, replace=False)]
    chosen = small + others
    lats, fields, sts = [], [], []
    for i in chosen:
        s = specs[i]
        groups, mu = stencils.choose(s["m"])
        f = W.batch_fields(s)
        lat = Lattice(groups, mu, s["tau"], s["L"], s["L"], dtype="f32", v0=0.0)
        lat.init(f["n"], f["ux"], f["uy"], f["T"])
        lats.append(lat)
        fields.append(f)
        sts.append(dict(groups=groups, m=mu, v0=lat.info()["v0"]))
    batch_step(lats, 2)
    for j, i in enumerate(chosen):
        s, f, lat = specs[i], fields[j], lats[j]
        got = lat.moments()
        if i in small:
            o = oracle_lattice(sts[j], s["tau"], f["n"].shape)
            o.init(f["n"], f["ux"], f["uy"], f["T"])
            o.step(2)
            e = errors(got, o.macros())
            assert max(e.values()) < 1e-5, (i, e)
        else:
            h = lat.info()["halo"]
            r = 2 * h + 1
            L = s["L"]
            for (y, x) in [(L // 2, L // 2), (L // 2, L // 2 - 1), tuple(rng.integers(0, L, 2))]:
                iy = (np.arange(y - r, y + r + 1) % L)[:, None]
                ix = (np.arange(x - r, x + r + 1) % L)[None, :]
                win = {k: v[iy, ix] for k, v in f.items()}
                o = oracle_lattice(sts[j], s["tau"], (2 * r + 1, 2 * r + 1))
                o.init(win["n"], win["ux"], win["uy"], win["T"])
                o.step(2)
                mac = o.macros()
                for k in ("n", "T"):
                    assert abs(got[k][y, x] / mac[k][r, r] - 1) < 1e-5, (i, k)
                # the errors() normalisation: the lattice's largest velocity
                scale = max(np.abs(got["ux"]).max(), np.abs(got["uy"]).max(), 1e-3)
                for k in ("ux", "uy"):
                    assert abs(got[k][y, x] - mac[k][r, r]) < 1e-5 * scale, (i, k)
    batch_step(lats, 8)
    for j, i in enumerate(small):
        s, f = specs[i], fields[j]
        o = oracle_lattice(sts[j], s["tau"], f["n"].shape)
        o.init(f["n"], f["ux"], f["uy"], f["T"])
        o.step(10)
        e = errors(lats[j].moments(), o.macros())
        assert max(e.values()) < 1e-5, (i, e)
    for lat in lats:
        lat.close()
