"""The seeded input recipes (the synthetic stand-ins for the paper's initial
states) produce what their description says: shapes, means, spreads,
smoothing width, the parameter ranges of the batch, the disc of the blast,
the jumps of the shock tube and the Taylor-Green mode.  Same seed, same
arrays.  No lattice arithmetic is involved."""
import math

import numpy as np
import pytest

from paper_1703_04605_gb300 import workloads as W


def test_random_flow_recipe():
    N = 512
    f = W.random_flow(N)
    assert all(a.shape == (N, N) for a in f.values())
    for k, mean, std in (("n", 1.0, 0.01), ("T", 1.0, 0.01), ("ux", 0.0, 0.05), ("uy", 0.0, 0.05)):
        assert abs(f[k].mean() - mean) < 1e-12 and abs(f[k].std() / std - 1.0) < 1e-9, k
    # four independent draws
    g = [(f[k] - f[k].mean()) / f[k].std() for k in ("n", "T", "ux", "uy")]
    for i in range(4):
        for j in range(i):
            assert abs(np.mean(g[i] * g[j])) < 0.1
    # Gaussian smoothing of width sigma = 8: autocorrelation exp(-r^2/(4 sigma^2))
    for r, want in ((8, math.exp(-0.25)), (16, math.exp(-1.0)), (32, math.exp(-4.0))):
        c = np.mean([np.mean(x * np.roll(x, r, axis=1)) for x in g] + [np.mean(x * np.roll(x, r, axis=0)) for x in g])
        assert abs(c - want) < 0.05, (r, c, want)
    # periodic: no seam at the wrap
    d_wrap = np.abs(f["n"][:, 0] - f["n"][:, -1]).max()
    d_in = np.abs(np.diff(f["n"], axis=1)).max()
    assert d_wrap <= 1.5 * d_in
    # seeded
    assert np.array_equal(W.random_flow(64)["n"], W.random_flow(64)["n"])
    assert W.seed(2) == 1705


def test_batch_recipe():
    specs = W.batch_specs()
    assert len(specs) == 256
    L = np.array([s["L"] for s in specs])
    assert L.min() >= 64 and L.max() <= 1024
    # log-uniform side: log L uniform on [log 64, log 1024]
    u = (np.log(L) - math.log(64)) / (math.log(1024) - math.log(64))
    assert abs(u.mean() - 0.5) < 0.06 and abs(u.std() - 1 / math.sqrt(12)) < 0.04
    md = np.array([s["m_drawn"] for s in specs])
    assert md.min() >= 0.1 and md.max() <= 10.0
    um = (np.log(md) - math.log(0.1)) / (math.log(10.0) - math.log(0.1))
    assert abs(um.mean() - 0.5) < 0.06
    assert all(s["m"] == max(s["m_drawn"], 0.36) for s in specs)
    tau = np.array([s["tau"] for s in specs])
    assert tau.min() >= 0.6 and tau.max() <= 1.5
    for i, s in enumerate(specs):
        if i % 2 == 0:
            assert s["kind"] == "sod"
            assert all(0.5 <= x <= 1.5 for x in s["n"] + s["T_drawn"])
            tl, tr = s["T"]
            assert abs(0.5 * (tl + tr) - 1.0) < 1e-12 and max(tl, tr) / min(tl, tr) <= 2.0 + 1e-12
        else:
            assert s["kind"] == "tg" and 0.01 <= s["u0"] <= 0.1


def test_blast_recipe():
    N, R = 1024, 64
    f = W.blast(N, R)
    inside = f["T"] > 1.0
    assert abs(inside.sum() / (math.pi * R * R) - 1.0) < 0.01
    assert np.allclose(f["T"][inside], 4.0 / 3.0) and np.allclose(f["T"][~inside], 2.0 / 3.0)
    assert np.all(f["n"] == 1.0) and not f["ux"].any() and not f["uy"].any()
    ys, xs = np.nonzero(inside)
    assert abs(xs.mean() - (N - 1) / 2) < 0.5 and abs(ys.mean() - (N - 1) / 2) < 0.5


def test_sod_recipe():
    f = W.sod()
    n, T = f["n"][0], f["T"][0]
    assert f["n"].shape == (1, 800)
    assert np.all(n[:400] == 1.0) and np.all(n[400:] == 0.5)
    assert np.all(T[:400] == 1.0) and np.all(T[400:] == 0.8)
    assert not f["ux"].any() and not f["uy"].any()


@pytest.mark.parametrize("N", [48, 512])
def test_taylor_green_recipe(N):
    u0 = 0.05
    f = W.taylor_green(N, u0=u0)
    k = 2 * math.pi / N
    for x, y in ((3, 5), (N // 4, N // 3), (N - 1, 0)):
        assert abs(f["ux"][y, x] - u0 * math.sin(k * x) * math.cos(k * y)) < 1e-15
        assert abs(f["uy"][y, x] + u0 * math.cos(k * x) * math.sin(k * y)) < 1e-15
    # a single divergence-free mode: its spectrum has the four wavevectors (+-1, +-1) only
    s = np.abs(np.fft.fft2(f["ux"]))
    assert np.count_nonzero(s > 1e-9 * s.max()) == 4
