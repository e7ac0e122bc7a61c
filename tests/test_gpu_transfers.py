"""Host transfers of the C ABI: rlbm_init checks the uploaded fields on the
device (the first invalid site is named, the lattice is left as it was, the
reference density is the same on every call), and the read-out writes
page-locked memory directly with the same values as the staged copy into
pageable memory."""
import re

import numpy as np
import pytest

from gpu_common import smooth_fields
from paper_1703_04605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1703_04605_gb300 import build
    build.build()


def _fields(Nx, Ny, seed=5):
    f = smooth_fields(Nx, Ny, seed=seed, dn=0.1, dT=0.1, du=0.1)
    return {k: np.array(v, dtype=np.float64, copy=True) for k, v in f.items()}


# (field, bad value); the 2D check covers n > 0, T > 0, |u| < 1, all finite
BAD = [("n", 0.0), ("n", -2.0), ("n", np.nan), ("n", np.inf), ("T", 0.0), ("T", np.nan),
       ("ux", 1.0), ("uy", -1.5), ("ux", np.nan)]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16dev"])
@pytest.mark.parametrize("field,value", BAD)
def test_init_names_the_first_invalid_site(dtype, field, value):
    """Bad values at three sites in different check blocks: EINVAL names the
    smallest index with its (x, y), and the lattice keeps its previous
    state (the populations are written only after the check passed)."""
    from paper_1703_04605_gb300 import Lattice, RLBMError, _abi as A
    st = W.STENCIL_M1
    Nx, Ny = 300, 211                      # 63 300 sites: 248 check blocks of 256
    good = _fields(Nx, Ny)
    with Lattice(st["groups"], st["m"], 0.8, Nx, Ny, dtype=dtype, v0=st["v0"]) as lat:
        lat.init(good["n"], good["ux"], good["uy"], good["T"])
        lat.step(3)
        before = lat.moments()
        bad = {k: v.copy() for k, v in good.items()}
        sites = [51_234, 1_777, 40_001]    # the smallest is not the first one written
        for s in sites:
            bad[field].reshape(-1)[s] = value
        with pytest.raises(RLBMError) as ei:
            lat.init(bad["n"], bad["ux"], bad["uy"], bad["T"])
        assert ei.value.status == A.RLBM_EINVAL
        first = min(sites)
        m = re.search(r"site (\d+) \(x=(\d+), y=(\d+)\)", str(ei.value))
        assert m, str(ei.value)
        assert (int(m.group(1)), int(m.group(2)), int(m.group(3))) == (first, first % Nx, first // Nx)
        after = lat.moments()
        for k in before:
            assert np.array_equal(before[k], after[k]), k
        lat.step(1)                        # still usable
        lat.sync()


def test_init_check_on_a_large_lattice():
    """1024^2 sites (the check's full 1024 blocks, 1024 sites each): the
    smallest of bad sites in the first and last blocks is reported."""
    from paper_1703_04605_gb300 import Lattice, RLBMError
    st = W.STENCIL_G16
    N = 1024
    f = {k: np.full((N, N), v) for k, v in (("n", 1.0), ("ux", 0.0), ("uy", 0.0), ("T", 1.0))}
    f["T"].reshape(-1)[N * N - 1] = -1.0
    f["n"].reshape(-1)[1023] = 0.0
    with Lattice(st["groups"], st["m"], 0.8, N, N, dtype="f32", v0=st["v0"]) as lat:
        with pytest.raises(RLBMError, match=r"site 1023 \(x=1023, y=0\)"):
            lat.init(f["n"], f["ux"], f["uy"], f["T"])
        f["n"].reshape(-1)[1023] = 1.0
        with pytest.raises(RLBMError, match=r"site %d \(x=1023, y=1023\)" % (N * N - 1)):
            lat.init(f["n"], f["ux"], f["uy"], f["T"])


@pytest.mark.parametrize("dtype", ["f32", "bf16dev"])
def test_init_is_repeatable(dtype):
    """The reference density (mean of n, summed per check block in a fixed
    order) and hence the stored state are the same on every call."""
    from paper_1703_04605_gb300 import Lattice
    st = W.STENCIL_S2
    Nx, Ny = 517, 389
    f = _fields(Nx, Ny, seed=9)
    f["n"] *= 0.37                          # mean far from 1: the reference matters
    with Lattice(st["groups"], st["m"], 0.8, Nx, Ny, dtype=dtype, v0=st["v0"]) as lat:
        outs = []
        for _ in range(2):
            lat.init(f["n"], f["ux"], f["uy"], f["T"])
            lat.step(5)
            outs.append(lat.moments())
        for k in outs[0]:
            assert np.array_equal(outs[0][k], outs[1][k]), k


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16dev"])
def test_readout_into_pinned_memory_equals_staged_copy(dtype):
    """Page-locked output is written by the read-out kernel itself, pageable
    output through the context's device buffer: identical values."""
    import torch
    from paper_1703_04605_gb300 import Lattice
    st = W.STENCIL_M1
    Nx, Ny = 133, 97
    f = _fields(Nx, Ny, seed=13)
    mask = 0x7F                             # every 2D field, 19 planes
    with Lattice(st["groups"], st["m"], 0.8, Nx, Ny, dtype=dtype, v0=st["v0"]) as lat:
        lat.init(f["n"], f["ux"], f["uy"], f["T"])
        lat.step(4)
        size = lat.moments_size(mask)
        pinned = torch.empty(size, dtype=torch.float64, pin_memory=True).numpy()
        pageable = np.empty(size, dtype=np.float64)
        a = lat.moments(mask, out=pinned)
        b = lat.moments(mask, out=pageable)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
        assert np.isfinite(pinned).all()


def test_readout_3d_into_pinned_memory_equals_staged_copy():
    import torch
    from paper_1703_04605_gb300 import Lattice3D
    st = W.STENCIL_M1
    N = 24
    f = W.random_flow3d(N)
    with Lattice3D(st["groups"], st["m"], 0.8, N, N, N, dtype="f32", v0=st["v0"]) as lat:
        lat.init(f["n"], f["ux"], f["uy"], f["uz"], f["T"])
        lat.step(3)
        mask = 0x9F
        size = lat.moments_size(mask)
        pinned = torch.empty(size, dtype=torch.float64, pin_memory=True).numpy()
        a = lat.moments(mask, out=pinned)
        b = lat.moments(mask, out=np.empty(size, dtype=np.float64))
        for k in a:
            assert np.array_equal(a[k], b[k]), k


TOL0 = {"f64": 1e-12, "f32": 2e-6, "bf16dev": 2e-3}


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16dev"])
@pytest.mark.parametrize("name", ["STENCIL_M1", "STENCIL_G16", "STENCIL_E5", "STENCIL_S2"])
def test_moments_right_after_init_are_the_fields(dtype, name):
    """The state at t = 0 is f^eq of the input fields: its moments return
    them (the FP32 path reads the freshly written state in place), and
    reading them does not change what the first steps compute."""
    from paper_1703_04605_gb300 import Lattice, batch_step
    st = getattr(W, name)
    Nx, Ny = 75, 61
    f = _fields(Nx, Ny, seed=21)
    with Lattice(st["groups"], st["m"], 0.8, Nx, Ny, dtype=dtype, v0=st["v0"]) as a, \
            Lattice(st["groups"], st["m"], 0.8, Nx, Ny, dtype=dtype, v0=st["v0"]) as b:
        a.init(f["n"], f["ux"], f["uy"], f["T"])
        m0 = a.moments()
        for k in ("n", "T"):
            assert np.max(np.abs(m0[k] / f[k] - 1)) < TOL0[dtype], k
        for k in ("ux", "uy"):
            assert np.max(np.abs(m0[k] - f[k])) < TOL0[dtype], k
        b.init(f["n"], f["ux"], f["uy"], f["T"])
        a.step(3)
        if dtype == "f64":
            b.step(3)                       # batches take compiled FP32 / BF16 lattices only
        else:
            batch_step([b], 3)
        ma, mb = a.moments(), b.moments()
        for k in ma:
            assert np.array_equal(ma[k], mb[k]), k
