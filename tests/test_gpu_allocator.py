"""Caller-supplied device allocator (rlbm_set_allocator): contexts created
while torch's caching allocator is installed take every device buffer from
it (visible in torch.cuda.memory_allocated), give it back on close, and step
exactly as contexts on cudaMalloc do."""
import numpy as np
import pytest

from gpu_common import errors, smooth_fields
from paper_1703_04605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1703_04605_gb300 import build
    build.build()


def _run(dtype, f, steps):
    from paper_1703_04605_gb300 import Lattice
    st = W.STENCIL_M1
    Ny, Nx = f["n"].shape
    lat = Lattice(st["groups"], st["m"], 0.8, Nx, Ny, dtype=dtype, v0=st["v0"])
    lat.init(f["n"], f["ux"], f["uy"], f["T"])
    lat.step(steps)
    return lat


@pytest.mark.parametrize("dtype", ["f32", "bf16dev", "f64"])
def test_torch_caching_allocator_owns_the_buffers(dtype):
    import torch
    from paper_1703_04605_gb300 import use_cuda_malloc, use_torch_allocator
    f = smooth_fields(40, 36, seed=11, du=0.08)
    ref = _run(dtype, f, 6)
    m_ref = ref.moments()
    ref.close()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    use_torch_allocator()
    try:
        lat = _run(dtype, f, 6)
        held = torch.cuda.memory_allocated() - before
        assert held >= lat.info()["device_bytes"] > 0
        m = lat.moments()
        e = errors(m, m_ref)
        assert max(e.values()) == 0.0, e          # same kernels, same inputs
        lat.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
    finally:
        use_cuda_malloc()
    # contexts created afterwards are on cudaMalloc again
    lat = _run(dtype, f, 1)
    assert torch.cuda.memory_allocated() == before
    lat.close()


def test_torch_allocator_for_a_3d_lattice():
    import torch
    from paper_1703_04605_gb300 import Lattice3D, use_cuda_malloc, use_torch_allocator
    st = W.STENCIL_M1
    rng = np.random.default_rng(3)
    n = 1.0 + 0.01 * rng.standard_normal((6, 7, 8))
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    use_torch_allocator()
    try:
        with Lattice3D(st["groups"], st["m"], 0.8, 8, 7, 6, dtype="f32", v0=st["v0"]) as lat:
            assert torch.cuda.memory_allocated() - before >= lat.info()["device_bytes"] > 0
            lat.init(n, 0.0, 0.0, 0.0, 1.0)
            lat.step(3)
            out = lat.moments()
            assert np.all(np.isfinite(out["n"]))
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
    finally:
        use_cuda_malloc()
