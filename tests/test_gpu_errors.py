"""Device-side physicality flags: fields handed to rlbm_init_device are not
checked on the host, so an out-of-range site (n <= 0, |u| >= 1, T <= 0) must
surface as RLBM_ENONPHYS at the next synchronising call, and the flag is
cleared once reported (a valid re-initialisation then steps cleanly).  No
fault is involved: the kernels only set bits in the context's error word."""
import pytest

from paper_1703_04605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1703_04605_gb300 import build
    build.build()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("field,value,bit", [("n", -1.0, "n <= 0"), ("ux", 1.0, "|u| >= 1"), ("T", 0.0, "T <= 0")])
def test_out_of_range_device_fields_report_enonphys(dtype, field, value, bit):
    import torch
    from paper_1703_04605_gb300 import Lattice, RLBMError
    st = W.STENCIL_M1
    Nx, Ny = 16, 12
    ones = torch.ones(Nx * Ny, dtype=torch.float64, device="cuda")
    zeros = torch.zeros_like(ones)
    with Lattice(st["groups"], st["m"], 0.8, Nx, Ny, dtype=dtype, v0=st["v0"]) as lat:
        f = {"n": ones.clone(), "ux": zeros.clone(), "uy": zeros.clone(), "T": ones.clone()}
        f[field][37] = value
        lat.init_device(f["n"], f["ux"], f["uy"], f["T"])
        with pytest.raises(RLBMError, match="ENONPHYS") as ei:
            lat.sync()
        assert bit in str(ei.value)
        # reported once, then cleared
        lat.init_device(ones, zeros, zeros, ones)
        lat.step(3)
        lat.sync()
        out = lat.moments()
        assert abs(float(out["n"].mean()) - 1.0) < 1e-12
