"""rlbm_moments_noalloc: the read-out for callers that may not allocate device
memory (it keeps its scratch in a static device array).  Its result must match
rlbm_moments of a normal context on the same state, and the oracle's macroscopic
fields of that state, within the FP64 parity tolerance, on two calls in a row
(the second call reuses the scratch left by the first).  Collected last on
purpose."""
import ctypes as C

import numpy as np
import pytest

from gpu_common import oracle_lattice, smooth_fields
from paper_1703_04605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_readout_matches_rlbm_moments_twice():
    import torch
    from paper_1703_04605_gb300 import Lattice, build, _abi as A
    build.build()
    L = A.load()
    st = W.STENCIL_M1
    Nx, Ny, tau = 40, 28, 0.8
    mask = A.M_N | A.M_UX | A.M_UY | A.M_T | A.M_E | A.M_TMN
    f = smooth_fields(Nx, Ny, seed=23, du=0.2)
    # the existing entry point: a context advanced by rlbm_step
    refs = []
    with Lattice(st["groups"], st["m"], tau, Nx, Ny, dtype="f64", v0=st["v0"]) as lat:
        lat.init(f["n"], f["ux"], f["uy"], f["T"])
        refs.append(lat.moments(mask))
        lat.step(1)
        refs.append(lat.moments(mask))
    # the same states as plain populations f(., t), t = 0, 1 (library order)
    o = oracle_lattice(st, tau, (Ny, Nx))
    o.init(f["n"], f["ux"], f["uy"], f["T"])
    pops = [o.f.copy()]
    macs = [o.macros()]
    o.step(1)
    pops.append(o.f.copy())
    macs.append(o.macros())
    groups = A.int_array(st["groups"])
    stream = torch.cuda.current_stream()
    size = 11 * Nx * Ny
    for fpop, ref, mac in zip(pops, refs, macs):
        dev = torch.from_numpy(np.ascontiguousarray(fpop)).cuda()
        out = np.full(size, np.nan)
        s = L.rlbm_moments_noalloc(groups, 6, st["m"], st["v0"], Nx, Ny, C.c_void_p(dev.data_ptr()),
                                   out.ctypes.data_as(C.POINTER(C.c_double)), mask,
                                   C.c_void_p(stream.cuda_stream))
        assert s == A.RLBM_OK, L.rlbm_last_error(None)
        names = ["n", "ux", "uy", "T", "e", "T00", "T0x", "T0y", "Txx", "Txy", "Tyy"]
        got = {k: out[i * Nx * Ny:(i + 1) * Nx * Ny].reshape(Ny, Nx) for i, k in enumerate(names)}
        assert np.max(np.abs(got["n"] / ref["n"] - 1)) < 1e-12
        assert np.max(np.abs(got["T"] / ref["T"] - 1)) < 1e-12
        umax = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
        assert np.max(np.abs(got["ux"] - ref["ux"])) < 1e-12 * umax
        assert np.max(np.abs(got["uy"] - ref["uy"])) < 1e-12 * umax
        for k in ("e", "T00", "T0x", "T0y", "Txx", "Txy", "Tyy"):
            assert np.max(np.abs(got[k] - ref[k])) < 1e-12 * np.abs(ref["T00"]).max(), k
        # and the oracle's fields of the same populations
        assert np.max(np.abs(got["n"] / mac["n"] - 1)) < 1e-12
        assert np.max(np.abs(got["T"] / mac["T"] - 1)) < 1e-12
        umax = max(np.abs(mac["ux"]).max(), np.abs(mac["uy"]).max())
        assert np.max(np.abs(got["ux"] - mac["ux"])) < 1e-12 * umax
        assert np.max(np.abs(got["uy"] - mac["uy"])) < 1e-12 * umax
        escale = np.abs(mac["Tmn"][..., 0, 0]).max()
        assert np.max(np.abs(got["e"] - mac["e"])) < 1e-12 * escale
        for k, (a, b) in zip(("T00", "T0x", "T0y", "Txx", "Txy", "Tyy"),
                             ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
            assert np.max(np.abs(got[k] - mac["Tmn"][..., a, b])) < 1e-12 * escale, k


def test_noalloc_rejects_eleven_group_stencils():
    import torch
    from paper_1703_04605_gb300 import build, _abi as A
    build.build()
    L = A.load()
    st = W.STENCIL_O3
    groups = A.int_array(st["groups"])
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = np.zeros(8)
    s = L.rlbm_moments_noalloc(groups, 11, st["m"], st["v0"], 2, 2, C.c_void_p(dummy.data_ptr()),
                               out.ctypes.data_as(C.POINTER(C.c_double)), A.M_N, None)
    assert s == A.RLBM_EINVAL
    assert b"six-group" in L.rlbm_last_error(None)


def test_noalloc_rejects_results_beyond_the_static_scratch():
    import torch
    from paper_1703_04605_gb300 import build, _abi as A
    build.build()
    L = A.load()
    st = W.STENCIL_M1
    groups = A.int_array(st["groups"])
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = np.zeros(8)
    # 11 planes x 1024 x 1024 doubles does not fit in 8 MiB
    s = L.rlbm_moments_noalloc(groups, 6, st["m"], st["v0"], 1024, 1024, C.c_void_p(dummy.data_ptr()),
                               out.ctypes.data_as(C.POINTER(C.c_double)), 0x7F, None)
    assert s == A.RLBM_EINVAL
    assert b"static scratch" in L.rlbm_last_error(None)
