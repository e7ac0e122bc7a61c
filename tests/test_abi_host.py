"""The C-ABI library without a GPU: it loads, exports every declared entry
point, validates arguments before touching a device, refuses to run without
one, and its host-side stencil builder reproduces the paper's printed
quadrature and the oracle."""
import ctypes as C
import os
import re
from decimal import Decimal

import numpy as np
import pytest

from conftest import ROOT, read_golden
from oracle import quadrature as QD
from oracle import special as S

A = pytest.importorskip("paper_1703_04605_gb300._abi")


@pytest.fixture(scope="module")
def lib():
    from paper_1703_04605_gb300 import build
    build.build()
    return A.load()


def _header_functions():
    with open(os.path.join(ROOT, "include", "rlbm.h")) as fh:
        txt = fh.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rlbm3?_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    declared = _header_functions()
    assert set(declared) == set(A.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_version(lib):
    assert b"sm_103a" in lib.rlbm_version()


def test_weights_reproduce_printed_quadrature(lib):
    gold = read_golden("quadrature_m5_G1-G6.txt")
    w = A.quadrature_weights([1, 2, 3, 4, 5, 6], 5.0, float(gold["v0"]))
    for k in range(6):
        assert abs(w[k] - float(gold["w%d" % (k + 1)])) < 1e-10


def test_window_reproduces_printed_pruning_points(lib):
    gold = read_golden("quadrature_m5_G1-G6.txt")
    lo, hi, nwin = A.quadrature_window([1, 2, 3, 4, 5, 6], 5.0)
    assert nwin == 1
    assert abs(lo - float(gold["v0_w2_zero"])) < 1e-10
    assert abs(hi - float(gold["v0_w3_zero"])) < 1e-10


@pytest.mark.parametrize("groups,m,v0", [([5, 12, 14, 17, 21, 26], 1.0, 0.23342),
                                         ([1, 14, 49, 51, 60, 70], 0.36, 0.1488232),
                                         ([1, 2, 3, 4, 5, 6], 5.0, 0.398)])
def test_weights_match_oracle(lib, groups, m, v0):
    w = A.quadrature_weights(groups, m, v0)
    wo = QD.weights_dec(groups, m, Decimal(v0))
    for a, b in zip(w, wo):
        assert abs(a / float(b) - 1) < 1e-13


def test_window_matches_oracle_m1(lib):
    lo, hi, _ = A.quadrature_window([5, 12, 14, 17, 21, 26], 1.0)
    (olo, ohi), = QD.positive_window([5, 12, 14, 17, 21, 26], 1.0, 0.2330, 0.2338, samples=17)
    assert abs(lo - olo) < 1e-9 and abs(hi - ohi) < 1e-9


O3 = [1, 2, 5, 6, 7, 9, 10, 11, 12, 13, 15]


def test_third_order_weights_and_window_match_oracle(lib):
    # eleven groups: the 11 x 11 system of the third-order conditions
    w = A.quadrature_weights(O3, 5.0, 0.27438)
    wo = QD.weights_dec(O3, 5.0, Decimal(0.27438))
    assert len(w) == 11
    for a, b in zip(w, wo):
        assert abs(a / float(b) - 1) < 1e-12
    lo, hi, nwin = A.quadrature_window(O3, 5.0)
    (olo, ohi), = QD.positive_window(O3, 5.0, 0.2730, 0.2755, samples=26)
    assert nwin == 1
    assert abs(lo - olo) < 1e-9 and abs(hi - ohi) < 1e-9


def test_third_order_create_validates_before_device(lib):
    assert _create(lib, groups=O3[:10] + [1], m=5.0, v0=0.27438)[0] == A.RLBM_EINVAL
    assert _create(lib, groups=O3, m=5.0, v0=0.26)[0] == A.RLBM_ENOQUAD
    assert b"weight" in lib.rlbm_last_error(None)
    assert _create(lib, groups=O3, m=5.0, v0=0.27438, dtype=2)[0] == A.RLBM_ENOTSUP


def test_ratio_tables_against_oracle_bessel(lib):
    rng = np.random.default_rng(3)
    z = np.exp(rng.uniform(np.log(2.0 ** -18), np.log(2.0 ** 18), 60))
    for x in z:
        ref = float(S.kv_dec(1, x) / S.kv_dec(2, x))
        assert abs(A.bessel_ratio(x, 64) / ref - 1) < 5e-16, x
        assert abs(A.bessel_ratio(x, 32) / ref - 1) < 3e-7, x


def _create(lib, groups=(5, 12, 14, 17, 21, 26), m=1.0, tau=0.8, Nx=8, Ny=8, dtype=1, v0=0.23342):
    g = A.int_array(groups)
    st = A.Stencil(len(groups), g, v0)
    ctx = C.c_void_p()
    s = lib.rlbm_create(C.byref(st), m, tau, Nx, Ny, dtype, None, C.byref(ctx))
    return s, ctx


def test_create_validates_before_device(lib):
    assert _create(lib, tau=0.5)[0] == A.RLBM_EINVAL
    assert _create(lib, Nx=0)[0] == A.RLBM_EINVAL
    assert _create(lib, Nx=65536, Ny=32768)[0] == A.RLBM_EINVAL      # 2^31 sites: 32-bit site index
    # fewer than 2^31 sites, but a plane of 32 x (2^31 - 1) padded elements:
    # beyond the kernels' 32-bit element indices (refused before any device work)
    assert _create(lib, Nx=1, Ny=2 ** 31 - 1)[0] == A.RLBM_ENOTSUP
    assert _create(lib, groups=(5, 12, 14, 17, 21))[0] == A.RLBM_EINVAL
    assert _create(lib, groups=(5, 12, 14, 17, 21, 21))[0] == A.RLBM_EINVAL
    assert _create(lib, groups=(5, 12, 14, 17, 21, 85))[0] == A.RLBM_EINVAL
    assert _create(lib, m=-1.0)[0] == A.RLBM_EINVAL
    assert _create(lib, dtype=7)[0] == A.RLBM_EINVAL
    # a v0 outside the positive window is rejected (Sec. III D: w > 0)
    s, _ = _create(lib, v0=0.20)
    assert s == A.RLBM_ENOQUAD
    assert b"weight" in lib.rlbm_last_error(None)


@pytest.mark.skipif(os.environ.get("CUDA_VISIBLE_DEVICES") is None and os.path.exists("/dev/nvidia0"),
                    reason="a GPU is visible")
def test_no_device_is_an_error_not_a_fallback(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is visible")
    except ImportError:
        pass
    s, ctx = _create(lib)
    assert s == A.RLBM_ECUDA and not ctx.value
    assert b"device" in lib.rlbm_last_error(None)


def test_null_context_calls(lib):
    assert lib.rlbm_step(None, 1) == A.RLBM_EINVAL
    assert lib.rlbm_sync(None) == A.RLBM_EINVAL
    assert lib.rlbm_moments_size(None, 1) == 0
    lib.rlbm_destroy(None)
    assert lib.rlbm_batch_step(None, 1, 1) == A.RLBM_EINVAL
    assert lib.rlbm_batch_tuning(None, 1, None, None) == A.RLBM_EINVAL
    null2 = (C.c_void_p * 2)(None, None)
    assert lib.rlbm_batch_step(null2, 2, 1) == A.RLBM_EINVAL
    assert lib.rlbm_batch_tuning(null2, 2, None, None) == A.RLBM_EINVAL


def test_noalloc_size_check_does_not_wrap(lib):
    """planes x Nx x Ny beyond 2^64 must still be rejected by the size check,
    which runs before any device call (the pointer is never dereferenced)."""
    g = A.int_array([5, 12, 14, 17, 21, 26])
    out = np.zeros(1)
    big = 2 ** 31 - 1                                  # 11 x big^2 wraps 64 bits
    s = lib.rlbm_moments_noalloc(g, 6, 1.0, 0.23342, big, big, C.c_void_p(256),
                                 out.ctypes.data_as(C.POINTER(C.c_double)), 0x7F, None)
    assert s == A.RLBM_EINVAL
    assert b"static scratch" in lib.rlbm_last_error(None)
    s = lib.rlbm_moments_noalloc(g, 11, 1.0, 0.23342, 4, 4, C.c_void_p(256),
                                 out.ctypes.data_as(C.POINTER(C.c_double)), 0x01, None)
    assert s == A.RLBM_EINVAL
    assert b"six-group" in lib.rlbm_last_error(None)


def test_3d_entry_points_without_device(lib):
    g = A.int_array([1, 2, 3, 4, 5, 6])
    st = A.Stencil(6, g, 0.398)
    ctx = C.c_void_p()
    assert lib.rlbm3_create(C.byref(st), 5.0, 0.8, 4, 4, 0, 0, None, C.byref(ctx)) == A.RLBM_EINVAL
    assert lib.rlbm3_create(C.byref(st), 5.0, 0.8, 2048, 1024, 1024, 0, None, C.byref(ctx)) == A.RLBM_EINVAL
    assert lib.rlbm3_create(C.byref(st), 5.0, 0.5, 4, 4, 4, 0, None, C.byref(ctx)) == A.RLBM_EINVAL
    assert lib.rlbm3_create(C.byref(st), 5.0, 0.8, 4, 4, 4, 2, None, C.byref(ctx)) == A.RLBM_ENOTSUP
    s = lib.rlbm3_create(C.byref(st), 5.0, 0.8, 4, 4, 4, 0, None, C.byref(ctx))
    assert s == A.RLBM_ECUDA and not ctx.value
    assert b"device" in lib.rlbm3_last_error(None)
    assert lib.rlbm3_step(None, 1) == A.RLBM_EINVAL
    assert lib.rlbm3_sync(None) == A.RLBM_EINVAL
    assert lib.rlbm3_moments_size(None, 1) == 0
    lib.rlbm3_destroy(None)


def test_init_device_refuses_fields_it_cannot_read():
    # the device initialiser reads Nx*Ny doubles per pointer: host arrays,
    # CPU tensors, other dtypes and other sizes are refused before the call
    torch = pytest.importorskip("torch")
    from paper_1703_04605_gb300.lattice import Lattice
    lat = Lattice.__new__(Lattice)
    lat.Nx, lat.Ny = 4, 3
    ok = torch.zeros(12, dtype=torch.float64)
    for bad in (np.zeros(12), ok, torch.zeros(12, dtype=torch.float32), torch.zeros(11, dtype=torch.float64)):
        with pytest.raises(ValueError):
            lat.init_device(bad, ok, ok, ok)


def test_allocator_setter_validates_and_resets(lib):
    from paper_1703_04605_gb300 import use_cuda_malloc, use_torch_allocator
    fa = A.ALLOC_FN(lambda nbytes, dev, stream, user: None)
    ff = A.FREE_FN(lambda ptr, user: None)
    alloc, free = C.cast(fa, C.c_void_p), C.cast(ff, C.c_void_p)
    assert lib.rlbm_set_allocator(alloc, None, None) == A.RLBM_EINVAL
    assert lib.rlbm_set_allocator(None, free, None) == A.RLBM_EINVAL
    assert b"both" in lib.rlbm_last_error(None)
    assert lib.rlbm_set_allocator(alloc, free, None) == A.RLBM_OK
    assert lib.rlbm_set_allocator(None, None, None) == A.RLBM_OK
    use_torch_allocator()           # installs ctypes callbacks; no device is touched
    use_cuda_malloc()


def test_binding_rejects_unknown_storage_types():
    from paper_1703_04605_gb300 import Lattice, Lattice3D
    with pytest.raises(ValueError, match="dtype"):
        Lattice([5, 12, 14, 17, 21, 26], 1.0, 0.8, 8, 8, dtype="f16")
    with pytest.raises(ValueError, match="dtype"):
        Lattice3D([5, 12, 14, 17, 21, 26], 1.0, 0.8, 4, 4, 4, dtype="fp32")
