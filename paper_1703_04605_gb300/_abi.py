"""ctypes declarations of include/rlbm.h (argument marshalling only).

The shared library must exist (build it with ``paper_1703_04605_gb300.build``);
there is no fallback implementation: every step of the method runs in the
library's CUDA kernels."""
import ctypes as C
import os

from . import build as _build

RLBM_OK, RLBM_EINVAL, RLBM_ENOQUAD, RLBM_ENOMEM, RLBM_ECUDA, RLBM_ENONPHYS, RLBM_ETIMEOUT, RLBM_ENOTSUP = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOQUAD", "ENOMEM", "ECUDA", "ENONPHYS", "ETIMEOUT", "ENOTSUP"]
DTYPES = {"f64": 0, "f32": 1, "bf16dev": 2}

M_N, M_UX, M_UY, M_T, M_E, M_NVEC, M_TMN, M_UZ = 0x01, 0x02, 0x04, 0x08, 0x10, 0x20, 0x40, 0x80
MASK_PLANES = [(M_N, ["n"]), (M_UX, ["ux"]), (M_UY, ["uy"]), (M_T, ["T"]), (M_E, ["e"]),
               (M_NVEC, ["N0", "Nx", "Ny"]), (M_TMN, ["T00", "T0x", "T0y", "Txx", "Txy", "Tyy"])]
MASK_PLANES3 = [(M_N, ["n"]), (M_UX, ["ux"]), (M_UY, ["uy"]), (M_T, ["T"]), (M_E, ["e"]),
                (M_NVEC, ["N0", "Nx", "Ny", "Nz"]),
                (M_TMN, ["T00", "T0x", "T0y", "T0z", "Txx", "Txy", "Txz", "Tyy", "Tyz", "Tzz"]), (M_UZ, ["uz"])]

# every entry point declared in include/rlbm.h
EXPORTS = ["rlbm_create", "rlbm_init", "rlbm_init_device", "rlbm_step", "rlbm_moments",
           "rlbm_moments_size", "rlbm_sync", "rlbm_get_info", "rlbm_last_error", "rlbm_destroy",
           "rlbm_quadrature_weights", "rlbm_quadrature_window", "rlbm_bessel_ratio", "rlbm_version",
           "rlbm_moments_noalloc", "rlbm_batch_step", "rlbm_set_extended_sums", "rlbm_fp64_fma_rate",
           "rlbm_batch_set_options", "rlbm_batch_engine", "rlbm_batch_tuning", "rlbm_set_allocator",
           "rlbm3_create", "rlbm3_init", "rlbm3_step", "rlbm3_moments", "rlbm3_moments_size", "rlbm3_sync",
           "rlbm3_get_info", "rlbm3_last_error", "rlbm3_destroy"]


# rlbm_alloc_fn(bytes, device, stream, user) -> pointer; rlbm_free_fn(ptr, user)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_int, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Stencil(C.Structure):
    _fields_ = [("ngroups", C.c_int), ("groups", C.POINTER(C.c_int)), ("v0", C.c_double)]


class BatchOptions(C.Structure):
    _fields_ = [("engine", C.c_int), ("spin_limit", C.c_uint), ("wait_offset", C.c_uint)]


BATCH_AUTO, BATCH_GRAPH, BATCH_PERSISTENT = 0, 1, 2


class Info(C.Structure):
    _fields_ = [("Nx", C.c_int), ("Ny", C.c_int), ("Q", C.c_int), ("halo", C.c_int),
                ("dtype", C.c_int), ("m", C.c_double), ("tau", C.c_double), ("v0", C.c_double),
                ("w_group", C.c_double * 11), ("t", C.c_longlong), ("bytes_per_site", C.c_size_t),
                ("extra_bytes_per_site", C.c_size_t), ("device_bytes", C.c_size_t), ("kernel", C.c_int),
                ("order", C.c_int), ("extended_sums", C.c_int)]


class Info3(C.Structure):
    _fields_ = [("Nx", C.c_int), ("Ny", C.c_int), ("Nz", C.c_int), ("Q", C.c_int), ("halo", C.c_int),
                ("dtype", C.c_int), ("m", C.c_double), ("tau", C.c_double), ("v0", C.c_double),
                ("t", C.c_longlong), ("bytes_per_site", C.c_size_t), ("device_bytes", C.c_size_t),
                ("kernel", C.c_int), ("order", C.c_int)]


class RLBMError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))


_lib = None


def lib_path():
    return _build.LIB


def load():
    """Load librlbm.so; raises ImportError when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError("librlbm.so is not built (run paper_1703_04605_gb300.build.build()); "
                          "there is no fallback implementation")
    L = C.CDLL(path)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    sig = {
        "rlbm_create": (C.c_int, [C.POINTER(Stencil), C.c_double, C.c_double, C.c_int, C.c_int,
                                  C.c_int, P, C.POINTER(P)]),
        "rlbm_init": (C.c_int, [P, dp, dp, dp, dp]),
        "rlbm_init_device": (C.c_int, [P, P, P, P, P]),
        "rlbm_step": (C.c_int, [P, C.c_int]),
        "rlbm_set_extended_sums": (C.c_int, [P, C.c_int]),
        "rlbm_fp64_fma_rate": (C.c_int, [P, dp]),
        "rlbm_batch_set_options": (C.c_int, [C.POINTER(BatchOptions)]),
        "rlbm_batch_engine": (C.c_int, [C.POINTER(P), C.c_int, ip, ip, ip]),
        "rlbm_moments": (C.c_int, [P, dp, C.c_uint]),
        "rlbm_moments_size": (C.c_size_t, [P, C.c_uint]),
        "rlbm_sync": (C.c_int, [P]),
        "rlbm_get_info": (C.c_int, [P, C.POINTER(Info)]),
        "rlbm_last_error": (C.c_char_p, [P]),
        "rlbm_destroy": (None, [P]),
        "rlbm_quadrature_weights": (C.c_int, [ip, C.c_int, C.c_double, C.c_double, dp]),
        "rlbm_quadrature_window": (C.c_int, [ip, C.c_int, C.c_double, dp, dp, ip]),
        "rlbm_bessel_ratio": (C.c_double, [C.c_double, C.c_int]),
        "rlbm_version": (C.c_char_p, []),
        "rlbm_batch_step": (C.c_int, [C.POINTER(P), C.c_int, C.c_int]),
        # the two callbacks as pointers (ALLOC_FN / FREE_FN instances cast to
        # c_void_p, or None for NULL)
        "rlbm_set_allocator": (C.c_int, [P, P, P]),
        "rlbm_batch_tuning": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "rlbm_moments_noalloc": (C.c_int, [ip, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, P, dp,
                                           C.c_uint, P]),
        "rlbm3_create": (C.c_int, [C.POINTER(Stencil), C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                                   C.c_int, P, C.POINTER(P)]),
        "rlbm3_init": (C.c_int, [P, dp, dp, dp, dp, dp]),
        "rlbm3_step": (C.c_int, [P, C.c_int]),
        "rlbm3_moments": (C.c_int, [P, dp, C.c_uint]),
        "rlbm3_moments_size": (C.c_size_t, [P, C.c_uint]),
        "rlbm3_sync": (C.c_int, [P]),
        "rlbm3_get_info": (C.c_int, [P, C.POINTER(Info3)]),
        "rlbm3_last_error": (C.c_char_p, [P]),
        "rlbm3_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(status, ctx=None, three_d=False):
    if status != RLBM_OK:
        L = load()
        msg = (L.rlbm3_last_error if three_d else L.rlbm_last_error)(ctx)
        raise RLBMError(status, msg.decode() if msg else "")


def int_array(values):
    arr = (C.c_int * len(values))(*[int(v) for v in values])
    return arr


def quadrature_weights(groups, m, v0):
    out = (C.c_double * len(groups))()
    g = int_array(groups)
    check(load().rlbm_quadrature_weights(g, len(groups), float(m), float(v0), out))
    return list(out)


def quadrature_window(groups, m):
    lo, hi, nw = C.c_double(), C.c_double(), C.c_int()
    g = int_array(groups)
    check(load().rlbm_quadrature_window(g, len(groups), float(m), C.byref(lo), C.byref(hi), C.byref(nw)))
    return lo.value, hi.value, nw.value


def bessel_ratio(zeta, precision=64):
    return load().rlbm_bessel_ratio(float(zeta), int(precision))
