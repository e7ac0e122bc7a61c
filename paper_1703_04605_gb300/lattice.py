"""Python handle on one lattice context of librlbm (marshalling only)."""
import ctypes as C

import numpy as np

from . import _abi as A


def _dtype_code(dtype, allowed):
    if dtype not in allowed:
        raise ValueError("dtype must be one of %s, not %r" % (", ".join(repr(d) for d in allowed), dtype))
    return A.DTYPES[dtype]


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Lattice:
    """A periodic Nx x Ny lattice advanced by the library's CUDA kernels.

    groups  six group ids of Table I (second-order equilibrium) or eleven
    (third order); m = m/T_R; tau in lattice steps;
    dtype   'f64' | 'f32' | 'bf16dev';  v0 = 0 picks the centre of the widest
    positive-weight window.  stream: a cudaStream_t as int (default: torch's
    current stream when torch sees a GPU, else the legacy default stream)."""

    def __init__(self, groups, m, tau, Nx, Ny, dtype="f32", v0=0.0, stream=None):
        L = A.load()
        self._lib = L
        self._ctx = C.c_void_p()
        self._groups = A.int_array(groups)
        st = A.Stencil(len(groups), self._groups, float(v0))
        if stream is None:
            stream = _default_stream()
        code = _dtype_code(dtype, ("f64", "f32", "bf16dev"))
        A.check(L.rlbm_create(C.byref(st), float(m), float(tau), int(Nx), int(Ny), code,
                              C.c_void_p(stream) if stream else None, C.byref(self._ctx)))
        self.Nx, self.Ny = int(Nx), int(Ny)
        self.dtype = dtype

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._lib.rlbm_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls --------------------------------------------------------------
    def _chk(self, status):
        A.check(status, self._ctx)

    def init(self, n, ux, uy, T):
        """Host FP64 fields (anything convertible to [Ny, Nx] float64)."""
        arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (self.Ny, self.Nx)))
                for a in (n, ux, uy, T)]
        ptrs = [a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs]
        self._chk(self._lib.rlbm_init(self._ctx, *ptrs))

    def init_device(self, n, ux, uy, T):
        """Device fields: four contiguous CUDA float64 tensors of Nx*Ny elements
        (the kernel reads Nx*Ny doubles from each pointer, so any other dtype
        or size is refused here)."""
        import torch
        for t in (n, ux, uy, T):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                    and t.is_contiguous() and t.numel() == self.Nx * self.Ny):
                raise ValueError("device fields must be contiguous CUDA tensors of Nx*Ny float64")
        self._chk(self._lib.rlbm_init_device(self._ctx, *[C.c_void_p(t.data_ptr()) for t in (n, ux, uy, T)]))

    def set_extended_sums(self, level=1):
        """FP32 storage on a compiled stencil: moment sums in extended
        precision (rlbm_set_extended_sums; level 0 off, 1 mass and energy,
        2 also momentum; True means 1)."""
        self._chk(self._lib.rlbm_set_extended_sums(self._ctx, int(level)))

    def step(self, k=1):
        self._chk(self._lib.rlbm_step(self._ctx, int(k)))

    def sync(self):
        self._chk(self._lib.rlbm_sync(self._ctx))

    def moments_size(self, mask=A.M_N | A.M_UX | A.M_UY | A.M_T | A.M_E):
        """Doubles that moments(mask) writes (rlbm_moments_size)."""
        return int(self._lib.rlbm_moments_size(self._ctx, mask))

    def moments(self, mask=A.M_N | A.M_UX | A.M_UY | A.M_T | A.M_E, out=None):
        """Fields of the current state as [Ny, Nx] views of one buffer.  out:
        an optional C-contiguous float64 array of at least
        rlbm_moments_size(mask) elements to receive them (page-locked host
        memory makes the device-to-host copy direct); default a new array."""
        size = self._lib.rlbm_moments_size(self._ctx, mask)
        if out is None:
            out = np.empty(size, dtype=np.float64)
        else:
            out = np.asarray(out)
            if out.dtype != np.float64 or not out.flags.c_contiguous or out.size < size:
                raise ValueError("out must be a C-contiguous float64 array of at least %d elements" % size)
            out = out.reshape(-1)
        self._chk(self._lib.rlbm_moments(self._ctx, out.ctypes.data_as(C.POINTER(C.c_double)), mask))
        res = {}
        plane = 0
        N = self.Nx * self.Ny
        for bit, names in A.MASK_PLANES:
            if mask & bit:
                for nm in names:
                    res[nm] = out[plane * N:(plane + 1) * N].reshape(self.Ny, self.Nx)
                    plane += 1
        return res

    def info(self):
        inf = A.Info()
        self._chk(self._lib.rlbm_get_info(self._ctx, C.byref(inf)))
        out = {k: (list(getattr(inf, k)) if k == "w_group" else getattr(inf, k)) for k, _ in A.Info._fields_}
        out["w_group"] = out["w_group"][: 11 if out["order"] == 3 else 6]
        return out


# The callbacks handed to rlbm_set_allocator stay referenced for the life of
# the process: a context frees through the pair it was created with.
_ALLOCATORS = []


def _torch_alloc(nbytes, device, stream, user):
    try:
        import torch
        return torch.cuda.caching_allocator_alloc(int(nbytes), device=int(device), stream=int(stream or 0))
    except Exception:
        return None            # the library reports ENOMEM


def _torch_free(ptr, user):
    try:
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:
        pass


def use_torch_allocator():
    """Contexts created from now on (2D and 3D) take their device memory from
    torch's caching allocator, on the context's stream (rlbm_set_allocator)."""
    pair = (A.ALLOC_FN(_torch_alloc), A.FREE_FN(_torch_free))
    _ALLOCATORS.append(pair)
    A.check(A.load().rlbm_set_allocator(C.cast(pair[0], C.c_void_p), C.cast(pair[1], C.c_void_p), None))


def use_cuda_malloc():
    """Contexts created from now on allocate with cudaMalloc (the default)."""
    A.check(A.load().rlbm_set_allocator(None, None, None))


def batch_step(lattices, k=1):
    """Advance every lattice by k steps as one batch (rlbm_batch_step)."""
    L = A.load()
    arr = (C.c_void_p * len(lattices))(*[lat._ctx.value for lat in lattices])
    A.check(L.rlbm_batch_step(arr, len(lattices), int(k)))


def set_batch_options(engine="auto", spin_limit=0, wait_offset=0):
    """Process-wide batch engine choice ('auto', 'graph' or 'persistent') and
    the persistent engine's bounded waits (rlbm_batch_set_options);
    wait_offset > 0 makes every wait unmeetable (testing the timeout path)."""
    codes = {"auto": A.BATCH_AUTO, "graph": A.BATCH_GRAPH, "persistent": A.BATCH_PERSISTENT}
    if engine not in codes:
        raise ValueError("engine must be one of %s" % ", ".join(sorted(codes)))
    opt = A.BatchOptions(codes[engine], int(spin_limit), int(wait_offset))
    A.check(A.load().rlbm_batch_set_options(C.byref(opt)))


def batch_engine(lattices):
    """The engine chosen for a batch: dict(engine='graph'|'persistent',
    param=G or sites per thread, launches=per step (graph) or per call)."""
    L = A.load()
    arr = (C.c_void_p * len(lattices))(*[lat._ctx.value for lat in lattices])
    out = [C.c_int(0) for _ in range(3)]
    A.check(L.rlbm_batch_engine(arr, len(lattices), *[C.byref(o) for o in out]))
    return dict(engine={A.BATCH_GRAPH: "graph", A.BATCH_PERSISTENT: "persistent"}.get(out[0].value, "?"),
                param=out[1].value, launches=out[2].value)


def batch_tuning(lattices):
    """The autotuner's choice for a batch already tuned by batch_step:
    dict(steps_per_graph, launches_per_step)."""
    L = A.load()
    arr = (C.c_void_p * len(lattices))(*[lat._ctx.value for lat in lattices])
    out = [C.c_int(0) for _ in range(2)]
    A.check(L.rlbm_batch_tuning(arr, len(lattices), *[C.byref(o) for o in out]))
    return dict(steps_per_graph=out[0].value, launches_per_step=out[1].value)


class Lattice3D:
    """A periodic Nx x Ny x Nz lattice with the unfolded stencil (the
    rlbm3_* entry points).  Fields are [Nz, Ny, Nx] arrays; dtype 'f64' or
    'f32'; v0 = 0 picks the centre of the widest positive-weight window."""

    def __init__(self, groups, m, tau, Nx, Ny, Nz, dtype="f64", v0=0.0, stream=None):
        L = A.load()
        self._lib = L
        self._ctx = C.c_void_p()
        self._groups = A.int_array(groups)
        st = A.Stencil(len(groups), self._groups, float(v0))
        if stream is None:
            stream = _default_stream()
        code = _dtype_code(dtype, ("f64", "f32", "bf16dev"))
        A.check(L.rlbm3_create(C.byref(st), float(m), float(tau), int(Nx), int(Ny), int(Nz), code,
                               C.c_void_p(stream) if stream else None, C.byref(self._ctx)), None, True)
        self.Nx, self.Ny, self.Nz = int(Nx), int(Ny), int(Nz)
        self.dtype = dtype

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._lib.rlbm3_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _chk(self, status):
        A.check(status, self._ctx, True)

    def init(self, n, ux, uy, uz, T):
        shape = (self.Nz, self.Ny, self.Nx)
        arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shape))
                for a in (n, ux, uy, uz, T)]
        ptrs = [a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs]
        self._chk(self._lib.rlbm3_init(self._ctx, *ptrs))

    def step(self, k=1):
        self._chk(self._lib.rlbm3_step(self._ctx, int(k)))

    def sync(self):
        self._chk(self._lib.rlbm3_sync(self._ctx))

    def moments_size(self, mask=A.M_N | A.M_UX | A.M_UY | A.M_UZ | A.M_T | A.M_E):
        """Doubles that moments(mask) writes (rlbm3_moments_size)."""
        return int(self._lib.rlbm3_moments_size(self._ctx, mask))

    def moments(self, mask=A.M_N | A.M_UX | A.M_UY | A.M_UZ | A.M_T | A.M_E, out=None):
        """Fields as [Nz, Ny, Nx] views of one buffer; out as in Lattice.moments."""
        size = self._lib.rlbm3_moments_size(self._ctx, mask)
        if out is None:
            out = np.empty(size, dtype=np.float64)
        else:
            out = np.asarray(out)
            if out.dtype != np.float64 or not out.flags.c_contiguous or out.size < size:
                raise ValueError("out must be a C-contiguous float64 array of at least %d elements" % size)
            out = out.reshape(-1)
        self._chk(self._lib.rlbm3_moments(self._ctx, out.ctypes.data_as(C.POINTER(C.c_double)), mask))
        res, plane = {}, 0
        N = self.Nx * self.Ny * self.Nz
        for bit, names in A.MASK_PLANES3:
            if mask & bit:
                for nm in names:
                    res[nm] = out[plane * N:(plane + 1) * N].reshape(self.Nz, self.Ny, self.Nx)
                    plane += 1
        return res

    def info(self):
        inf = A.Info3()
        self._chk(self._lib.rlbm3_get_info(self._ctx, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in A.Info3._fields_}
