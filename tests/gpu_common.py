"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare macroscopic fields."""
from decimal import Decimal

import numpy as np

from oracle import lattice as OL
from oracle import quadrature as QD


def smooth_fields(Nx, Ny, seed, dn=0.1, dT=0.1, du=0.1, modes=3):
    """Periodic smooth random fields: a few random Fourier modes per field."""
    rng = np.random.default_rng(seed)
    x = np.arange(Nx)[None, :]
    y = np.arange(Ny)[:, None]

    def field():
        f = np.zeros((Ny, Nx))
        for _ in range(modes):
            kx = rng.integers(0, 3) * 2 * np.pi / Nx
            ky = rng.integers(0, 3) * 2 * np.pi / Ny
            f += rng.uniform(-1, 1) * np.cos(kx * x + ky * y + rng.uniform(0, 2 * np.pi))
        return f / modes

    return dict(n=1 + dn * field(), T=1 + dT * field(), ux=du * field(), uy=du * field())


def run_gpu(stencil, tau, fields, dtype, steps, Nx=None, Ny=None):
    from paper_1703_04605_gb300 import Lattice
    Ny_, Nx_ = fields["n"].shape
    with Lattice(stencil["groups"], stencil["m"], tau, Nx_, Ny_, dtype=dtype, v0=stencil["v0"]) as lat:
        lat.init(fields["n"], fields["ux"], fields["uy"], fields["T"])
        lat.step(steps)
        out = lat.moments()
        info = lat.info()
    return out, info


def oracle_lattice(stencil, tau, shape):
    # the exact binary value of v0 that the library receives
    st = QD.Stencil(stencil["groups"], stencil["m"], stencil["v0"],
                    w=QD.weights(stencil["groups"], stencil["m"], Decimal(stencil["v0"])))
    return OL.Lattice(st, tau, shape)


def run_oracle(stencil, tau, fields, steps):
    lat = oracle_lattice(stencil, tau, fields["n"].shape)
    lat.init(fields["n"], fields["ux"], fields["uy"], fields["T"])
    lat.step(steps)
    return lat.macros()


def errors(got, ref):
    """max relative error of n and T; max |du| / max |u_ref| for velocities."""
    en = np.max(np.abs(got["n"] / ref["n"] - 1))
    eT = np.max(np.abs(got["T"] / ref["T"] - 1))
    umax = max(np.max(np.abs(ref["ux"])), np.max(np.abs(ref["uy"])), 1e-300)
    eu = max(np.max(np.abs(got["ux"] - ref["ux"])), np.max(np.abs(got["uy"] - ref["uy"]))) / umax
    return dict(n=en, T=eT, u=eu)
