"""Seeded synthetic inputs (initial fields and run parameters) of the five
benchmark workloads.  Input generation only: none of the method's arithmetic
lives here.  Shared by the tests, the benchmark and the oracle runs.

Stencils (six groups of Table I, folded to 2D):
  M1   G5, G12, G14, G17, G21, G26 at m = 1, v0 = 0.23342 (all weights
       positive for v0 in (0.233245, 0.233591)), Q = 58, halo 4
  G16  G1..G6 at m = 5, v0 = 0.398 (the paper's worked example), Q = 39, halo 2
  E5   G1, G14, G49, G51, G60, G70 at m = 0.36 (the stencil of the paper's
       BAMPS comparison), v0 = 0.1488232 (window (0.14882301, 0.14882336)),
       Q = 73, halo 6
"""
import math

import numpy as np

STENCIL_M1 = dict(groups=[5, 12, 14, 17, 21, 26], m=1.0, v0=0.23342)
STENCIL_G16 = dict(groups=[1, 2, 3, 4, 5, 6], m=5.0, v0=0.398)
STENCIL_E5 = dict(groups=[1, 14, 49, 51, 60, 70], m=0.36, v0=0.1488232)


def seed(config_index):
    return 1703 + int(config_index)


def _smooth_unit(rng, N, sigma):
    """White N(0,1) on an N x N periodic grid, Gaussian-smoothed (width sigma
    cells) by FFT, rescaled to zero mean and unit standard deviation."""
    g = rng.standard_normal((N, N))
    k = np.fft.fftfreq(N) * 2 * np.pi
    kx, ky = np.meshgrid(k, k)
    filt = np.exp(-0.5 * sigma * sigma * (kx * kx + ky * ky))
    s = np.real(np.fft.ifft2(np.fft.fft2(g) * filt))
    s -= s.mean()
    return s / s.std()


def sod(Nx=800, Ny=1, n=(1.0, 0.5), T=(1.0, 0.8), x0=None):
    """Quasi-1D relativistic shock tube: left state for x < x0."""
    x0 = Nx // 2 if x0 is None else x0
    x = np.arange(Nx)[None, :].repeat(Ny, 0)
    left = x < x0
    return dict(n=np.where(left, n[0], n[1]).astype(np.float64),
                ux=np.zeros((Ny, Nx)), uy=np.zeros((Ny, Nx)),
                T=np.where(left, T[0], T[1]).astype(np.float64))


def sod_tau(eta_over_s=0.1, v0=STENCIL_M1["v0"], n=1.0, T=1.0, d_g=16.0):
    """tau for a target eta/s, reading eta = (2/3) P (tau - 1/2)/v0 in units
    dx = c = T_R = 1 (Sec. IV: tau = tau_f v0/dx, eta = (2/3) P (tau_f - dt/2)),
    with s = 4n - n ln(n/n_eq), n_eq = d_g T^3/pi^2 (Sec. IV), left state."""
    s = 4 * n - n * math.log(n / (d_g * T ** 3 / math.pi ** 2))
    P = n * T
    return 0.5 + 1.5 * eta_over_s * s * v0 / P


def taylor_green(N=512, u0=0.05, n0=1.0, T0=1.0):
    k = 2 * np.pi / N
    x = np.arange(N)
    X, Y = np.meshgrid(x, x)
    return dict(n=np.full((N, N), n0), T=np.full((N, N), T0),
                ux=u0 * np.sin(k * X) * np.cos(k * Y), uy=-u0 * np.cos(k * X) * np.sin(k * Y))


def random_flow(N=4096, sigma=8.0, dn=0.01, dT=0.01, du=0.05, config_index=2):
    rng = np.random.default_rng(seed(config_index))
    g = [_smooth_unit(rng, N, sigma) for _ in range(4)]
    return dict(n=1.0 + dn * g[0], T=1.0 + dT * g[1], ux=du * g[2], uy=du * g[3])


def random_flow_crop(N_full=4096, crop=1024, **kw):
    """The same generator at full size, cropped (the crop is not periodic)."""
    f = random_flow(N_full, **kw)
    return {k: np.ascontiguousarray(v[:crop, :crop]) for k, v in f.items()}


def blast(N=8192, R=512, T_in=2.0, T_out=1.0):
    x = np.arange(N) - N / 2 + 0.5
    X, Y = np.meshgrid(x, x)
    inside = X * X + Y * Y < R * R
    return dict(n=np.ones((N, N)), ux=np.zeros((N, N)), uy=np.zeros((N, N)),
                T=np.where(inside, T_in, T_out))


def batch_specs(count=256, Lmin=64, Lmax=1024, mT=(0.1, 10.0), tau=(0.6, 1.5), m_min=0.36,
                config_index=3):
    """Independent lattices: side log-uniform, m/T log-uniform (clamped below
    at m_min, the smallest m with a positive quadrature here), tau uniform;
    even index Sod tube, odd index Taylor-Green vortex."""
    rng = np.random.default_rng(seed(config_index))
    out = []
    for i in range(count):
        L = int(round(math.exp(rng.uniform(math.log(Lmin), math.log(Lmax)))))
        m = math.exp(rng.uniform(math.log(mT[0]), math.log(mT[1])))
        spec = dict(L=L, m_drawn=m, m=max(m, m_min), tau=rng.uniform(*tau))
        if i % 2 == 0:
            nl, nr, tl, tr = rng.uniform(0.5, 1.5, 4)
            spec.update(kind="sod", n=(nl, nr), T=(tl, tr))
        else:
            spec.update(kind="tg", u0=rng.uniform(0.01, 0.1))
        out.append(spec)
    return out


def batch_fields(spec):
    L = spec["L"]
    if spec["kind"] == "sod":
        return sod(L, L, n=spec["n"], T=spec["T"])
    return taylor_green(L, u0=spec["u0"])
