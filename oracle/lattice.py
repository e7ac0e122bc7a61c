"""One relativistic lattice Boltzmann step, written out in the paper's order.

State: the pre-collision populations f_i(x, t) on a periodic lattice, shape
[Q, Ny, Nx] (folded 2D stencil) or [Q, Nz, Ny, Nx] (unfolded 3D stencil).

Per site (Sec. II A, Eq. 16-20, 28-29, 49):
 1. moments  N^a = sum_i f_i p_i^a,  T^ab = sum_i f_i p_i^a p_i^b  (Eq. 4-5 / 18)
 2. Landau frame: T^ab U_b = e U^a with U.U = 1, U^0 > 0 (Eq. 20); the
    eigenvector with a timelike direction is taken (np.linalg.eig, a library
    eigen-solver; the paper does not name its method)
 3. n = U_a N^a (Eq. 19)
 4. T from the equation of state e/n = 3T + m K1(m/T)/K2(m/T) (Eq. 28) by a
    bracketed Newton iteration to round-off (Sec. II B); e/n is strictly
    increasing in T so the root is unique
 5. f_i^eq (Eq. 16): route (i) of ``equilibrium`` on a second-order
    stencil, ``third_order`` on a third-order one
 6. Anderson-Witting relaxation with weight p_i.U/(p_i^0 tau) (Eq. 49)
 7. exact streaming by the integer displacement n_i (Eq. 49-50).

Metric diag(1,-1,-1,-1) (Sec. II), c = k_B = T_R = 1, lattice units dx = 1.
For the folded stencil the z components are absent from the moments (they
vanish by symmetry while U^z = 0) and the eigenproblem is 3 x 3.

TEST INFRASTRUCTURE ONLY (see the package docstring)."""
import numpy as np

from . import equilibrium as EQ
from . import polynomials as P
from . import quadrature as QD
from . import special as S
from . import third_order as TO


def landau(Tmn, dim):
    """Solve T^ab eta_bc U^c = e U^a per site.  Tmn[..., dim, dim] -> (e, U[..., dim])."""
    eta = np.diag([1.0] + [-1.0] * (dim - 1))
    M = Tmn @ eta
    shp = M.shape[:-2]
    vals, vecs = np.linalg.eig(M.reshape(-1, dim, dim))
    vals = vals.real
    vecs = vecs.real
    norm = vecs[:, 0, :] ** 2 - np.sum(vecs[:, 1:, :] ** 2, axis=1)   # U.U of each eigenvector
    score = np.where(norm > 0, vals, -np.inf)
    k = np.argmax(score, axis=1)
    idx = np.arange(vecs.shape[0])
    U = vecs[idx, :, k]
    U = U / np.sqrt(norm[idx, k])[:, None]
    U = U * np.sign(U[:, :1])
    e = vals[idx, k]
    return e.reshape(shp), U.reshape(shp + (dim,))


def temperature(e_over_n, m, max_iter=200):
    """Unique T with 3T + m R(m/T) = e/n (Eq. 28), R = K1/K2.
    Bracket: 0 < zeta (1 - R(zeta)) < 3/2 gives (e/n - m)/3 < T < (e/n - m)/1.5."""
    y = np.asarray(e_over_n, dtype=np.float64)
    lo = (y - m) / 3.0
    hi = (y - m) / 1.5
    if np.any(lo <= 0):
        raise ValueError("e/n must exceed m (Eq. 28)")
    T = 0.5 * (lo + hi)
    for _ in range(max_iter):
        z = m / T
        R = S.bessel_ratio_k1k2(z)
        g = 3.0 * T + m * R - y
        dR = R * R + 3.0 * R / z - 1.0            # dR/dzeta from the Bessel recurrences
        dg = 3.0 - z * z * dR                     # dg/dT
        lo = np.where(g < 0, T, lo)
        hi = np.where(g > 0, T, hi)
        Tn = T - g / dg
        bad = ~((Tn > lo) & (Tn < hi))
        Tn = np.where(bad, 0.5 * (lo + hi), Tn)
        done = np.abs(Tn - T) <= 1e-16 * np.abs(T)
        T = Tn
        if np.all(done):
            break
    return T


class Lattice:
    """Periodic lattice advanced by Eq. 49.  ``two_d`` selects the folded stencil."""

    def __init__(self, stencil, tau, shape, two_d=True):
        self.st = stencil
        self.tau = float(tau)
        self.two_d = two_d
        self.m = stencil.mbar
        self.consts = P.Constants(stencil.mbar)
        if two_d:
            self.w, self.p, self.d, _, _ = stencil.populations2d()
            self.dim = 3
            assert len(shape) == 2
        else:
            self.w, self.p, self.d, _ = stencil.populations3d()
            self.dim = 4
            assert len(shape) == 3
        self.shape = tuple(shape)
        self.Q = len(self.w)
        self.order = stencil.order
        self.eq3 = TO.ThirdOrder(stencil, two_d) if self.order == 3 else None
        self.f = None
        self.t = 0

    # -- fields -------------------------------------------------------------
    def four_velocity(self, ux, uy, uz=None):
        uz = np.zeros_like(ux) if uz is None else uz
        g = 1.0 / np.sqrt(1.0 - ux * ux - uy * uy - uz * uz)
        return np.stack([g, g * ux, g * uy, g * uz], axis=-1)

    def equilibrium(self, n, U, T):
        if self.eq3 is not None:
            return self.eq3.feq(self.w, n, U, T)
        return EQ.feq_route_i(self.w, self.p, n, U, T, self.consts)

    def init(self, n, ux, uy, T, uz=None):
        """f = f^eq(n, U, T) (the initial state; a collision leaves it unchanged)."""
        n = np.asarray(n, np.float64).reshape(self.shape)
        T = np.asarray(T, np.float64).reshape(self.shape)
        U = self.four_velocity(np.asarray(ux, np.float64).reshape(self.shape),
                               np.asarray(uy, np.float64).reshape(self.shape),
                               None if uz is None else np.asarray(uz, np.float64).reshape(self.shape))
        self.f = self.equilibrium(n, U, T)
        self.t = 0

    # -- per-site steps -----------------------------------------------------
    def moments(self, f=None):
        f = self.f if f is None else f
        pd = self.p[:, : self.dim]
        N = np.tensordot(pd.T, f, axes=([1], [0]))                       # [dim, ...]
        Tmn = np.einsum("ia,ib,i...->ab...", pd, pd, f)                  # [dim, dim, ...]
        return np.moveaxis(N, 0, -1), np.moveaxis(Tmn, (0, 1), (-2, -1))

    def macros(self, f=None):
        """n, U (contravariant, 4 components), T, e, N, T^ab of the pre-collision state."""
        N, Tmn = self.moments(f)
        e, Ud = landau(Tmn, self.dim)
        n = Ud[..., 0] * N[..., 0] - np.sum(Ud[..., 1:] * N[..., 1:], axis=-1)
        T = temperature(e / n, self.m)
        U = np.zeros(Ud.shape[:-1] + (4,))
        U[..., : self.dim] = Ud
        return dict(n=n, U=U, T=T, e=e, N=N, Tmn=Tmn,
                    ux=U[..., 1] / U[..., 0], uy=U[..., 2] / U[..., 0], uz=U[..., 3] / U[..., 0])

    def collide(self, f=None):
        """Post-collision populations f* = f - (p.U/(p0 tau)) (f - f^eq) (Eq. 49)."""
        f = self.f if f is None else f
        mac = self.macros(f)
        feq = self.equilibrium(mac["n"], mac["U"], mac["T"])
        U = mac["U"]
        pU = (self.p[:, 0, None] * U[..., 0].reshape(1, -1)
              - self.p[:, 1, None] * U[..., 1].reshape(1, -1)
              - self.p[:, 2, None] * U[..., 2].reshape(1, -1))
        if not self.two_d:
            pU = pU - self.p[:, 3, None] * U[..., 3].reshape(1, -1)
        omega = (pU / (self.p[:, 0, None] * self.tau)).reshape(f.shape)
        return f - omega * (f - feq)

    def stream(self, fstar):
        """f_i(x + n_i, t + 1) = f*_i(x, t) on the periodic lattice (Eq. 49-50)."""
        out = np.empty_like(fstar)
        nd = len(self.shape)
        axes = tuple(range(-1, -nd - 1, -1))                             # x, y, (z)
        for i in range(self.Q):
            out[i] = np.roll(fstar[i], shift=tuple(int(s) for s in self.d[i][:nd]), axis=axes)
        return out

    def step(self, k=1):
        for _ in range(k):
            self.f = self.stream(self.collide())
            self.t += 1


def make_lattice(group_ids, mbar, v0, tau, shape, two_d=True, w=None):
    return Lattice(QD.Stencil(group_ids, mbar, v0, w=w), tau, shape, two_d)
