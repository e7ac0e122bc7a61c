"""Quadratures with prescribed abscissae (Sec. III C-D) and the 2D fold.

A stencil is a list of groups of Table I.  With a common velocity parameter
v0 the i-th vector n_{i,k} of group k carries the four-momentum (Eq. 48)

    p_{i,k} = mbar * gamma_k * (1, v0 n_{i,k}),   gamma_k = 1/sqrt(1 - v0^2 ||n_k||^2)

(T_R = 1, so momenta are in units of T_R).  The weights w_k solve Eq. 47
(discrete orthonormality of the polynomials of Sec. III A up to second
order).  Discrete orthonormality of all polynomials of degree <= 2 is the same
as exactness of the quadrature for every product of two of them, i.e. every
on-shell monomial of degree <= 4.  For full-symmetric groups the odd monomials
vanish on both sides and p0^2 = mbar^2 + |p|^2 holds at every node, so the
conditions reduce to the six monomials of ``special.MONOMIALS6`` -- the "6
linearly independent components" of Sec. III D -- giving the square system
A(v0) w = b of Eq. 52 with A[phi][k] = sum_{i in G_k} phi(p_{i,k}) and
b[phi] = <phi> (rest-frame moment of the weight).  A third-order stencil (11
groups) is exact for every product of two polynomials of degree <= 3, i.e.
every monomial of degree <= 6, and the eleven monomials of
``special.MONOMIALS11`` give the square 11 x 11 system (Sec. III D: eleven
independent components at third order).  It is solved in 60-digit
decimal arithmetic (the system is ill conditioned for small mbar, Sec. III D)
and rounded to FP64 at the end.

TEST INFRASTRUCTURE ONLY (see the package docstring)."""
from decimal import Decimal

import numpy as np

from . import groups as G
from . import special as S


def _gamma_dec(v0, len2):
    return Decimal(1) / (Decimal(1) - v0 * v0 * Decimal(len2)).sqrt()


def _phi_dec(name, p0, px, py, pz):
    if name == "1":
        return Decimal(1)
    if name == "p0":
        return p0
    if name == "px2":
        return px * px
    if name == "p0px2":
        return p0 * px * px
    if name == "px4":
        return px ** 4
    if name == "px2py2":
        return px * px * py * py
    if name == "p0px4":
        return p0 * px ** 4
    if name == "p0px2py2":
        return p0 * px * px * py * py
    if name == "px6":
        return px ** 6
    if name == "px4py2":
        return px ** 4 * py * py
    if name == "px2py2pz2":
        return px * px * py * py * pz * pz
    raise KeyError(name)


def order_of(group_ids):
    """Expansion order fixed by the number of groups (Sec. III D): 6 -> 2, 11 -> 3."""
    n = len(group_ids)
    if n == 6:
        return 2
    if n == 11:
        return 3
    raise ValueError("a stencil needs 6 groups (second order) or 11 groups (third order), Sec. III D")


def monomials_for(order):
    return S.MONOMIALS6 if order == 2 else S.MONOMIALS11


def _solve_dec(A, b):
    """Gaussian elimination with partial pivoting on lists of Decimals."""
    n = len(b)
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for c in range(n):
        piv = max(range(c, n), key=lambda r: abs(M[r][c]))
        if M[piv][c] == 0:
            raise ValueError("singular quadrature system")
        M[c], M[piv] = M[piv], M[c]
        for r in range(c + 1, n):
            fac = M[r][c] / M[c][c]
            for k in range(c, n + 1):
                M[r][k] -= fac * M[c][k]
    x = [Decimal(0)] * n
    for r in range(n - 1, -1, -1):
        s = M[r][n] - sum(M[r][k] * x[k] for k in range(r + 1, n))
        x[r] = s / M[r][r]
    return x


class MomentCache:
    """Rest-frame moments b[phi] of one mbar and order (they do not depend on v0)."""

    def __init__(self, mbar, order=2):
        self.mbar = S._dec(mbar)
        self.order = order
        self.b = [S.rest_moment_dec(nm, self.mbar) for nm in monomials_for(order)]


def system_dec(group_ids, mbar, v0, cache=None):
    """A(v0) and b of Eq. 52 in decimal arithmetic (rows = the order's
    monomials, cols = groups)."""
    order = order_of(group_ids)
    if cache is None or cache.order != order:
        cache = MomentCache(mbar, order)
    names = monomials_for(order)
    K = len(group_ids)
    m = cache.mbar
    v0 = S._dec(v0)
    A = [[Decimal(0)] * K for _ in range(K)]
    for k, gid in enumerate(group_ids):
        len2 = G.length2(gid)
        if v0 * v0 * len2 >= 1:
            raise ValueError("v0 * ||n_k|| must stay below the speed of light (Sec. III C)")
        gam = _gamma_dec(v0, len2)
        p0 = m * gam
        for vec in G.orbit(gid):
            px = m * gam * v0 * vec[0]
            py = m * gam * v0 * vec[1]
            pz = m * gam * v0 * vec[2]
            for r, nm in enumerate(names):
                A[r][k] += _phi_dec(nm, p0, px, py, pz)
    return A, list(cache.b)


def weights_dec(group_ids, mbar, v0, cache=None):
    """Group weights w_k (decimal) solving Eq. 52 for the given v0."""
    A, b = system_dec(group_ids, mbar, v0, cache)
    return _solve_dec(A, b)


def weights(group_ids, mbar, v0, cache=None):
    """Group weights w_k rounded to FP64."""
    return np.array([float(w) for w in weights_dec(group_ids, mbar, v0, cache)])


def positive_window(group_ids, mbar, v_lo, v_hi, samples=4000, cache=None):
    """All maximal v0 intervals inside (v_lo, v_hi) where every w_k > 0
    (Sec. III D), located on a uniform scan and refined by bisection on the
    weight that changes sign; returns a list of (lo, hi) floats."""
    if cache is None or cache.order != order_of(group_ids):
        cache = MomentCache(mbar, order_of(group_ids))

    def minw(v):
        return min(weights_dec(group_ids, mbar, Decimal(repr(float(v))), cache))

    xs = np.linspace(v_lo, v_hi, samples)
    pos = [minw(float(v)) > 0 for v in xs]
    out = []
    i = 0
    while i < len(xs):
        if pos[i]:
            j = i
            while j + 1 < len(xs) and pos[j + 1]:
                j += 1
            lo = _bisect_edge(minw, xs[i - 1], xs[i]) if i > 0 else xs[i]
            hi = _bisect_edge(minw, xs[j + 1], xs[j]) if j + 1 < len(xs) else xs[j]
            out.append((lo, hi))
            i = j + 1
        else:
            i += 1
    return out


def _bisect_edge(minw, bad, good, iters=60):
    for _ in range(iters):
        mid = 0.5 * (bad + good)
        if minw(mid) > 0:
            good = mid
        else:
            bad = mid
    return 0.5 * (bad + good)


def zero_of_weight(group_ids, mbar, k, lo, hi, iters=200, cache=None):
    """v0 in (lo, hi) where the weight of the k-th listed group vanishes, by
    decimal bisection (the pruned quadratures of Sec. III D)."""
    if cache is None or cache.order != order_of(group_ids):
        cache = MomentCache(mbar, order_of(group_ids))
    lo = S._dec(lo)
    hi = S._dec(hi)
    flo = weights_dec(group_ids, mbar, lo, cache)[k]
    for _ in range(iters):
        mid = (lo + hi) / 2
        fm = weights_dec(group_ids, mbar, mid, cache)[k]
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return (lo + hi) / 2


class Stencil:
    """A stencil at (mbar, v0): per-population momenta and weights, unfolded
    (3D) or folded onto the xy plane.  Six groups give a second-order
    stencil, eleven a third-order one (``order``).

    Folding (2D lattices): the populations (n_x, n_y, +n_z) and (n_x, n_y, -n_z)
    of one group stream identically on an Nx x Ny lattice (Nz = 1) and stay
    equal while U^z = 0, so each pair is merged into one population of weight
    2 w_k that keeps p_z^2 (needed by the z-even polynomials).  The 2D lattice
    of the paper is a 1 x 800 x 800 lattice of the 3D model (Sec. IV), which
    this reproduces exactly.
    """

    def __init__(self, group_ids, mbar, v0, w=None):
        self.group_ids = list(group_ids)
        self.order = order_of(self.group_ids)
        self.mbar = float(mbar)
        self.v0 = float(v0)
        self.w_group = np.asarray(w if w is not None else weights(group_ids, mbar, v0), dtype=np.float64)
        rows = []
        for k, gid in enumerate(self.group_ids):
            len2 = G.length2(gid)
            gam = 1.0 / np.sqrt(1.0 - self.v0 ** 2 * len2)
            for vec in G.orbit(gid):
                rows.append((k, gid, vec, gam))
        self._rows = rows
        self.Q3 = len(rows)

    def populations3d(self):
        """(w, p[Q,4] = (p0, px, py, pz), d[Q,3] integer displacements, group index)."""
        w, p, d, gi = [], [], [], []
        for k, gid, vec, gam in self._rows:
            w.append(self.w_group[k])
            p.append([self.mbar * gam, self.mbar * gam * self.v0 * vec[0],
                      self.mbar * gam * self.v0 * vec[1], self.mbar * gam * self.v0 * vec[2]])
            d.append(vec)
            gi.append(k)
        return np.array(w), np.array(p), np.array(d, dtype=np.int64), np.array(gi)

    def population_vectors(self, two_d):
        """(group index, n_x, n_y, n_z or |n_z|, multiplicity) per population,
        in the order of ``populations2d`` (two_d) or ``populations3d``."""
        if not two_d:
            return [(k, vec[0], vec[1], vec[2], 1) for k, gid, vec, gam in self._rows]
        seen = {}
        order = []
        for k, gid, vec, gam in self._rows:
            key = (k, vec[0], vec[1], abs(vec[2]))
            if key not in seen:
                seen[key] = 0
                order.append(key)
            seen[key] += 1
        return [key + (seen[key],) for key in order]

    def populations2d(self):
        """Folded populations: (w, p[Q,4] with p[:,3] = |p_z|, d[Q,2], group index, multiplicity)."""
        seen = {}
        order = []
        for k, gid, vec, gam in self._rows:
            key = (k, vec[0], vec[1], abs(vec[2]))
            if key not in seen:
                seen[key] = [k, gid, vec, gam, 0]
                order.append(key)
            seen[key][4] += 1
        w, p, d, gi, mult = [], [], [], [], []
        for key in order:
            k, gid, vec, gam, cnt = seen[key]
            w.append(self.w_group[k] * cnt)
            p.append([self.mbar * gam, self.mbar * gam * self.v0 * vec[0],
                      self.mbar * gam * self.v0 * vec[1], self.mbar * gam * self.v0 * abs(vec[2])])
            d.append((vec[0], vec[1]))
            gi.append(k)
            mult.append(cnt)
        return np.array(w), np.array(p), np.array(d, dtype=np.int64), np.array(gi), np.array(mult)
