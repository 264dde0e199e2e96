"""The cut-cell geometric multigrid method (Sec. 5).

  A22LU        LU factorisation of the PLG-PLG block in the curve ordering,
               with the corner blocks of Lemma 5.2 handled as in Def. 5.3:
               A22 = [[B, P], [Q, S]] = [[L_B, 0], [Y, L_S]] [[U_B, X], [0, U_S]]
               (banded LU of B, X = L_B^-1 P, Y = Q U_B^-1, LU of S - Y X),
               all without pivoting.
  smooth       the block smoother T_omega of Def. 5.6: weighted Jacobi on the
               SFV unknowns with the old PLG values (Eq. 5.7), then the exact
               solve L22 U22 u2 = b2 - A21 u1 (Eq. 5.8).  D11 is the constant
               centre weight of the SFV stencil (the reading that reproduces
               Table 2).  A variant outside the paper replaces the Jacobi step
               by multicolour Gauss-Seidel (colours, smoother = "mcgs").
  restrict     Eq. 5.10: the average of the 4 children; the residual of the
               exactly solved cells is 0 after a sweep (Sec. 5.3) and is
               taken as exactly 0.
  interpolate  Eq. 5.11: piecewise-constant injection; a fine cell whose
               parent control volume was merged away reads the cell that
               absorbed it.
  cycle        Alg. 2 (gamma = 1) and the same recursion visited twice per
               level (gamma = 2, a W-cycle built from the same components).
  fmg          Alg. 3.
  two_grid     the two-grid operator of Eq. 5.12 as a linear map.

Everything is FP64 and uses the explicitly assembled level matrices.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

from workloads import Domain
from . import discretize as D
from . import geometry as G

BAND_CAP = 64     # couplings farther apart than this in the curve order go to the corner blocks


class A22LU:
    """Def. 5.3 for the PLG block of one level."""

    def __init__(self, d: D.Disc):
        self.order = np.array(d.plg_order, dtype=np.int64)
        m = self.m = len(self.order)
        if m == 0:
            return
        pos = {int(k): r for r, k in enumerate(self.order)}
        A = d.A
        ent = {}
        for r, k in enumerate(self.order):
            row = A.getrow(int(k))
            for c, v in zip(row.indices, row.data):
                if int(c) in pos:
                    ent[(r, pos[int(c)])] = ent.get((r, pos[int(c)]), 0.0) + v
        near = [abs(r - c) for (r, c) in ent if abs(r - c) <= BAND_CAP]
        p = max(near) if near else 0
        far = [max(r, c) for (r, c) in ent if abs(r - c) > p]
        k = (m - min(far)) if far else 0
        mb = m - k
        self.p, self.k, self.mb = p, k, mb
        # B in band storage: Bd[i, c - i + p] = B[i, c]
        Bd = np.zeros((mb, 2 * p + 1))
        P = np.zeros((mb, k))
        Q = np.zeros((k, mb))
        S = np.zeros((k, k))
        for (r, c), v in ent.items():
            if r < mb and c < mb:
                if abs(r - c) > p:
                    raise RuntimeError("A22 entry outside the band of B")
                Bd[r, c - r + p] = v
            elif r < mb:
                P[r, c - mb] = v
            elif c < mb:
                Q[r - mb, c] = v
            else:
                S[r - mb, c - mb] = v
        # (a) banded LU of B without pivoting; L (unit diagonal) below, U on/above
        for i in range(mb):
            piv = Bd[i, p]
            if piv == 0.0:
                raise ZeroDivisionError("zero pivot in the LU of A22")
            for r in range(i + 1, min(i + p + 1, mb)):
                l = Bd[r, i - r + p] / piv
                if l == 0.0:
                    continue
                Bd[r, i - r + p] = l
                w = min(i + p, mb - 1) - i          # columns i+1 .. i+w
                Bd[r, i + 1 - r + p:i + 1 + w - r + p] -= l * Bd[i, p + 1:p + 1 + w]
        self.Bd = Bd
        # (b) X = L_B^-1 P, (c) Y = Q U_B^-1, (d) LU of S - Y X
        self.X = np.column_stack([self._fwd(P[:, j]) for j in range(k)]) if k else np.zeros((mb, 0))
        self.Y = np.vstack([self._bwd_T(Q[j, :]) for j in range(k)]) if k else np.zeros((0, mb))
        Sp = S - self.Y @ self.X
        for i in range(k):
            if Sp[i, i] == 0.0:
                raise ZeroDivisionError("zero pivot in the LU of the corner block")
            Sp[i + 1:, i] /= Sp[i, i]
            Sp[i + 1:, i + 1:] -= np.outer(Sp[i + 1:, i], Sp[i, i + 1:])
        self.LUS = Sp

    # L_B z = t (unit lower, band p)
    def _fwd(self, t):
        p, Bd, mb = self.p, self.Bd, self.mb
        z = np.array(t, dtype=np.float64)
        for i in range(mb):
            lo = max(0, i - p)
            if i > lo:
                z[i] -= Bd[i, lo - i + p:p] @ z[lo:i]
        return z

    # U_B x = z (upper, band p)
    def _bwd(self, z):
        p, Bd, mb = self.p, self.Bd, self.mb
        x = np.array(z, dtype=np.float64)
        for i in range(mb - 1, -1, -1):
            hi = min(mb - 1, i + p)
            if hi > i:
                x[i] -= Bd[i, p + 1:p + 1 + hi - i] @ x[i + 1:hi + 1]
            x[i] /= Bd[i, p]
        return x

    # y U_B = q, i.e. U_B^T y = q (lower triangular solve with U_B^T)
    def _bwd_T(self, q):
        p, Bd, mb = self.p, self.Bd, self.mb
        y = np.array(q, dtype=np.float64)
        for c in range(mb):
            lo = max(0, c - p)
            if c > lo:
                # column c of U_B above the diagonal: U[r, c] = Bd[r, c - r + p], r in [lo, c)
                rs = np.arange(lo, c)
                y[c] -= Bd[rs, c - rs + p] @ y[lo:c]
            y[c] /= Bd[c, p]
        return y

    def solve(self, t):
        """u2 = U22^-1 L22^-1 t (Eq. 5.8), t in curve order."""
        mb, k = self.mb, self.k
        z1 = self._fwd(t[:mb])
        z2 = t[mb:] - self.Y @ z1
        Sp = self.LUS
        for i in range(k):               # L_S (unit lower)
            z2[i] -= Sp[i, :i] @ z2[:i]
        x2 = z2.copy()
        for i in range(k - 1, -1, -1):   # U_S
            x2[i] = (x2[i] - Sp[i, i + 1:] @ x2[i + 1:]) / Sp[i, i]
        x1 = self._bwd(z1 - self.X @ x2)
        return np.concatenate([x1, x2])


@dataclass
class Hierarchy:
    levels: List[D.Disc]
    lus: List[A22LU]
    bottom: np.ndarray               # dense inverse-free: LU factors via numpy solve
    omega: float = 0.5
    smoother: str = "jacobi"         # "jacobi" (Def. 5.6) or "mcgs" (the multicolour variant)

    @property
    def nl(self):
        return len(self.levels)


def build_hierarchy(dom: Domain, n: int, a: float, b: float, c: float,
                    eps: float = 0.1, min_coarse: int = 4,
                    max_levels: int = 32, omega: float = 0.5,
                    hole_cells: float = 2.0, smoother: str = "jacobi") -> Hierarchy:
    """Eq. 5.9: rediscretise every level h_f 2^l; the coarsest level is the
    smallest N >= min_coarse reached by halving while every level resolves
    the domain: single-component cut cells (Alg. 1 precondition), every hole
    at least hole_cells cells across its smaller semi-axis on the coarse
    levels, and every PLG fit possible."""
    levels = []
    nl = n
    while len(levels) < max_levels:
        h = (dom.x1 - dom.x0) / nl
        if levels and any(G.hole_halfwidth(e) < hole_cells * h for e in dom.holes):
            break
        lev = G.build_level(dom, nl, eps)
        if not lev.resolved:
            if not levels:
                raise G.GeometryError(lev.reason)
            break
        try:
            d = D.discretize(lev, a, b, c)
        except D.FitError:
            if not levels:
                raise
            break
        levels.append(d)
        if nl % 2 or nl // 2 < min_coarse:
            break
        nl //= 2
    lus = [A22LU(d) for d in levels]
    bottom = levels[-1].A.toarray()
    return Hierarchy(levels, lus, bottom, omega, smoother)


def residual(d: D.Disc, u: np.ndarray, b: np.ndarray) -> np.ndarray:
    """r = b - A u (Eq. 4.23)."""
    return (b.ravel() - d.A @ u.ravel()).reshape(u.shape)


def colours(d: D.Disc) -> np.ndarray:
    """Colour classes of the cells for the multicolour Gauss-Seidel variant, so
    that no two SFV cells of one class are coupled.  A row couples to the
    cells its stencil (Eq. 4.7a,b) reaches and, next to a box wall, to the
    four inward cells each ghost value is formed from (Sec. 4.1), up to 3
    cells from the row's own along the wall normal.  With b = 0 the couplings
    are along the axes, up to 3 cells, and the 4 classes (i + j) mod 4
    separate them; with b != 0 they are the 5 x 5 box plus offsets (3, t) and
    (t, 3), |t| <= 2, and the 15 classes (i + 4 j) mod 15 do (the smallest
    such colouring of the form (i + k j) mod m)."""
    n = d.n
    j, i = np.mgrid[0:n, 0:n]
    if d.b == 0.0:
        return (i + j) % 4
    return (i + 4 * j) % 15


def smooth(H: Hierarchy, l: int, u: np.ndarray, b: np.ndarray) -> np.ndarray:
    """One sweep of the block smoother T_omega (Def. 5.6, Eq. 5.7-5.8), or of
    its multicolour variant: the SFV unknowns relaxed colour by colour, each
    class with the latest values of the others (u_i += omega r_i / D), then
    the same exact block solve."""
    d, lu = H.levels[l], H.lus[l]
    blk = np.zeros(d.n * d.n, dtype=bool)
    blk[lu.order] = True
    jac = (d.kind.ravel() == D.SFV) & ~blk
    uf = u.ravel()
    if H.smoother == "mcgs":
        col = colours(d).ravel()
        un = uf.copy()
        for c in range(int(col.max()) + 1):
            m = jac & (col == c)
            r = b.ravel() - d.A @ un
            un[m] = un[m] + H.omega * r[m] / d.diag
    else:
        r = b.ravel() - d.A @ uf
        un = uf.copy()
        un[jac] = uf[jac] + H.omega * r[jac] / d.diag
    if lu.m:
        u1 = un.copy()
        u1[blk] = 0.0
        rows = lu.order
        t = b.ravel()[rows] - d.A[rows] @ u1
        un[rows] = lu.solve(t)
    return un.reshape(u.shape)


def restrict(H: Hierarchy, l: int, r: np.ndarray, zero_plg: bool = True) -> np.ndarray:
    """Eq. 5.10 from level l to level l+1."""
    d = H.levels[l]
    rr = r.copy()
    if zero_plg:
        rr.ravel()[H.lus[l].order] = 0.0
    rr[d.kind == D.EMPTY] = 0.0
    n = d.n
    rc = 0.25 * (rr[0::2, 0::2] + rr[1::2, 0::2] + rr[0::2, 1::2] + rr[1::2, 1::2])
    rc[H.levels[l + 1].kind == D.EMPTY] = 0.0
    return rc


def interpolate(H: Hierarchy, l: int, ec: np.ndarray) -> np.ndarray:
    """Eq. 5.11 from level l+1 to level l."""
    dc = H.levels[l + 1]
    nc = dc.n
    own = dc.lev.owner                        # coarse control volume -> coarse cell
    ext = np.where(own >= 0, ec.ravel()[np.maximum(own, 0)], 0.0)
    e = np.repeat(np.repeat(ext, 2, axis=0), 2, axis=1)
    e[H.levels[l].kind == D.EMPTY] = 0.0
    return e


def bottom_solve(H: Hierarchy, b: np.ndarray) -> np.ndarray:
    return np.linalg.solve(H.bottom, b.ravel()).reshape(b.shape)


def cycle(H: Hierarchy, l: int, u: np.ndarray, b: np.ndarray, nu1: int, nu2: int,
          gamma: int = 1, w_depth: int = 0) -> np.ndarray:
    """Alg. 2 (gamma = 1: V-cycle; gamma = 2: W-cycle).  With w_depth > 0
    only the w_depth finest levels repeat their coarse-grid correction gamma
    times; coarser levels recurse once (a cycle shape outside the paper)."""
    if l == H.nl - 1:
        return bottom_solve(H, b)
    for _ in range(nu1):
        u = smooth(H, l, u, b)
    rc = restrict(H, l, residual(H.levels[l], u, b))
    ec = np.zeros_like(rc)
    g = gamma if (w_depth == 0 or l < w_depth) else 1
    for _ in range(g):
        ec = cycle(H, l + 1, ec, rc, nu1, nu2, gamma, w_depth)
    u = u + interpolate(H, l, ec)
    for _ in range(nu2):
        u = smooth(H, l, u, b)
    return u


def fmg(H: Hierarchy, l: int, r: np.ndarray, nu1: int, nu2: int, gamma: int = 1,
        w_depth: int = 0) -> np.ndarray:
    """Alg. 3: an approximation of (A^h)^-1 r."""
    if l == H.nl - 1:
        return bottom_solve(H, r)
    rc = restrict(H, l, r, zero_plg=False)
    ec = fmg(H, l + 1, rc, nu1, nu2, gamma, w_depth)
    e = interpolate(H, l, ec)
    return cycle(H, l, e, r, nu1, nu2, gamma, w_depth)


@dataclass
class SolveResult:
    u: np.ndarray
    history: List[float] = field(default_factory=list)   # relative residual after each cycle
    iterates: List[np.ndarray] = field(default_factory=list)


def solve(H: Hierarchy, b: np.ndarray, u0: Optional[np.ndarray] = None, tol: float = 1e-10,
          nu1: int = 3, nu2: int = 3, gamma: int = 1, method: str = "cycle",
          max_cycles: int = 100, keep_iterates: bool = False, w_depth: int = 0) -> SolveResult:
    """Repeat cycles (Alg. 2) or the FMG residual iteration (Alg. 3 loop)
    until ||b - A u||_inf / ||b||_inf < tol."""
    d = H.levels[0]
    u = np.zeros_like(b) if u0 is None else u0.copy()
    bn = np.abs(b).max()
    res = SolveResult(u)
    for _ in range(max_cycles):
        if method == "fmg":
            r = residual(d, u, b)
            u = u + fmg(H, 0, r, nu1, nu2, gamma, w_depth)
        else:
            u = cycle(H, 0, u, b, nu1, nu2, gamma, w_depth)
        rel = np.abs(residual(d, u, b)).max() / bn
        res.history.append(float(rel))
        if keep_iterates:
            res.iterates.append(u.copy())
        if rel < tol or not math.isfinite(rel):
            break
    res.u = u
    return res


def two_grid_operator(H: Hierarchy, nu1: int, nu2: int):
    """TG of Eq. 5.12 on level 0 with an exact solve on level 1, as a
    scipy LinearOperator on the vector of all control volumes."""
    from scipy.sparse.linalg import LinearOperator
    import scipy.sparse.linalg as spl
    d0, d1 = H.levels[0], H.levels[1]
    n = d0.n
    zero = np.zeros((n, n))
    A1 = spl.splu(d1.A.tocsc())       # the exact coarse solve of Eq. 5.12, factored once

    def mv(v):
        e = np.asarray(v, dtype=np.float64).reshape(n, n).copy()
        e[d0.kind == D.EMPTY] = 0.0
        for _ in range(nu1):
            e = smooth(H, 0, e, zero)
        rc = restrict(H, 0, -residual(d0, e, zero))        # R A e
        ec = A1.solve(rc.ravel()).reshape(rc.shape)
        e = e - interpolate(H, 0, ec)
        for _ in range(nu2):
            e = smooth(H, 0, e, zero)
        return e.ravel()

    return LinearOperator((n * n, n * n), matvec=mv, dtype=np.float64)
