"""The linear system A u = f - N g of one level (Sec. 4, Eq. 4.20-4.22).

Every non-empty cut cell gets one row.  SFV cells (Def. 4.1) use the
fourth-order finite-volume formulas (Eq. 4.7a,b): the second derivative
(-1, 16, -30, 16, -1)/(12 h^2) along each axis and, for the cross term, the
gradient (1, -8, 0, 8, -1)/(12 h) applied along x and then along y.  Where the
stencil leaves the box it reads ghost cells, filled from the four interior
cells and the wall datum (Sec. 4.1); the ghost terms in the datum move to N.
PLG cells (Sec. 4.2) use coefficients beta from the weighted minimum-norm fit
on a poised lattice of 15 cells plus, for irregular cells, the boundary
average (Eq. 4.11-4.19).

Rows of empty control volumes are identity rows with right-hand side 0, so
level vectors are plain n x n arrays.

The poised-lattice search is cited by the paper but not given in it; the
rule used here is a reading (parity with the paper unpinned), see
`choose_lattice`.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp

from workloads import (BC, DIRICHLET, NEUMANN, ROBIN,
                                               Domain, Separable)
from . import geometry as G
from .ghost import extrapolation_coefficients, ghost_coefficients

EMPTY, SFV, PLG = 0, 1, 2
GRAD = {-2: 1.0, -1: -8.0, 0: 0.0, 1: 8.0, 2: -1.0}          # x 1/(12 h)
LAP = {-2: -1.0, -1: 16.0, 0: -30.0, 1: 16.0, 2: -1.0}      # x 1/(12 h^2)
PLG_RADIUS = 4
PLG_RADIUS_MAX = 6    # larger boxes are searched only when the 9 x 9 box has no lattice
PLG_RADIUS_FAR = 12   # the far search, only when the 13 x 13 box has none
EXT = extrapolation_coefficients()


class FitError(RuntimeError):
    pass


def bc_alpha(bc: BC) -> Tuple[float, float]:
    if bc.kind == DIRICHLET:
        return 1.0, 0.0
    if bc.kind == NEUMANN:
        return 0.0, 1.0
    return bc.alpha1, bc.alpha2


def bc_of_id(dom: Domain, bid: int) -> BC:
    return dom.box_bc[bid] if bid < 4 else dom.hole_bc[bid - 4]


@dataclass
class Disc:
    lev: G.Level
    a: float
    b: float
    c: float
    kind: np.ndarray                  # [n, n] EMPTY / SFV / PLG
    A: sp.csr_matrix                  # n^2 x n^2
    Nmat: sp.csr_matrix               # n^2 x (4 n + len(bd_cells))
    bd_cells: List[int]               # irregular cells carrying a boundary datum, row-major
    plg_order: List[int]              # cells of the exactly solved block, in the order of Def. 5.1
    lattices: Dict[int, List[int]] = field(default_factory=dict)
    betas: Dict[int, np.ndarray] = field(default_factory=dict)

    @property
    def n(self):
        return self.lev.n

    @property
    def h(self):
        return self.lev.h

    @property
    def diag(self) -> float:
        """Centre weight of the SFV stencil, -5 (a + c) / (2 h^2) (Eq. 4.7b)."""
        return -30.0 * (self.a + self.c) / (12.0 * self.h * self.h)


def stencil(a: float, b: float, c: float, h: float) -> Dict[Tuple[int, int], float]:
    """Offsets (di, dj) -> weight of the SFV stencil of L (Eq. 4.7a,b)."""
    w: Dict[Tuple[int, int], float] = {}
    for m, v in LAP.items():
        w[(m, 0)] = w.get((m, 0), 0.0) + a * v / (12 * h * h)
        w[(0, m)] = w.get((0, m), 0.0) + c * v / (12 * h * h)
    if b != 0.0:
        for m1, g1 in GRAD.items():
            for m2, g2 in GRAD.items():
                if g1 != 0.0 and g2 != 0.0:
                    w[(m1, m2)] = w.get((m1, m2), 0.0) + b * g1 * g2 / (144 * h * h)
    return w


def _extendable(lev: G.Level, wall: int, t: int) -> bool:
    """Whether the wall cell of row/column t on wall `wall` (0=S,1=E,2=N,3=W)
    is extendable: its wall face lies on the boundary and the four cells
    along the inward normal are regular (Sec. 4.1, Eq. 4.3)."""
    n = lev.n
    if n < 4:
        return False
    for k in range(4):
        if wall == 0:
            i, j = t, k
        elif wall == 1:
            i, j = n - 1 - k, t
        elif wall == 2:
            i, j = t, n - 1 - k
        else:
            i, j = k, t
        if lev.ctype[j, i] != G.REGULAR:
            return False
    return True


def _ghost_ref(n: int, ii: int, jj: int):
    """For an offset cell outside the box: (wall, t, m) for a ghost beyond
    one wall (m the depth), or ('corner', wx, wy, mx, my) beyond two walls."""
    out_x = ii < 0 or ii >= n
    out_y = jj < 0 or jj >= n
    if out_x and out_y:
        wx, mx = (3, -ii) if ii < 0 else (1, ii - n + 1)
        wy, my = (0, -jj) if jj < 0 else (2, jj - n + 1)
        return ('corner', wx, wy, mx, my)
    if ii >= n:
        return 1, jj, ii - n + 1
    if ii < 0:
        return 3, jj, -ii
    if jj >= n:
        return 2, ii, jj - n + 1
    return 0, ii, -jj


def _ghost_valid(gr, ext, n) -> bool:
    """A normal ghost needs its wall cell extendable; a corner ghost needs
    the five wall cells nearest the corner extendable on both walls."""
    if gr[0] == 'corner':
        _, wx, wy, _, _ = gr
        if n < 5:
            return False
        low_y = wy == 0
        low_x = wx == 3
        for q in range(5):
            if not ext[(wx, q if low_y else n - 1 - q)]:
                return False
            if not ext[(wy, q if low_x else n - 1 - q)]:
                return False
        return True
    return ext[(gr[0], gr[1])]


def _inward_cell(n: int, wall: int, t: int, k: int) -> Tuple[int, int]:
    if wall == 0:
        return t, k
    if wall == 1:
        return n - 1 - k, t
    if wall == 2:
        return t, n - 1 - k
    return k, t


def sample_column(lev: G.Level, ki: int, kj: int) -> np.ndarray:
    """<phi_alpha>_j for the scaled basis about the centre of cell i (Eq. 4.19)."""
    n = lev.n
    ji, ii = divmod(ki, n)
    jj, ij = divmod(kj, n)
    m = G.shift_moments(lev.moments(kj), ij - ii, jj - ji)
    return np.array([m[G.MIDX[al]] / m[0] for al in G.BASIS])


def _L_column(lev: G.Level, ki: int, a: float, b: float, c: float) -> np.ndarray:
    """<L phi_alpha>_i for every basis function (right-hand side of Eq. 4.14)."""
    m = lev.moments(ki)
    avg = lambda p, q: m[G.MIDX[(p, q)]] / m[0]
    h2 = lev.h * lev.h
    out = np.zeros(G.NB)
    for k, (p, q) in enumerate(G.BASIS):
        v = 0.0
        if p >= 2:
            v += a * p * (p - 1) * avg(p - 2, q)
        if p >= 1 and q >= 1:
            v += b * p * q * avg(p - 1, q - 1)
        if q >= 2:
            v += c * q * (q - 1) * avg(p, q - 2)
        out[k] = v / h2
    return out


def _boundary_column(lev: G.Level, ki: int) -> np.ndarray:
    """<<N phi_alpha>>_i over the cut boundary B_i (last column of Eq. 4.15)."""
    cc = lev.cut[ki]
    px, py = lev.center(ki)
    h = lev.h
    num = np.zeros(G.NB)
    wsum = 0.0
    for (x, y, nx, ny, w, bid) in cc.bnodes:
        a1, a2 = bc_alpha(bc_of_id(lev.dom, bid))
        X = (x - px) / h
        Y = (y - py) / h
        for k, (p, q) in enumerate(G.BASIS):
            phi = X ** p * Y ** q
            gx = p * X ** (p - 1) * Y ** q / h if p else 0.0
            gy = q * X ** p * Y ** (q - 1) / h if q else 0.0
            num[k] += w * (a1 * phi + a2 * (gx * nx + gy * ny))
        wsum += w
    return num / wsum


ROW_COUNTS = (5, 4, 3, 2, 1)
CUT_PENALTY = 2      # cost of a cut cell (other than the cell itself) in a lattice


def _best_rows(avail: Dict[int, List[int]], cost: Dict[Tuple[int, int], int], radius: int):
    """Choose 5 distinct lines v and assign them the counts 5,4,3,2,1 so that
    the chosen cells (the c cheapest of each line) minimise the total cost.
    Ties: lexicographically larger count vector (c_-R, ..., c_R).
    Returns (cost, key, {v: c}) or None."""
    vs = list(range(-radius, radius + 1))
    full = (1 << len(ROW_COUNTS)) - 1
    nxt = {full: (0, (), {})}
    for v in reversed(vs):
        cur = {}
        us = avail.get(v, [])
        for mask in range(full + 1):
            opts = []
            if mask in nxt:
                c0, k0, a0 = nxt[mask]
                opts.append((c0, (0,) + k0, a0))
            for bit, cnt in enumerate(ROW_COUNTS):
                if mask & (1 << bit) or len(us) < cnt:
                    continue
                m2 = mask | (1 << bit)
                if m2 not in nxt:
                    continue
                c1, k1, a1 = nxt[m2]
                rc = sum(cost[(u, v)] for u in us[:cnt])
                a = dict(a1)
                a[v] = cnt
                opts.append((c1 + rc, (-cnt,) + k1, a))
            if opts:
                cur[mask] = min(opts, key=lambda o: (o[0], o[1]))
        nxt = cur
    return nxt.get(0)


def choose_lattice(lev: G.Level, ki: int) -> List[int]:
    """Poised lattice of 15 cells for PLG cell ki (reading of Def. 4.3).

    The lattice is made of 5 distinct grid lines (rows, or else columns)
    holding 5, 4, 3, 2 and 1 present cells of the 9 x 9 box centred on the
    cell (11 x 11, then 13 x 13, where the 9 x 9 box holds none, as in thin
    wedges at the kinks of a union of holes, and on to 25 x 25 near the tips
    of the thinnest wedges); such a set is poised in Pi_4 for point values (a line with 5
    distinct points fixes a quartic on it, and the rest recurses on Pi_3),
    and hence for cell averages, which are an invertible map of Pi_4.  A
    cell at offset (u, v) costs u^2 + v^2, plus CUT_PENALTY if it is a cut
    cell other than the cell itself (a cut cell's centroid is off its grid
    point; without the penalty a few lattices ended in a far sliver and gave
    rows with a positive diagonal).  On each line the cheapest cells are
    used (negative u first on a tie); among all such lattices the one of
    least total cost is taken, rows before columns on a tie.
    """
    for radius in range(PLG_RADIUS, PLG_RADIUS_FAR + 1):
        lat = _lattice_in_box(lev, ki, radius)
        if lat is not None:
            return lat
    n = lev.n
    raise FitError(f"no poised lattice for cell {divmod(ki, n)[::-1]}")


def _lattice_in_box(lev: G.Level, ki: int, radius: int):
    best = None
    for orient in (0, 1):             # 0: lines of constant dj; 1: of constant di
        r = _lattice_in_box_orient(lev, ki, radius, orient)
        if r is None:
            continue
        cand = (r[0], orient, r[1])
        if best is None or cand < best[0]:
            best = (cand, r[2])
    return None if best is None else best[1]


def _lattice_in_box_orient(lev: G.Level, ki: int, radius: int, orient: int):
    """The cheapest lattice of the box of this radius on lines of one
    orientation: (cost, tie key, sorted cells), or None."""
    n = lev.n
    j0, i0 = divmod(ki, n)
    avail: Dict[int, List[int]] = {}
    cost: Dict[Tuple[int, int], int] = {}
    for v in range(-radius, radius + 1):
        us = []
        for u in range(-radius, radius + 1):
            di, dj = (u, v) if orient == 0 else (v, u)
            i, j = i0 + di, j0 + dj
            if 0 <= i < n and 0 <= j < n and lev.present[j, i]:
                us.append(u)
                cut = lev.ctype[j, i] != G.REGULAR and (di, dj) != (0, 0)
                cost[(u, v)] = u * u + v * v + (CUT_PENALTY if cut else 0)
        us.sort(key=lambda u: (cost[(u, v)], u))
        avail[v] = us
    r = _best_rows(avail, cost, radius)
    if r is None:
        return None
    cells = []
    for v, cnt in sorted(r[2].items()):
        for u in avail[v][:cnt]:
            di, dj = (u, v) if orient == 0 else (v, u)
            cells.append((j0 + dj) * n + (i0 + di))
    return r[0], r[1], sorted(cells)


def lattice_candidates(lev: G.Level, ki: int) -> List[List[int]]:
    """The alternatives to the chosen lattice (for a row whose own coefficient
    is not negative): the cheapest lattice of
    each box (9 x 9, 11 x 11, 13 x 13) and orientation (rows, then columns),
    in that order."""
    out = []
    for radius in range(PLG_RADIUS, PLG_RADIUS_MAX + 1):
        for orient in (0, 1):
            r = _lattice_in_box_orient(lev, ki, radius, orient)
            if r is not None:
                out.append(r[2])
    return out


def row_diagonal(ki: int, lattice: List[int], beta) -> float:
    """The coefficient of cell ki in its own PLG row (0 if ki is not in its
    lattice)."""
    return float(beta[lattice.index(ki)]) if ki in lattice else 0.0


def fit_beta(lev: G.Level, ki: int, lattice: List[int], a, b, c, with_boundary: bool):
    """beta from Eq. 4.14 (square) or the weighted minimum norm of Eq. 4.17-4.18."""
    n = lev.n
    j0, i0 = divmod(ki, n)
    M = np.column_stack([sample_column(lev, ki, kj) for kj in lattice])
    rhs = _L_column(lev, ki, a, b, c)
    if not with_boundary:
        return np.linalg.solve(M, rhs), None
    M = np.column_stack([M, _boundary_column(lev, ki)])
    w = []
    for kj in lattice:
        jj, ij = divmod(kj, n)
        w.append(max(math.hypot(ij - i0, jj - j0), 0.5))
    w.append(0.5)
    # Eq. 4.17 minimises the W^{-1}-norm of beta under M beta = phi, with
    # W^{-1} = diag(w_k).  Its closed form W M^T (M W M^T)^{-1} phi (Lemma 4.4)
    # is evaluated as beta = W^{1/2} gamma, gamma the minimum 2-norm solution
    # of (M W^{1/2}) gamma = phi, which avoids squaring the condition number.
    sw = 1.0 / np.sqrt(np.array(w))       # diagonal of W^{1/2}
    gamma = np.linalg.lstsq(M * sw[None, :], rhs, rcond=None)[0]
    beta = sw * gamma
    return beta[:-1], beta[-1]


def _curve_order(lev: G.Level, plg: List[int]) -> List[int]:
    """Def. 5.1: order PLG cells by the parameter of the closest boundary
    point, the cells near one curve consecutively.  Curves are the box and
    each group of mutually overlapping holes."""
    dom, n, h = lev.dom, lev.n, lev.h
    curves = [G.make_curve(e) for e in dom.holes]
    # groups of overlapping ellipses
    grp = list(range(len(curves)))

    def root(k):
        while grp[k] != k:
            k = grp[k]
        return k
    ts = np.linspace(0, 2 * math.pi, 2048, endpoint=False)
    pts = [c.point(ts) for c in curves]
    for a_ in range(len(curves)):
        for b_ in range(a_ + 1, len(curves)):
            if np.any(curves[b_].level(*pts[a_]) < 0):
                grp[root(a_)] = root(b_)
    groups = sorted(set(root(k) for k in range(len(curves))))
    gid = {g: r for r, g in enumerate(groups)}
    L = dom.x1 - dom.x0
    keys = []
    for k in plg:
        x, y = lev.center(k)
        # distance to the box and its CCW perimeter parameter
        dists = [y - dom.y0, dom.x1 - x, dom.y1 - y, x - dom.x0]
        side = int(np.argmin(dists))
        sbox = [x - dom.x0, L + y - dom.y0, 2 * L + dom.x1 - x, 3 * L + dom.y1 - y][side]
        best = (dists[side], 0, sbox)
        for ci, c in enumerate(curves):
            px, py = pts[ci]
            d2 = (px - x) ** 2 + (py - y) ** 2
            a_ = int(np.argmin(d2))
            d = math.sqrt(d2[a_])
            if d < best[0]:
                g = gid[root(ci)]
                if len([q for q in range(len(curves)) if root(q) == root(ci)]) == 1:
                    s = ts[a_]
                else:  # a group: polar angle about the mean centre of the group
                    mem = [curves[q].e for q in range(len(curves)) if root(q) == root(ci)]
                    gx = sum(e.cx for e in mem) / len(mem)
                    gy = sum(e.cy for e in mem) / len(mem)
                    s = math.atan2(py[a_] - gy, px[a_] - gx) % (2 * math.pi)
                best = (d, 1 + g, s)
        keys.append((best[1], best[2], k))
    keys.sort()
    return [k for (_, _, k) in keys]


def discretize(lev: G.Level, a: float, b: float, c: float) -> Disc:
    """Assemble A and N for one level (Eq. 4.20)."""
    if b * b - 4 * a * c >= 0:
        raise ValueError("the operator must be elliptic: b^2 < 4ac")
    n, h, dom = lev.n, lev.h, lev.dom
    st = stencil(a, b, c, h)
    ext = {(w, t): _extendable(lev, w, t) for w in range(4) for t in range(n)}
    gc = [ghost_coefficients(bc.kind, bc.alpha1, bc.alpha2, h) for bc in dom.box_bc]
    kind = np.zeros((n, n), dtype=np.int8)
    rowsA, colsA, valsA = [], [], []
    rowsN, colsN, valsN = [], [], []
    # --- classification (Def. 4.1) ---------------------------------------
    for j in range(n):
        for i in range(n):
            if not lev.present[j, i]:
                continue
            ok = lev.ctype[j, i] == G.REGULAR
            if ok:
                for (di, dj) in st:
                    ii, jj = i + di, j + dj
                    if 0 <= ii < n and 0 <= jj < n:
                        if lev.ctype[jj, ii] != G.REGULAR:
                            ok = False
                            break
                    else:
                        if not _ghost_valid(_ghost_ref(n, ii, jj), ext, n):
                            ok = False
                            break
            kind[j, i] = SFV if ok else PLG
    # --- SFV rows ---------------------------------------------------------
    for j in range(n):
        for i in range(n):
            k = j * n + i
            if kind[j, i] != SFV:
                continue
            for (di, dj), w in st.items():
                ii, jj = i + di, j + dj
                if 0 <= ii < n and 0 <= jj < n:
                    rowsA.append(k); colsA.append(jj * n + ii); valsA.append(w)
                    continue
                gr = _ghost_ref(n, ii, jj)
                if gr[0] == 'corner':
                    # Corner ghost: the ghost column of one wall at depth mx,
                    # extrapolated to depth my beyond the other wall from the
                    # five rows nearest the corner, averaged with the same
                    # construction in the other order.
                    _, wx, wy, mx, my = gr
                    low_x, low_y = wx == 3, wy == 0
                    terms = []
                    for q in range(5):
                        terms.append((0.5 * EXT[my - 1][q], wx, q if low_y else n - 1 - q, mx))
                        terms.append((0.5 * EXT[mx - 1][q], wy, q if low_x else n - 1 - q, my))
                else:
                    terms = [(1.0, gr[0], gr[1], gr[2])]
                for (sc, wall, t, m) in terms:
                    coef = gc[wall][m - 1]
                    for q in range(4):
                        ci, cj = _inward_cell(n, wall, t, q)
                        rowsA.append(k); colsA.append(cj * n + ci); valsA.append(sc * w * coef[q])
                    rowsN.append(k); colsN.append(wall * n + t); valsN.append(sc * w * coef[4])
    # --- PLG rows ---------------------------------------------------------
    plg = [k for k in range(n * n) if kind.flat[k] == PLG]
    bd_cells = [k for k in plg if k in lev.cut and lev.cut[k].bnodes]
    bd_index = {k: r for r, k in enumerate(bd_cells)}
    lattices, betas = {}, {}
    for k in plg:
        lat = choose_lattice(lev, k)
        withb = k in bd_index
        beta, beta_b = fit_beta(lev, k, lat, a, b, c, withb)
        if row_diagonal(k, lat, beta) >= 0.0:
            # a row whose own coefficient is not negative takes the first
            # alternative lattice whose fit gives a negative one, if any
            for alt in lattice_candidates(lev, k):
                if alt == lat:
                    continue
                try:
                    beta2, beta_b2 = fit_beta(lev, k, alt, a, b, c, withb)
                except np.linalg.LinAlgError:
                    continue
                if row_diagonal(k, alt, beta2) < 0.0:
                    lat, beta, beta_b = alt, beta2, beta_b2
                    break
        lattices[k] = lat
        betas[k] = beta
        for kj, bv in zip(lat, beta):
            rowsA.append(k); colsA.append(kj); valsA.append(bv)
        if withb:
            rowsN.append(k); colsN.append(4 * n + bd_index[k]); valsN.append(beta_b)
    # --- identity rows for empty control volumes -------------------------
    for k in range(n * n):
        if kind.flat[k] == EMPTY:
            rowsA.append(k); colsA.append(k); valsA.append(1.0)
    A = sp.csr_matrix((valsA, (rowsA, colsA)), shape=(n * n, n * n))
    A.sum_duplicates()
    Nm = sp.csr_matrix((valsN, (rowsN, colsN)), shape=(n * n, 4 * n + len(bd_cells)))
    Nm.sum_duplicates()
    block = plg + corner_block_cells(n, b, kind)
    order = _curve_order(lev, sorted(block)) if block else []
    return Disc(lev, a, b, c, kind, A, Nm, bd_cells, order, lattices, betas)


CORNER_BLOCK = 4


def corner_block_cells(n: int, b: float, kind: np.ndarray) -> List[int]:
    """SFV cells that the block smoother solves exactly together with the PLG
    cells: with a cross term (b != 0), the CORNER_BLOCK x CORNER_BLOCK cells
    at each box corner.  Their rows use the corner ghosts, whose weights on
    interior cells are large; solving them exactly instead of relaxing them
    lowers the two-grid spectral radius (0.43 -> 0.37 for (a,b,c)=(1,0.5,2),
    0.68 -> 0.31 for (1.5,-0.8,1) on the unit square).  The discretisation is
    unchanged; only the split of Def. 5.6 into a Jacobi part and an exactly
    solved part moves."""
    if b == 0.0:
        return []
    out = []
    r = min(CORNER_BLOCK, n)
    for j in range(n):
        for i in range(n):
            if kind[j, i] != SFV:
                continue
            if min(i, n - 1 - i) < r and min(j, n - 1 - j) < r:
                out.append(j * n + i)
    return out


# ---------------------------------------------------------------------------
# Inputs of a manufactured problem on this level (oracle-side quadrature)
# ---------------------------------------------------------------------------
_GL_INNER = np.polynomial.legendre.leggauss(8)


def cell_averages(lev: G.Level, fun) -> np.ndarray:
    """<fun>_i over every present cut cell (Eq. 4.1).

    Full cells: exact averages when `fun` is a separable workload function,
    else a 6 x 6 tensor Gauss rule.  Cut cells: Green's theorem,
    integral of fun dA = contour integral of F dy with
    F(x, y) = integral from p_x to x of fun(s, y) ds, the inner integral by
    8-point Gauss-Legendre; the lower limit p_x is the centre of the control
    volume, which keeps F of order h and avoids cancellation on small cells.
    """
    from workloads import Separable, regular_cell_averages
    n, h = lev.n, lev.h
    if isinstance(fun, Separable):
        out = regular_cell_averages(fun, lev.dom, n)
    else:
        g, w = np.polynomial.legendre.leggauss(6)
        xs = lev.dom.x0 + h * (np.arange(n)[None, :, None, None] + 0.5 + 0.5 * g[None, None, :, None])
        ys = lev.dom.y0 + h * (np.arange(n)[:, None, None, None] + 0.5 + 0.5 * g[None, None, None, :])
        vals = np.broadcast_to(fun(xs, ys), (n, n, len(g), len(g)))
        out = np.einsum('jiab,a,b->ji', vals, 0.5 * w, 0.5 * w)
    out = np.array(out, dtype=np.float64)
    out[~lev.present] = 0.0
    curves = [G.make_curve(e) for e in lev.dom.holes]
    gi, wi = _GL_INNER
    for k, cc in lev.cut.items():
        j, i = divmod(k, n)
        px = lev.dom.x0 + (i + 0.5) * h
        tot = 0.0
        for p in cc.pieces:
            x, y, dx, dy = G._nodes(p, curves)
            half = 0.5 * (x - px)
            s = px + half[:, None] * (1.0 + gi[None, :])
            F = half * np.sum(wi[None, :] * fun(s, y[:, None]), axis=1)
            tot += float(np.sum(F * dy))
        out[j, i] = tot / lev.vol[j, i]
    return out


def boundary_data(disc: Disc, u) -> np.ndarray:
    """g = [4 n wall face averages (S, E, N, W)] + [<<N u>>_i per boundary cell]."""
    from workloads import bc_value, wall_face_data
    lev = disc.lev
    g = [wall_face_data(u, lev.dom, lev.n)]
    tail = np.zeros(len(disc.bd_cells))
    for r, k in enumerate(disc.bd_cells):
        num = 0.0
        wsum = 0.0
        for (x, y, nx, ny, w, bid) in lev.cut[k].bnodes:
            num += w * float(bc_value(u, bc_of_id(lev.dom, bid), x, y, nx, ny))
            wsum += w
        tail[r] = num / wsum
    g.append(tail)
    return np.concatenate(g)


def rhs(disc: Disc, f_avg: np.ndarray, g: np.ndarray) -> np.ndarray:
    """b = f - N g (Eq. 4.20); zero on empty control volumes."""
    b = f_avg.ravel().copy() - disc.Nmat @ g
    b[disc.kind.ravel() == EMPTY] = 0.0
    return b.reshape(disc.n, disc.n)
