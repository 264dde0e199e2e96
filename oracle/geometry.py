"""Cut cells of a box minus a union of ellipses (Sec. 3, Alg. 1).

For a level of grid size h the box is divided into N x N control volumes
C_i = (i h, (i+1) h) (Eq. 3.1); the cut cell is C_i intersected with the
domain (Sec. 3.1).  Each cut cell is described by the pieces of its boundary:
straight pieces of its four faces that lie in the domain, and arcs of hole
boundaries that lie in the cell.  Pieces are oriented with the cut cell on
their left, so Green's theorem turns every area integral into a boundary
integral (Sec. 4.2, the quadrature paragraph):

    integral over C of X^p Y^q dA = contour integral of X^(p+1) Y^q / (p+1) dY

in the scaled coordinates X = (x - p_x)/h, Y = (y - p_y)/h about the centre p
of the control volume.  Straight pieces are integrated exactly by 6-point
Gauss-Legendre; arcs by composite 8-point Gauss-Legendre in the angle, with
sub-arcs no longer than 0.2 rad.

The merging step of Alg. 1 (cells of volume fraction below epsilon) is
applied with the reading listed in the design notes: cells are visited once
in row-major order (y index outer), the volume is the current one, a merge
target is a present cell reachable through a shared face piece of positive
length, the argmin ties go to the first neighbour in the order -x, +x, -y,
+y.  The step of Alg. 1 for cells with several connected components comes
first: such a cell keeps its largest component, and every other component
joins the face neighbour (through one of its own face pieces, in the order
-x, +x, -y, +y, near-ties to the first) whose volume with it comes closest
to h^2 (a reading: the paper does not say where the extra components go).  A cell of one component may also hold a whole hole
(an inner loop, counted in its moments); a cell of several components that
also holds an inner loop, or of none, is reported as unresolved.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np

from workloads import Domain, Ellipse, Flower, OutsideRect

EMPTY, REGULAR, IRREGULAR = 0, 1, 2

# Monomials of total degree <= 4 in the order used everywhere in the oracle:
# by total degree, then by the power of Y.
BASIS: List[Tuple[int, int]] = [(d - q, q) for d in range(5) for q in range(d + 1)]
NB = len(BASIS)   # 15 = dim Pi_4^2
# Moments up to degree 6 are kept so that <L phi> of every basis function and
# the shift of moments to another centre stay exact.
MOMS: List[Tuple[int, int]] = [(d - q, q) for d in range(7) for q in range(d + 1)]
MIDX: Dict[Tuple[int, int], int] = {pq: k for k, pq in enumerate(MOMS)}

_GL6 = np.polynomial.legendre.leggauss(6)
_GL8 = np.polynomial.legendre.leggauss(8)


class GeometryError(RuntimeError):
    pass


# ---------------------------------------------------------------------------
# Ellipse helpers
# ---------------------------------------------------------------------------
class Curve:
    """Ellipse P(t) = c + R(theta) (r1 cos t, r2 sin t); t increases CCW."""

    def __init__(self, e: Ellipse):
        self.e = e
        self.co = math.cos(e.theta)
        self.si = math.sin(e.theta)

    def point(self, t):
        ct, st = np.cos(t), np.sin(t)
        e = self.e
        return (e.cx + self.co * e.r1 * ct - self.si * e.r2 * st,
                e.cy + self.si * e.r1 * ct + self.co * e.r2 * st)

    def deriv(self, t):
        ct, st = np.cos(t), np.sin(t)
        e = self.e
        return (-self.co * e.r1 * st - self.si * e.r2 * ct,
                -self.si * e.r1 * st + self.co * e.r2 * ct)

    def level(self, x, y):
        e = self.e
        dx = np.asarray(x) - e.cx
        dy = np.asarray(y) - e.cy
        xp = self.co * dx + self.si * dy
        yp = -self.si * dx + self.co * dy
        return (xp / e.r1) ** 2 + (yp / e.r2) ** 2 - 1.0

    def _solve_trig(self, A, B, C):
        """t in [0, 2pi) with A cos t + B sin t = C."""
        R = math.hypot(A, B)
        if abs(C) >= R:
            return []
        phi = math.atan2(B, A)
        d = math.acos(C / R)
        return [(phi + d) % (2 * math.pi), (phi - d) % (2 * math.pi)]

    def cross_x(self, X):
        e = self.e
        return self._solve_trig(self.co * e.r1, -self.si * e.r2, X - e.cx)

    def cross_y(self, Y):
        e = self.e
        return self._solve_trig(self.si * e.r1, self.co * e.r2, Y - e.cy)

    def bbox(self):
        e = self.e
        hx = math.hypot(e.r1 * self.co, e.r2 * self.si)
        hy = math.hypot(e.r1 * self.si, e.r2 * self.co)
        return e.cx - hx, e.cx + hx, e.cy - hy, e.cy + hy


class FlowerCurve:
    """Polar curve P(t) = c + r(t) (cos t, sin t), r(t) = r0 + amp cos(k t)
    (Sec. 6.2); t increases CCW.  Its crossings with a grid line are found on
    the arcs between consecutive extrema of the curve's coordinate (taken
    cyclically), where the coordinate is monotone: one crossing at most per
    arc, refined by bisection.  A line that meets the curve only at an
    extremum of the coordinate touches it without crossing, and gives no
    crossing (the flower's tips and valleys lie on grid lines of the paper's
    grids)."""

    NS = 4096          # samples of t for the extrema of each coordinate
    TOL = 1e-13        # a coordinate this close to a line at an extremum touches it

    def __init__(self, e: Flower):
        self.e = e
        self._ext = {0: self._extrema(0), 1: self._extrema(1)}

    def r(self, t):
        return self.e.r0 + self.e.amp * np.cos(self.e.k * t)

    def point(self, t):
        rr = self.r(t)
        return self.e.cx + rr * np.cos(t), self.e.cy + rr * np.sin(t)

    def deriv(self, t):
        rr = self.r(t)
        dr = -self.e.amp * self.e.k * np.sin(self.e.k * t)
        return dr * np.cos(t) - rr * np.sin(t), dr * np.sin(t) + rr * np.cos(t)

    def level(self, x, y):
        dx = np.asarray(x) - self.e.cx
        dy = np.asarray(y) - self.e.cy
        return np.hypot(dx, dy) - self.r(np.arctan2(dy, dx))

    @staticmethod
    def _bisect(fn, a, b):
        fa = fn(a)
        for _ in range(200):
            m = 0.5 * (a + b)
            fm = fn(m)
            if fm == 0.0 or b - a < 1e-15:
                return m
            if (fm < 0) == (fa < 0):
                a, fa = m, fm
            else:
                b = m
        return 0.5 * (a + b)

    def _extrema(self, axis):
        """Parameters in [0, 2 pi) where the coordinate `axis` is extremal (the
        sign changes of its derivative on NS samples, refined by bisection)."""
        dco = lambda s: float(self.deriv(s)[axis])
        t = [2 * math.pi * k / self.NS for k in range(self.NS + 1)]
        d = [dco(s) for s in t]
        out = []
        for k in range(self.NS):
            if d[k] == 0.0:
                out.append(t[k])
            elif d[k] * d[k + 1] < 0.0:
                out.append(self._bisect(dco, t[k], t[k + 1]))
        return out

    def _cross(self, axis, X):
        ext = self._ext[axis]
        f = lambda s: float(self.point(s)[axis]) - X
        out = []
        m = len(ext)
        for q in range(m):
            a = ext[q]
            b = ext[q + 1] if q + 1 < m else ext[0] + 2 * math.pi
            fa, fb = f(a), f(b)
            if abs(fa) <= self.TOL or abs(fb) <= self.TOL or fa * fb > 0.0:
                continue
            t = math.fmod(self._bisect(f, a, b), 2 * math.pi)
            out.append(0.0 if t < 0.0 or t >= 2 * math.pi else t)
        return sorted(set(out))

    def cross_x(self, X):
        return self._cross(0, X)

    def cross_y(self, Y):
        return self._cross(1, Y)

    def bbox(self):
        e = self.e
        R = e.r0 + e.amp
        return e.cx - R, e.cx + R, e.cy - R, e.cy + R


class RectCurve:
    """The boundary of the hole outside a rectangle (workloads.OutsideRect):
    the rectangle's sides, with the parameter t increasing clockwise around
    the rectangle (each side a quarter of [0, 2 pi)), so that, as for the
    other holes, the domain lies to the left of the curve followed from high
    to low t.  The corners are kinks: the arcs are split there
    (breakpoints()).  A grid line through a corner crosses there when the two
    sides at the corner lie on its two sides, and touches it otherwise."""

    TOL = 1e-13

    def __init__(self, e: OutsideRect):
        self.e = e
        c, s = math.cos(e.theta), math.sin(e.theta)
        v = [(e.cx, e.cy), (e.cx + e.w * c, e.cy + e.w * s),
             (e.cx + e.w * c - e.hgt * s, e.cy + e.w * s + e.hgt * c), (e.cx - e.hgt * s, e.cy + e.hgt * c)]
        self.ccw = v                            # counter-clockwise corners
        self.cw = [v[0], v[3], v[2], v[1]]      # the order of increasing t

    def point(self, t):
        t = np.asarray(t, dtype=np.float64)
        tm = np.mod(t, 2 * math.pi)
        k = np.minimum((tm // (math.pi / 2)).astype(int), 3)
        tau = (tm - k * (math.pi / 2)) / (math.pi / 2)
        W = np.array(self.cw + [self.cw[0]])
        x = W[k, 0] + tau * (W[k + 1, 0] - W[k, 0])
        y = W[k, 1] + tau * (W[k + 1, 1] - W[k, 1])
        return x, y

    def deriv(self, t):
        t = np.asarray(t, dtype=np.float64)
        tm = np.mod(t, 2 * math.pi)
        k = np.minimum((tm // (math.pi / 2)).astype(int), 3)
        W = np.array(self.cw + [self.cw[0]])
        return (W[k + 1, 0] - W[k, 0]) / (math.pi / 2), (W[k + 1, 1] - W[k, 1]) / (math.pi / 2)

    def level(self, x, y):
        """The distance inside the rectangle to its nearest side line (the
        smallest inward-normal distance): positive inside the rectangle,
        negative in the hole."""
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = None
        for i in range(4):
            (ax, ay), (bx, by) = self.ccw[i], self.ccw[(i + 1) % 4]
            L = math.hypot(bx - ax, by - ay)
            d = (-(by - ay) * (x - ax) + (bx - ax) * (y - ay)) / L
            out = d if out is None else np.minimum(out, d)
        return out

    def breakpoints(self):
        return [k * (math.pi / 2) for k in range(4)]

    def _cross(self, axis, X):
        W = self.cw
        out = []
        for k in range(4):
            f0 = W[k][axis] - X
            fp = W[(k - 1) % 4][axis] - X
            f1 = W[(k + 1) % 4][axis] - X
            if abs(f0) <= self.TOL:
                if fp * f1 < 0.0 and abs(fp) > self.TOL and abs(f1) > self.TOL:
                    out.append(k * (math.pi / 2))
                continue
            if abs(f1) <= self.TOL or f0 * f1 > 0.0:
                continue
            out.append(k * (math.pi / 2) + (math.pi / 2) * f0 / (f0 - f1))
        return sorted(out)

    def cross_x(self, X):
        return self._cross(0, X)

    def cross_y(self, Y):
        return self._cross(1, Y)

    def bbox(self):
        xs = [p[0] for p in self.ccw]
        ys = [p[1] for p in self.ccw]
        return min(xs), max(xs), min(ys), max(ys)


def make_curve(e):
    """The oracle's curve for a hole of the workload."""
    if isinstance(e, Flower):
        return FlowerCurve(e)
    if isinstance(e, OutsideRect):
        return RectCurve(e)
    return Curve(e)


def hole_halfwidth(e) -> float:
    """Half the smallest width of a hole: the smaller semi-axis of an ellipse,
    the smallest radius r0 - amp of a flower."""
    if isinstance(e, OutsideRect):
        return math.inf          # the hole is the outside: no coarse-level width limit
    return e.r0 - e.amp if isinstance(e, Flower) else min(e.r1, e.r2)


def _curve_crossings(ci: Curve, cj: Curve) -> List[float]:
    """Parameters t of curve i where it crosses curve j (sign changes of
    the level function of j along i, refined by bisection)."""
    n = 4096
    t = np.linspace(0.0, 2 * math.pi, n + 1)
    x, y = ci.point(t)
    f = cj.level(x, y)
    out = []
    for k in range(n):
        if f[k] == 0.0:
            out.append(float(t[k]))
        elif f[k] * f[k + 1] < 0.0:
            a, b = float(t[k]), float(t[k + 1])
            fa = float(f[k])
            for _ in range(200):
                m = 0.5 * (a + b)
                fm = float(cj.level(*ci.point(m)))
                if fm == 0.0 or b - a < 1e-16:
                    a = b = m
                    break
                if (fm < 0) == (fa < 0):
                    a, fa = m, fm
                else:
                    b = m
            out.append(0.5 * (a + b))
    return out


# ---------------------------------------------------------------------------
# Boundary pieces and their integrals
# ---------------------------------------------------------------------------
@dataclass
class Piece:
    kind: str                 # 'seg' or 'arc'
    p0: Tuple[float, float]   # start point
    p1: Tuple[float, float]   # end point
    curve: int = -1           # ellipse index for arcs
    ta: float = 0.0           # arc start parameter
    tb: float = 0.0           # arc end parameter (tb < ta: clockwise)
    bc: int = -1              # boundary id for pieces on the domain boundary
    face: int = -1            # 0..3 = bottom, right, top, left face of the cell


def _nodes(piece: Piece, curves: List[Curve]):
    """Quadrature nodes along a piece: x, y, dx/ds-weight, dy-weight, |ds|."""
    if piece.kind == 'seg':
        g, w = _GL6
        tau = 0.5 * (g + 1.0)
        wt = 0.5 * w
        (xa, ya), (xb, yb) = piece.p0, piece.p1
        x = xa + tau * (xb - xa)
        y = ya + tau * (yb - ya)
        dx = np.full_like(tau, xb - xa) * wt
        dy = np.full_like(tau, yb - ya) * wt
        return x, y, dx, dy
    c = curves[piece.curve]
    ta, tb = piece.ta, piece.tb
    nsub = max(1, int(math.ceil(abs(tb - ta) / 0.2)))
    g, w = _GL8
    xs, ys, dxs, dys = [], [], [], []
    for k in range(nsub):
        s0 = ta + (tb - ta) * k / nsub
        s1 = ta + (tb - ta) * (k + 1) / nsub
        t = 0.5 * (s0 + s1) + 0.5 * (s1 - s0) * g
        wt = 0.5 * (s1 - s0) * w
        x, y = c.point(t)
        dxt, dyt = c.deriv(t)
        xs.append(x)
        ys.append(y)
        dxs.append(dxt * wt)
        dys.append(dyt * wt)
    return (np.concatenate(xs), np.concatenate(ys), np.concatenate(dxs),
            np.concatenate(dys))


def piece_moments(piece: Piece, curves: List[Curve], px: float, py: float,
                  h: float) -> np.ndarray:
    """Green's-theorem contribution of one piece to the scaled moments
    integral X^p Y^q dX dY for every (p, q) in MOMS."""
    x, y, dx, dy = _nodes(piece, curves)
    X = (x - px) / h
    Y = (y - py) / h
    dY = dy / h
    out = np.zeros(len(MOMS))
    for k, (p, q) in enumerate(MOMS):
        out[k] = np.sum(X ** (p + 1) * Y ** q * dY) / (p + 1)
    return out


def shift_moments(m: np.ndarray, dx: float, dy: float) -> np.ndarray:
    """Moments about centre p re-expressed about centre p - (dx, dy) h,
    i.e. for X' = X + dx, Y' = Y + dy (binomial expansion)."""
    out = np.zeros_like(m)
    for k, (p, q) in enumerate(MOMS):
        s = 0.0
        for a in range(p + 1):
            for b in range(q + 1):
                s += (math.comb(p, a) * math.comb(q, b) * dx ** (p - a)
                      * dy ** (q - b) * m[MIDX[(a, b)]])
        out[k] = s
    return out


def regular_moments() -> np.ndarray:
    """Scaled moments of a full unit cell about its centre."""
    def m1(p):
        return 0.0 if p % 2 else 2.0 * 0.5 ** (p + 1) / (p + 1)
    return np.array([m1(p) * m1(q) for (p, q) in MOMS])


# ---------------------------------------------------------------------------
# A level of cut cells
# ---------------------------------------------------------------------------
@dataclass
class CutCell:
    pieces: List[Piece]
    mom: np.ndarray                # scaled moments about the own centre
    faces: List[bool]              # face k (bottom,right,top,left) has a cut face in the domain
    bnodes: list = field(default_factory=list)  # boundary quadrature: (x,y,nx,ny,w,bc)


@dataclass
class Level:
    dom: Domain
    n: int
    h: float
    eps: float
    present: np.ndarray            # [n, n] bool, non-empty after merging
    ctype: np.ndarray              # [n, n] EMPTY / REGULAR / IRREGULAR
    vol: np.ndarray                # [n, n] physical volume
    owner: np.ndarray              # [n, n] flat index of the cell holding this control volume, -1 if none
    cut: Dict[int, CutCell]        # flat index -> data of every non-regular present cell
    resolved: bool = True
    reason: str = ""

    def center(self, k):
        j, i = divmod(k, self.n)
        return (self.dom.x0 + (i + 0.5) * self.h, self.dom.y0 + (j + 0.5) * self.h)

    def moments(self, k) -> np.ndarray:
        """Scaled moments of present cell k about its own control-volume centre."""
        if k in self.cut:
            return self.cut[k].mom
        return regular_moments()


def _bc_of_curve(dom: Domain, e_idx: int) -> int:
    """Boundary ids: 0..3 = box sides S, E, N, W; 4 + k = hole k."""
    return 4 + e_idx


def build_level(dom: Domain, n: int, eps: float) -> Level:
    """Cut the box into n x n cells, clip against the holes, merge (Alg. 1)."""
    h = (dom.x1 - dom.x0) / n
    if abs((dom.y1 - dom.y0) - h * n) > 1e-12 * max(1.0, dom.y1 - dom.y0):
        raise GeometryError("the box must be square with square cells")
    curves = [make_curve(e) for e in dom.holes]
    x0, y0 = dom.x0, dom.y0

    def outside_all(x, y, skip=-1):
        for k, c in enumerate(curves):
            if k != skip and c.level(x, y) <= 0.0:
                return False
        return True

    # --- breakpoints on every ellipse: grid lines and other ellipses -------
    arcs_by_cell: Dict[int, List[Piece]] = {}
    xcross: Dict[int, List[float]] = {}   # vertical line i -> y of crossings
    ycross: Dict[int, List[float]] = {}   # horizontal line j -> x of crossings
    for ei, c in enumerate(curves):
        bx0, bx1, by0, by1 = c.bbox()
        ts = []
        for i in range(max(0, int(math.floor((bx0 - x0) / h))),
                       min(n, int(math.ceil((bx1 - x0) / h))) + 1):
            X = x0 + i * h
            for t in c.cross_x(X):
                ts.append(t)
                xcross.setdefault(i, []).append(float(c.point(t)[1]))
        for j in range(max(0, int(math.floor((by0 - y0) / h))),
                       min(n, int(math.ceil((by1 - y0) / h))) + 1):
            Y = y0 + j * h
            for t in c.cross_y(Y):
                ts.append(t)
                ycross.setdefault(j, []).append(float(c.point(t)[0]))
        for ej, c2 in enumerate(curves):
            if ej != ei:
                ts.extend(_curve_crossings(c, c2))
        if hasattr(c, "breakpoints"):
            ts.extend(c.breakpoints())
        ts = sorted(set(ts))
        if not ts:
            segs = [(2 * math.pi, 0.0)]
        else:
            segs = []
            for k in range(len(ts)):
                a = ts[k]
                b = ts[k + 1] if k + 1 < len(ts) else ts[0] + 2 * math.pi
                segs.append((b, a))       # clockwise: from b down to a
        for (tb_hi, ta_lo) in segs:
            tm = 0.5 * (tb_hi + ta_lo)
            xm, ym = c.point(tm)
            if not outside_all(xm, ym, skip=ei):
                continue
            ii = int(math.floor((xm - x0) / h))
            jj = int(math.floor((ym - y0) / h))
            if not (0 <= ii < n and 0 <= jj < n):
                raise GeometryError("a hole leaves the box")
            pa = c.point(tb_hi)
            pb = c.point(ta_lo)
            arcs_by_cell.setdefault(jj * n + ii, []).append(
                Piece('arc', (float(pa[0]), float(pa[1])), (float(pb[0]), float(pb[1])),
                      curve=ei, ta=tb_hi, tb=ta_lo, bc=_bc_of_curve(dom, ei)))

    ctype = np.zeros((n, n), dtype=np.int8)
    vol = np.zeros((n, n))
    cut: Dict[int, CutCell] = {}
    resolved, reason = True, ""

    # cells without arcs: regular or empty by the centre test
    xc = x0 + (np.arange(n) + 0.5) * h
    yc = y0 + (np.arange(n) + 0.5) * h
    XC, YC = np.meshgrid(xc, yc)
    inside_any = np.zeros((n, n), dtype=bool)
    for c in curves:
        inside_any |= c.level(XC, YC) <= 0.0
    ctype[~inside_any] = REGULAR
    vol[~inside_any] = h * h

    orphans = []   # (cell, pieces) of the components a cell does not keep
    for k, arcs in sorted(arcs_by_cell.items()):
        j, i = divmod(k, n)
        xl, xr = x0 + i * h, x0 + (i + 1) * h
        yb, yt = y0 + j * h, y0 + (j + 1) * h
        pieces = list(arcs)
        faces = [False, False, False, False]
        # faces, counter-clockwise: bottom, right, top, left
        edges = [((xl, yb), (xr, yb), ycross.get(j, []), 0),
                 ((xr, yb), (xr, yt), xcross.get(i + 1, []), 1),
                 ((xr, yt), (xl, yt), ycross.get(j + 1, []), 0),
                 ((xl, yt), (xl, yb), xcross.get(i, []), 1)]
        for f, (pa, pb, cr, axis) in enumerate(edges):
            # parameter along the edge is x (axis 0, horizontal) or y (vertical)
            coord_a = pa[0] if axis == 0 else pa[1]
            coord_b = pb[0] if axis == 0 else pb[1]
            cmin, cmax = min(coord_a, coord_b), max(coord_a, coord_b)
            cuts = sorted(v for v in cr if cmin < v < cmax)
            pts = [cmin] + cuts + [cmax]
            if coord_a > coord_b:
                pts = pts[::-1]
            for s in range(len(pts) - 1):
                ca, cb = pts[s], pts[s + 1]
                if axis == 0:
                    qa, qb = (ca, pa[1]), (cb, pa[1])
                else:
                    qa, qb = (pa[0], ca), (pa[0], cb)
                mx, my = 0.5 * (qa[0] + qb[0]), 0.5 * (qa[1] + qb[1])
                if outside_all(mx, my):
                    bc = -1
                    if f == 0 and j == 0:
                        bc = 0
                    elif f == 1 and i == n - 1:
                        bc = 1
                    elif f == 2 and j == n - 1:
                        bc = 2
                    elif f == 3 and i == 0:
                        bc = 3
                    pieces.append(Piece('seg', qa, qb, bc=bc, face=f))
                    faces[f] = True
        # chain pieces into loops: the connected components
        loops = _loops(pieces, h, curves, xl + 0.5 * h, yb + 0.5 * h)
        nloops_out = sum(1 for _, a in loops if a > 0)
        nloops_in = len(loops) - nloops_out
        if nloops_out >= 2 and nloops_in == 0:
            # Alg. 1, cells of several components: keep the largest here, the
            # others join a face neighbour below
            big = max(range(len(loops)), key=lambda q: (loops[q][1], -q))
            for q, (idx, _) in enumerate(loops):
                if q != big:
                    orphans.append((k, [pieces[t] for t in idx]))
            pieces = [pieces[t] for t in loops[big][0]]
            faces = [False, False, False, False]
            for pc in pieces:
                if pc.kind == 'seg':
                    faces[pc.face] = True
        elif nloops_out != 1:
            resolved = False
            reason = f"cell ({i},{j}) has {nloops_out} components"
        mom = np.zeros(len(MOMS))
        for p in pieces:
            mom += piece_moments(p, curves, xl + 0.5 * h, yb + 0.5 * h, h)
        if mom[0] <= 0.0:
            ctype[j, i] = EMPTY
            vol[j, i] = 0.0
            continue
        ctype[j, i] = IRREGULAR
        vol[j, i] = mom[0] * h * h
        cc = CutCell(pieces, mom, faces)
        cc.bnodes = _boundary_nodes(pieces, curves)
        cut[k] = cc

    present = ctype != EMPTY
    owner = np.where(present.ravel(), np.arange(n * n), -1).reshape(n, n)
    lev = Level(dom, n, h, eps, present, ctype, vol, owner, cut, resolved, reason)
    for k, pcs in orphans:
        if not _attach_component(lev, k, pcs, curves):
            lev.resolved = False
            lev.reason = f"a component of cell {divmod(k, n)[::-1]} has no neighbour"
    _merge_small(lev)
    return lev


def _attach_component(lev: Level, k: int, pcs: List[Piece], curves) -> bool:
    """Alg. 1, the step for cells of several components: the component of
    cell k bounded by pcs joins the face neighbour C_j (one across a face
    piece of the component, in the order -x, +x, -y, +y) minimising
    |vol_j + vol_component - h^2| (scores within 1e-9 h^2 of the smallest are
    ties, to the first); False if it touches no present neighbour."""
    n, h = lev.n, lev.h
    h2 = h * h
    j, i = divmod(k, n)
    px, py = lev.center(k)
    mk = np.zeros(len(MOMS))
    for p in pcs:
        mk += piece_moments(p, curves, px, py, h)
    vk = mk[0] * h2
    faces = {p.face for p in pcs if p.kind == 'seg'}
    nbrs = []
    for f, (di, dj) in ((3, (-1, 0)), (1, (1, 0)), (0, (0, -1)), (2, (0, 1))):
        ii, jj = i + di, j + dj
        if f not in faces or not (0 <= ii < n and 0 <= jj < n) or not lev.present[jj, ii]:
            continue
        nbrs.append(jj * n + ii)
    if not nbrs:
        return False
    score = [abs(lev.vol.flat[t] + vk - h2) for t in nbrs]
    smin = min(score)
    best = next(t for t, sc in zip(nbrs, score) if sc <= smin + 1e-9 * h2)
    bj, bi = divmod(best, n)
    tgt = lev.cut.get(best)
    if tgt is None:
        tgt = CutCell(_full_edges(lev, bi, bj), regular_moments().copy(), [True] * 4)
        tgt.bnodes = _wall_nodes(lev, bi, bj)
        lev.cut[best] = tgt
    tgt.mom = tgt.mom + shift_moments(mk, i - bi, j - bj)
    tgt.pieces = tgt.pieces + list(pcs)
    tgt.bnodes = tgt.bnodes + _boundary_nodes(list(pcs), curves)
    lev.vol[bj, bi] += vk
    lev.ctype[bj, bi] = IRREGULAR
    return True


def _count_loops(pieces: List[Piece], h: float, curves, px, py):
    """Number of outer (positive area) and inner loops formed by the pieces."""
    loops = _loops(pieces, h, curves, px, py)
    n_out = sum(1 for _, a in loops if a > 0)
    return n_out, len(loops) - n_out


def _loops(pieces: List[Piece], h: float, curves, px, py):
    """The closed loops formed by the pieces, each as (piece indices in
    chaining order, scaled area), in the order of their first pieces."""
    tol = 1e-9 * h
    left = list(range(len(pieces)))
    out = []
    while left:
        start = left.pop(0)
        loop = [start]
        cur_end = pieces[start].p1
        first = pieces[start].p0
        guard = 0
        while math.hypot(cur_end[0] - first[0], cur_end[1] - first[1]) > tol:
            nxt = None
            for idx in left:
                q = pieces[idx].p0
                if math.hypot(q[0] - cur_end[0], q[1] - cur_end[1]) <= tol:
                    nxt = idx
                    break
            if nxt is None:
                raise GeometryError("boundary pieces of a cut cell do not close")
            left.remove(nxt)
            loop.append(nxt)
            cur_end = pieces[nxt].p1
            guard += 1
            if guard > 10000:
                raise GeometryError("loop chaining did not terminate")
        area = sum(piece_moments(pieces[k], curves, px, py, h)[0] for k in loop)
        out.append((loop, area))
    return out


def _boundary_nodes(pieces: List[Piece], curves) -> list:
    """Quadrature nodes on the cut boundary B_i: x, y, outward normal, |ds|, bc."""
    out = []
    for p in pieces:
        if p.bc < 0:
            continue
        x, y, dx, dy = _nodes(p, curves)
        ds = np.hypot(dx, dy)
        # the cell lies to the left of the direction of travel, so the outward
        # normal of the domain is the right-hand normal (dy, -dx)/|ds|
        nx = dy / ds
        ny = -dx / ds
        for a in range(len(x)):
            out.append((float(x[a]), float(y[a]), float(nx[a]), float(ny[a]),
                        float(ds[a]), int(p.bc)))
    return out


def _full_edges(lev: Level, i: int, j: int) -> List[Piece]:
    """The four faces of a full cell, counter-clockwise."""
    n, h, d = lev.n, lev.h, lev.dom
    xl, xr = d.x0 + i * h, d.x0 + (i + 1) * h
    yb, yt = d.y0 + j * h, d.y0 + (j + 1) * h
    return [Piece('seg', (xl, yb), (xr, yb), bc=0 if j == 0 else -1, face=0),
            Piece('seg', (xr, yb), (xr, yt), bc=1 if i == n - 1 else -1, face=1),
            Piece('seg', (xr, yt), (xl, yt), bc=2 if j == n - 1 else -1, face=2),
            Piece('seg', (xl, yt), (xl, yb), bc=3 if i == 0 else -1, face=3)]


def _wall_nodes(lev: Level, i: int, j: int) -> list:
    """Boundary nodes of the box-wall faces of a full cell (used when a full
    cell on the wall absorbs a small cell and so becomes irregular)."""
    n, h, d = lev.n, lev.h, lev.dom
    xl, xr = d.x0 + i * h, d.x0 + (i + 1) * h
    yb, yt = d.y0 + j * h, d.y0 + (j + 1) * h
    segs = []
    if j == 0:
        segs.append(Piece('seg', (xl, yb), (xr, yb), bc=0, face=0))
    if i == n - 1:
        segs.append(Piece('seg', (xr, yb), (xr, yt), bc=1, face=1))
    if j == n - 1:
        segs.append(Piece('seg', (xr, yt), (xl, yt), bc=2, face=2))
    if i == 0:
        segs.append(Piece('seg', (xl, yt), (xl, yb), bc=3, face=3))
    return _boundary_nodes(segs, [])


def _merge_small(lev: Level) -> None:
    """Alg. 1, merging step: merge every cell of volume < eps h^2 into the face
    neighbour that brings the merged volume closest to h^2 (near-ties to the
    first neighbour in the order -x, +x, -y, +y)."""
    n, h = lev.n, lev.h
    h2 = h * h

    def find(k):
        while lev.owner.flat[k] != k:
            k = lev.owner.flat[k]
        return k

    for k in range(n * n):
        j, i = divmod(k, n)
        if not lev.present[j, i] or lev.vol[j, i] >= lev.eps * h2:
            continue
        faces = lev.cut[k].faces if k in lev.cut else [True] * 4
        nbrs = []
        for f, (di, dj) in ((3, (-1, 0)), (1, (1, 0)), (0, (0, -1)), (2, (0, 1))):
            ii, jj = i + di, j + dj
            if not faces[f] or not (0 <= ii < n and 0 <= jj < n):
                continue
            if lev.owner[jj, ii] < 0:
                continue
            t = find(jj * n + ii)
            if t != k and t not in nbrs:
                nbrs.append(t)
        if not nbrs:
            raise GeometryError(f"small cell ({i},{j}) has no neighbour to merge into")
        # the neighbour that brings the merged volume closest to h^2; scores
        # within 1e-9 h^2 of the smallest are ties (they differ by rounding
        # only, e.g. the mirror cells on a diagonal of a disk) and go to the
        # first neighbour in the order -x, +x, -y, +y
        score = [abs(lev.vol.flat[t] + lev.vol[j, i] - h2) for t in nbrs]
        smin = min(score)
        best = next(t for t, sc in zip(nbrs, score) if sc <= smin + 1e-9 * h2)
        bj, bi = divmod(best, n)
        # merge: volumes, moments about the target's centre, boundary pieces
        mk = lev.moments(k)
        mt = lev.moments(best)
        merged = mt + shift_moments(mk, i - bi, j - bj)
        src = lev.cut.get(k)
        tgt = lev.cut.get(best)
        if tgt is None:
            tgt = CutCell(_full_edges(lev, bi, bj), mt.copy(), [True] * 4)
            tgt.bnodes = _wall_nodes(lev, bi, bj)
            lev.cut[best] = tgt
        tgt.mom = merged
        if src is not None:
            tgt.pieces = tgt.pieces + src.pieces
            tgt.bnodes = tgt.bnodes + src.bnodes
            del lev.cut[k]
        lev.vol[bj, bi] += lev.vol[j, i]
        lev.vol[j, i] = 0.0
        lev.present[j, i] = False
        lev.ctype[j, i] = EMPTY
        lev.ctype[bj, bi] = IRREGULAR
        lev.owner[j, i] = best
    # compress owner chains
    for k in range(n * n):
        if lev.owner.flat[k] >= 0:
            lev.owner.flat[k] = find(k)
