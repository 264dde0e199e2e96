"""Seeded synthetic inputs: manufactured solutions, domains and right-hand sides.

This module is shared by the tests, the benchmark, the oracle and the
library's input helper (paper_2601_02975_gb300/inputs.py), and belongs to
none of them.  It holds no arithmetic of the method itself (no discretisation, no geometry
clipping, no cycles): only closed-form functions, their exact derivatives and
their exact averages over axis-aligned rectangles and segments, plus seeded
random domain and right-hand-side generators.

Problem class (Sec. 1, Eq. 1.1-1.2): L u = a u_xx + b u_xy + c u_yy = f on a
box minus a union of elliptic holes, with N u = g on the boundary, where N is
Dirichlet (u), Neumann (du/dn, n the outward normal of the domain) or Robin
(alpha1 u + alpha2 du/dn).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

# ---------------------------------------------------------------------------
# 1-D elementary factors: sin(k x), cos(k x), exp(k x) with exact calculus.
# ---------------------------------------------------------------------------
SIN, COS, EXP = 0, 1, 2


@dataclass(frozen=True)
class Factor:
    """s * F(k x) with F in {sin, cos, exp}."""
    kind: int
    k: float
    s: float = 1.0

    def __call__(self, x):
        x = np.asarray(x, dtype=np.float64)
        if self.kind == SIN:
            return self.s * np.sin(self.k * x)
        if self.kind == COS:
            return self.s * np.cos(self.k * x)
        return self.s * np.exp(self.k * x)

    def d(self) -> "Factor":
        if self.kind == SIN:
            return Factor(COS, self.k, self.s * self.k)
        if self.kind == COS:
            return Factor(SIN, self.k, -self.s * self.k)
        return Factor(EXP, self.k, self.s * self.k)

    def antid(self) -> "Factor":
        """An antiderivative (k != 0 for every factor used here)."""
        if self.kind == SIN:
            return Factor(COS, self.k, -self.s / self.k)
        if self.kind == COS:
            return Factor(SIN, self.k, self.s / self.k)
        return Factor(EXP, self.k, self.s / self.k)

    def avg(self, x0, x1):
        """Exact average over [x0, x1] (elementwise on arrays), written as
        F(midpoint) * S(z), z = k (x1 - x0) / 2, S = sin z / z for sin/cos and
        sinh z / z for exp, which avoids the cancellation of the difference of
        antiderivatives on short intervals."""
        x0 = np.asarray(x0, dtype=np.float64)
        x1 = np.asarray(x1, dtype=np.float64)
        xm = 0.5 * (x0 + x1)
        z = 0.5 * self.k * (x1 - x0)
        with np.errstate(invalid="ignore", divide="ignore"):
            if self.kind == EXP:
                S = np.where(z == 0.0, 1.0, np.sinh(z) / np.where(z == 0.0, 1.0, z))
            else:
                S = np.where(z == 0.0, 1.0, np.sin(z) / np.where(z == 0.0, 1.0, z))
        return self(xm) * S


@dataclass(frozen=True)
class Term:
    """coef * X(x) * Y(y)."""
    coef: float
    X: Factor
    Y: Factor


@dataclass
class Separable:
    """u(x, y) = sum of separable terms; all calculus is exact."""
    terms: List[Term]

    def __call__(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = np.zeros(np.broadcast(x, y).shape)
        for t in self.terms:
            out = out + t.coef * t.X(x) * t.Y(y)
        return out

    def dx(self) -> "Separable":
        return Separable([Term(t.coef, t.X.d(), t.Y) for t in self.terms])

    def dy(self) -> "Separable":
        return Separable([Term(t.coef, t.X, t.Y.d()) for t in self.terms])

    def scaled(self, s: float) -> "Separable":
        return Separable([Term(t.coef * s, t.X, t.Y) for t in self.terms])

    def __add__(self, other: "Separable") -> "Separable":
        return Separable(list(self.terms) + list(other.terms))

    def rect_avg(self, x0, x1, y0, y1):
        """Exact average over [x0,x1] x [y0,y1] (elementwise)."""
        out = 0.0
        for t in self.terms:
            out = out + t.coef * t.X.avg(x0, x1) * t.Y.avg(y0, y1)
        return out

    def xseg_avg(self, x0, x1, y):
        """Exact average over the horizontal segment [x0,x1] x {y}."""
        out = 0.0
        for t in self.terms:
            out = out + t.coef * t.X.avg(x0, x1) * t.Y(y)
        return out

    def yseg_avg(self, x, y0, y1):
        """Exact average over the vertical segment {x} x [y0,y1]."""
        out = 0.0
        for t in self.terms:
            out = out + t.coef * t.X(x) * t.Y.avg(y0, y1)
        return out


class Pointwise:
    """A smooth function given pointwise with its gradient (for manufactured
    solutions that are not sums of separable products).  Averages over cells
    and faces use 10-point Gauss-Legendre rules per direction: for the smooth
    functions used here on cells of size h <= 1/32 they are exact to rounding."""

    _G, _W = np.polynomial.legendre.leggauss(10)

    def __init__(self, f, fx=None, fy=None):
        self.f, self.fx, self.fy = f, fx, fy

    def __call__(self, x, y):
        return self.f(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))

    def dx(self) -> "Pointwise":
        return Pointwise(self.fx)

    def dy(self) -> "Pointwise":
        return Pointwise(self.fy)

    def rect_avg(self, x0, x1, y0, y1):
        x0, x1, y0, y1 = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (x0, x1, y0, y1)))
        g, w = self._G, 0.5 * self._W
        xs = 0.5 * (x0 + x1)[..., None, None] + 0.5 * (x1 - x0)[..., None, None] * g[:, None]
        ys = 0.5 * (y0 + y1)[..., None, None] + 0.5 * (y1 - y0)[..., None, None] * g[None, :]
        return np.einsum("...ab,a,b->...", self(xs, ys), w, w)

    def xseg_avg(self, x0, x1, y):
        x0, x1, y = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (x0, x1, y)))
        g, w = self._G, 0.5 * self._W
        xs = 0.5 * (x0 + x1)[..., None] + 0.5 * (x1 - x0)[..., None] * g
        return np.einsum("...a,a->...", self(xs, y[..., None]), w)

    def yseg_avg(self, x, y0, y1):
        x, y0, y1 = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (x, y0, y1)))
        g, w = self._G, 0.5 * self._W
        ys = 0.5 * (y0 + y1)[..., None] + 0.5 * (y1 - y0)[..., None] * g
        return np.einsum("...a,a->...", self(x[..., None], ys), w)


def u_flower() -> Pointwise:
    """u = r^4 cos(3 theta) = r (x^3 - 3 x y^2) about the origin (Sec. 6.2)."""
    def f(x, y):
        return np.hypot(x, y) * (x ** 3 - 3 * x * y ** 2)

    def fx(x, y):
        r = np.hypot(x, y)
        return x / r * (x ** 3 - 3 * x * y ** 2) + r * (3 * x ** 2 - 3 * y ** 2)

    def fy(x, y):
        r = np.hypot(x, y)
        return y / r * (x ** 3 - 3 * x * y ** 2) - 6 * r * x * y

    return Pointwise(f, fx, fy)


def f_flower() -> Pointwise:
    """Laplacian of u_flower: (16 - 9) r^2 cos(3 theta) = 7 (x^3 - 3 x y^2) / r."""
    return Pointwise(lambda x, y: 7.0 * (x ** 3 - 3 * x * y ** 2) / np.hypot(x, y))


def apply_L(u: Separable, a: float, b: float, c: float) -> Separable:
    """f = a u_xx + b u_xy + c u_yy, exact (Eq. 1.1)."""
    return (u.dx().dx().scaled(a) + u.dx().dy().scaled(b)
            + u.dy().dy().scaled(c))


# Manufactured solutions used by the paper's Table 3 and the workloads below.
def u_table3() -> Separable:
    """u = sin(4x) cos(3y) (Sec. 6.1, Eq. 6.2)."""
    return Separable([Term(1.0, Factor(SIN, 4.0), Factor(COS, 3.0))])


def u_sinpi() -> Separable:
    """u = sin(pi x) sin(pi y)."""
    return Separable([Term(1.0, Factor(SIN, math.pi), Factor(SIN, math.pi))])


def u_expcos() -> Separable:
    """u = exp(x) cos(2y)."""
    return Separable([Term(1.0, Factor(EXP, 1.0), Factor(COS, 2.0))])


def u_sinexp() -> Separable:
    """u = sin(3x) exp(y)."""
    return Separable([Term(1.0, Factor(SIN, 3.0), Factor(EXP, 1.0))])


def random_fourier(seed: int, modes: int = 16) -> Separable:
    """f = sum_{p,q<=modes} c_pq sin(p pi x) sin(q pi y), c_pq ~ N(0, 1/(p^2+q^2))."""
    rng = np.random.default_rng(seed)
    terms = []
    for p in range(1, modes + 1):
        for q in range(1, modes + 1):
            cpq = rng.normal(0.0, math.sqrt(1.0 / (p * p + q * q)))
            terms.append(Term(float(cpq), Factor(SIN, p * math.pi),
                              Factor(SIN, q * math.pi)))
    return Separable(terms)


# ---------------------------------------------------------------------------
# Domains: box minus a union of ellipses.
# ---------------------------------------------------------------------------
DIRICHLET, NEUMANN, ROBIN = 0, 1, 2


@dataclass(frozen=True)
class Ellipse:
    cx: float
    cy: float
    r1: float
    r2: float
    theta: float = 0.0

    def inside(self, x, y):
        """True strictly inside the (closed) hole's interior."""
        c, s = math.cos(self.theta), math.sin(self.theta)
        dx = np.asarray(x) - self.cx
        dy = np.asarray(y) - self.cy
        xp = c * dx + s * dy
        yp = -s * dx + c * dy
        return (xp / self.r1) ** 2 + (yp / self.r2) ** 2 < 1.0


@dataclass(frozen=True)
class Flower:
    """The hole bounded by the closed curve r = r0 + amp cos(k theta) in polar
    coordinates about (cx, cy) (Sec. 6.2): the domain keeps
    r > r0 + amp cos(k theta).  Requires 0 < amp < r0 and an integer k >= 1."""
    cx: float
    cy: float
    r0: float
    amp: float
    k: int


@dataclass(frozen=True)
class OutsideRect:
    """The hole that is everything outside the rectangle with corner (cx, cy)
    and sides w (along the direction theta) and hgt (along theta + pi/2):
    with it the domain is the (rotated) rectangle, cut from the box.  The
    rectangle must lie inside the box."""
    cx: float
    cy: float
    w: float
    hgt: float
    theta: float


@dataclass(frozen=True)
class BC:
    kind: int = DIRICHLET
    alpha1: float = 1.0
    alpha2: float = 0.0


@dataclass
class Domain:
    """Box [x0,x1]x[y0,y1] minus the union of `holes`.

    `box_bc` gives the condition on the four sides in the order
    (south y=y0, east x=x1, north y=y1, west x=x0); `hole_bc[k]` the
    condition on the boundary of hole k.
    """
    x0: float = 0.0
    y0: float = 0.0
    x1: float = 1.0
    y1: float = 1.0
    holes: List[object] = field(default_factory=list)    # Ellipse, Flower or OutsideRect
    box_bc: Tuple[BC, BC, BC, BC] = (BC(), BC(), BC(), BC())
    hole_bc: List[BC] = field(default_factory=list)


def bc_value(u: Separable, bc: BC, x, y, nx, ny):
    """Point value of N u at (x, y) with outward normal (nx, ny) (Eq. 1.2)."""
    val = u(x, y)
    dn = u.dx()(x, y) * nx + u.dy()(x, y) * ny
    if bc.kind == DIRICHLET:
        return val
    if bc.kind == NEUMANN:
        return dn
    return bc.alpha1 * val + bc.alpha2 * dn


def wall_face_data(u: Separable, dom: Domain, n: int) -> np.ndarray:
    """Exact face averages of N u on the 4 box sides, packed S, E, N, W.

    Each side has n faces; S and N are indexed by x, E and W by y.  The box
    is split into n x n square cells of size h = (x1-x0)/n.
    """
    h = (dom.x1 - dom.x0) / n
    xs = dom.x0 + h * np.arange(n)
    ys = dom.y0 + h * np.arange(n)
    out = []
    # (side, fixed coordinate, outward normal)
    for side, bc in enumerate(dom.box_bc):
        if side == 0:      # south, y = y0, n = (0,-1)
            val = u.xseg_avg(xs, xs + h, dom.y0)
            dn = -u.dy().xseg_avg(xs, xs + h, dom.y0)
        elif side == 1:    # east, x = x1, n = (1,0)
            val = u.yseg_avg(dom.x1, ys, ys + h)
            dn = u.dx().yseg_avg(dom.x1, ys, ys + h)
        elif side == 2:    # north, y = y1, n = (0,1)
            val = u.xseg_avg(xs, xs + h, dom.y1)
            dn = u.dy().xseg_avg(xs, xs + h, dom.y1)
        else:              # west, x = x0, n = (-1,0)
            val = u.yseg_avg(dom.x0, ys, ys + h)
            dn = -u.dx().yseg_avg(dom.x0, ys, ys + h)
        val = np.broadcast_to(np.asarray(val, dtype=np.float64), (n,))
        dn = np.broadcast_to(np.asarray(dn, dtype=np.float64), (n,))
        if bc.kind == DIRICHLET:
            out.append(val)
        elif bc.kind == NEUMANN:
            out.append(dn)
        else:
            out.append(bc.alpha1 * val + bc.alpha2 * dn)
    return np.concatenate(out)


def regular_cell_averages(fun: Separable, dom: Domain, n: int) -> np.ndarray:
    """Exact averages of `fun` over all n x n full cells, shape [n, n] = [y, x]."""
    h = (dom.x1 - dom.x0) / n
    xs = dom.x0 + h * np.arange(n)
    ys = dom.y0 + h * np.arange(n)
    X0 = xs[None, :]
    Y0 = ys[:, None]
    return np.asarray(fun.rect_avg(X0, X0 + h, Y0, Y0 + h) * np.ones((n, n)))


# ---------------------------------------------------------------------------
# Named workloads (seeded).
# ---------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    dom: Domain
    a: float
    b: float
    c: float
    u: Separable          # exact solution (None-like when unknown)
    f: Separable          # right-hand side
    exact: bool = True    # whether u is the exact solution


def problem_table3() -> Problem:
    """Unit square, (a,b,c) = (1,0,2), u = sin(4x)cos(3y), Dirichlet (Sec. 6.1)."""
    u = u_table3()
    return Problem("table3", Domain(), 1.0, 0.0, 2.0, u, apply_L(u, 1.0, 0.0, 2.0))


def problem_poisson_square() -> Problem:
    """Poisson on the unit square, u = sin(pi x) sin(pi y), Dirichlet."""
    u = u_sinpi()
    return Problem("poisson_square", Domain(), 1.0, 0.0, 1.0, u,
                   apply_L(u, 1.0, 0.0, 1.0))


def problem_disk() -> Problem:
    """Unit square minus the disk r=0.2 at (0.5,0.5); a=1, b=0.5, c=2;
    Dirichlet on the box, Neumann on the circle; u = exp(x) cos(2y)."""
    u = u_expcos()
    dom = Domain(holes=[Ellipse(0.5, 0.5, 0.2, 0.2, 0.0)],
                 hole_bc=[BC(NEUMANN, 0.0, 1.0)])
    return Problem("disk", dom, 1.0, 0.5, 2.0, u, apply_L(u, 1.0, 0.5, 2.0))


def problem_four_disks(kind: int = DIRICHLET) -> Problem:
    """Sec. 6, a square minus four disks: Poisson's equation on the unit
    square minus the union of four overlapping disks (six kinks on the
    union's boundary), u = sin(pi x) sin(pi y), Dirichlet on the square and
    `kind` (Dirichlet or Neumann) on the disks; the paper uses eps = 0.08."""
    u = u_sinpi()
    disks = [Ellipse(0.5, 0.5, 0.2, 0.2), Ellipse(0.5, 0.735, 0.1, 0.1),
             Ellipse(0.2965, 0.3825, 0.1, 0.1), Ellipse(0.7035, 0.3825, 0.1, 0.1)]
    bc = BC(DIRICHLET, 1.0, 0.0) if kind == DIRICHLET else BC(NEUMANN, 0.0, 1.0)
    dom = Domain(holes=disks, hole_bc=[bc] * 4)
    return Problem("four_disks_" + ("D" if kind == DIRICHLET else "N"), dom, 1.0, 0.0, 1.0, u,
                   apply_L(u, 1.0, 0.0, 1.0))


def problem_flower(kind: int = NEUMANN) -> Problem:
    """Sec. 6.2, a square minus a flower: Poisson's equation on
    (-0.5, 0.5)^2 minus the flower r <= 0.25 + 0.05 cos(6 theta) about the
    origin, u = r^4 cos(3 theta), Dirichlet on the square and `kind` on the
    flower (Neumann in the paper); the paper uses eps = 0.02."""
    u = u_flower()
    bc = BC(NEUMANN, 0.0, 1.0) if kind == NEUMANN else BC(DIRICHLET, 1.0, 0.0)
    dom = Domain(x0=-0.5, y0=-0.5, x1=0.5, y1=0.5, holes=[Flower(0.0, 0.0, 0.25, 0.05, 6)], hole_bc=[bc])
    return Problem("flower", dom, 1.0, 0.0, 1.0, u, f_flower())


def problem_rotated_square() -> Problem:
    """Sec. 6.1, the rotated square: Omega_r is (0,1)^2 rotated about the
    origin by pi/6, (a, b, c) = (5, -2 sqrt 3, 7) / 4, u the solution
    sin(4 x) cos(3 y) of the unit-square case rotated by pi/6, Dirichlet data.
    The computational box is [-0.625, 0.875] x [-0.125, 1.375] (side 1.5, so
    that h = 1/64 .. 1/512 divide it and Omega_r lies inside)."""
    th = math.pi / 6
    c, s = math.cos(th), math.sin(th)

    def back(x, y):            # rotate (x, y) by -pi/6
        return c * x + s * y, -s * x + c * y

    def u(x, y):
        xp, yp = back(x, y)
        return np.sin(4 * xp) * np.cos(3 * yp)

    def ux(x, y):
        xp, yp = back(x, y)
        gx, gy = 4 * np.cos(4 * xp) * np.cos(3 * yp), -3 * np.sin(4 * xp) * np.sin(3 * yp)
        return c * gx - s * gy

    def uy(x, y):
        xp, yp = back(x, y)
        gx, gy = 4 * np.cos(4 * xp) * np.cos(3 * yp), -3 * np.sin(4 * xp) * np.sin(3 * yp)
        return s * gx + c * gy

    def f(x, y):
        xp, yp = back(x, y)
        return -34.0 * np.sin(4 * xp) * np.cos(3 * yp)

    dom = Domain(x0=-0.625, y0=-0.125, x1=0.875, y1=1.375,
                 holes=[OutsideRect(0.0, 0.0, 1.0, 1.0, th)], hole_bc=[BC()])
    return Problem("rotated_square", dom, 1.25, -math.sqrt(3.0) / 2.0, 1.75, Pointwise(u, ux, uy),
                   Pointwise(f))


def _boundary_points(e: Ellipse, m: int = 720):
    t = np.linspace(0, 2 * math.pi, m, endpoint=False)
    c, s = math.cos(e.theta), math.sin(e.theta)
    return (e.cx + c * e.r1 * np.cos(t) - s * e.r2 * np.sin(t),
            e.cy + s * e.r1 * np.cos(t) + c * e.r2 * np.sin(t))


def _ellipse_union(rng) -> List[Ellipse]:
    """3-6 ellipses, centres U[0.3,0.7]^2, semi-axes U[0.06,0.16],
    rotation U[0,pi); accepted when at least one pair overlaps, every
    ellipse keeps 0.05 from the box (bounding-circle test), and every pair
    that does not overlap keeps 0.05 apart (no narrow channels)."""
    while True:
        k = int(rng.integers(3, 7))
        es = []
        for _ in range(k):
            cx, cy = rng.uniform(0.3, 0.7, size=2)
            r1, r2 = rng.uniform(0.06, 0.16, size=2)
            th = rng.uniform(0.0, math.pi)
            es.append(Ellipse(float(cx), float(cy), float(r1), float(r2), float(th)))
        ok_box = all(min(e.cx, e.cy, 1 - e.cx, 1 - e.cy) - max(e.r1, e.r2) >= 0.05
                     for e in es)
        if not ok_box:
            continue
        overl = False
        narrow = False
        pts = [_boundary_points(e) for e in es]
        for i in range(k):
            for j in range(i + 1, k):
                # overlap if some point of ellipse i lies inside ellipse j
                if np.any(es[j].inside(*pts[i])) or np.any(es[i].inside(*pts[j])):
                    overl = True
                else:
                    d = np.hypot(pts[i][0][:, None] - pts[j][0][None, :],
                                 pts[i][1][:, None] - pts[j][1][None, :]).min()
                    narrow = narrow or d < 0.05
        if overl and not narrow:
            return es


def problem_ellipses(seed: int = 0) -> Problem:
    """Unit square minus a seeded union of 3-6 ellipses; Robin
    (alpha1=1, alpha2=0.5) on every curve; a=1.5, b=-0.8, c=1;
    u = sin(3x) exp(y)."""
    rng = np.random.default_rng(1000 + seed)
    holes = _ellipse_union(rng)
    rb = BC(ROBIN, 1.0, 0.5)
    dom = Domain(holes=holes, box_bc=(rb, rb, rb, rb), hole_bc=[rb] * len(holes))
    u = u_sinexp()
    return Problem(f"ellipses{seed}", dom, 1.5, -0.8, 1.0, u,
                   apply_L(u, 1.5, -0.8, 1.0))


def problem_batch(seed: int) -> Tuple[Problem, int]:
    """Problem `seed` of the many-problem batch and its grid size N.

    N = 2^round(U[6, 10]) (log-uniform 64..1024); 1-8 holes, each a circle or
    an ellipse with semi-axes U[0.03, 0.15] and rotation U[0, pi), whose
    bounding circles keep 0.02 from the box and from one another; a, c ~
    U[0.5, 2], b ~ U(-sqrt(3ac), sqrt(3ac)); Dirichlet on the box and a
    condition drawn from {Dirichlet, Neumann, Robin(1, 0.5)} on each hole;
    f a 16 x 16-mode random Fourier series and g = 0 (u = 0 on the data; no
    exact solution)."""
    rng = np.random.default_rng(5000 + seed)
    n = 2 ** int(round(rng.uniform(6.0, 10.0)))
    nh = int(rng.integers(1, 9))
    holes: List[Ellipse] = []
    for _ in range(4000):
        if len(holes) == nh:
            break
        circle = rng.random() < 0.5
        r1 = float(rng.uniform(0.03, 0.15))
        r2 = r1 if circle else float(rng.uniform(0.03, 0.15))
        th = 0.0 if circle else float(rng.uniform(0.0, math.pi))
        cx, cy = (float(v) for v in rng.uniform(0.0, 1.0, 2))
        R = max(r1, r2)
        if min(cx, cy, 1.0 - cx, 1.0 - cy) - R < 0.02:
            continue
        if any(math.hypot(cx - o.cx, cy - o.cy) - R - max(o.r1, o.r2) < 0.02 for o in holes):
            continue
        holes.append(Ellipse(cx, cy, r1, r2, th))
    a = float(rng.uniform(0.5, 2.0))
    c = float(rng.uniform(0.5, 2.0))
    bmax = math.sqrt(3.0 * a * c)
    b = float(rng.uniform(-bmax, bmax))
    kinds = [BC(), BC(NEUMANN, 0.0, 1.0), BC(ROBIN, 1.0, 0.5)]
    hole_bc = [kinds[int(rng.integers(0, 3))] for _ in holes]
    dom = Domain(holes=holes, box_bc=(BC(), BC(), BC(), BC()), hole_bc=hole_bc)
    f = random_fourier(7000 + seed, 16)
    return Problem(f"batch{seed}", dom, a, b, c, Separable([]), f, exact=False), n
