"""Pins of the oracle against what the paper and mathematics fix.

Every check compares the oracle with something it does not compute itself:
values printed in the paper (tests/golden/*), closed-form polynomial
calculus, adaptive scipy quadrature over the exact disk complement, closed
form areas and moments, and a direct sparse solve.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spl
from scipy import integrate
from scipy.sparse.linalg import eigs

from oracle import discretize as D
from oracle import geometry as G
from oracle import multigrid as M
from oracle.ghost import extrapolation_coefficients, ghost_coefficients
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------
# closed-form polynomial calculus used as the independent reference
# ---------------------------------------------------------------------------
class Poly2:
    """P(x, y) = sum c[p, q] x^p y^q with exact calculus."""

    def __init__(self, c):
        self.c = np.array(c, dtype=np.float64)

    @staticmethod
    def random(deg, seed):
        rng = np.random.default_rng(seed)
        c = np.zeros((deg + 1, deg + 1))
        for p in range(deg + 1):
            for q in range(deg + 1 - p):
                c[p, q] = rng.standard_normal()
        return Poly2(c)

    def __call__(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = np.zeros(np.broadcast(x, y).shape)
        for p in range(self.c.shape[0]):
            for q in range(self.c.shape[1]):
                if self.c[p, q]:
                    out = out + self.c[p, q] * x ** p * y ** q
        return out

    def dx(self):
        c = np.zeros_like(self.c)
        c[:-1, :] = self.c[1:, :] * np.arange(1, self.c.shape[0])[:, None]
        return Poly2(c)

    def dy(self):
        c = np.zeros_like(self.c)
        c[:, :-1] = self.c[:, 1:] * np.arange(1, self.c.shape[1])[None, :]
        return Poly2(c)

    def L(self, a, b, c):
        f = self.dx().dx().c * a + self.dx().dy().c * b + self.dy().dy().c * c
        return Poly2(f)

    def rect_avg(self, x0, x1, y0, y1):
        out = 0.0
        for p in range(self.c.shape[0]):
            for q in range(self.c.shape[1]):
                if self.c[p, q]:
                    ix = (x1 ** (p + 1) - x0 ** (p + 1)) / ((p + 1) * (x1 - x0))
                    iy = (y1 ** (q + 1) - y0 ** (q + 1)) / ((q + 1) * (y1 - y0))
                    out = out + self.c[p, q] * ix * iy
        return out

    def seg_avg_x(self, x0, x1, y):
        out = 0.0
        for p in range(self.c.shape[0]):
            for q in range(self.c.shape[1]):
                if self.c[p, q]:
                    out = out + self.c[p, q] * (x1 ** (p + 1) - x0 ** (p + 1)) / ((p + 1) * (x1 - x0)) * y ** q
        return out

    def seg_avg_y(self, x, y0, y1):
        out = 0.0
        for p in range(self.c.shape[0]):
            for q in range(self.c.shape[1]):
                if self.c[p, q]:
                    out = out + self.c[p, q] * x ** p * (y1 ** (q + 1) - y0 ** (q + 1)) / ((q + 1) * (y1 - y0))
        return out


def _box_wall_data(P: Poly2, dom: W.Domain, n: int):
    """Exact face averages of N P on the box faces, packed S, E, N, W."""
    h = (dom.x1 - dom.x0) / n
    xs = dom.x0 + h * np.arange(n)
    ys = dom.y0 + h * np.arange(n)
    out = []
    for side, bc in enumerate(dom.box_bc):
        if side == 0:
            val, dn = P.seg_avg_x(xs, xs + h, dom.y0), -P.dy().seg_avg_x(xs, xs + h, dom.y0)
        elif side == 1:
            val, dn = P.seg_avg_y(dom.x1, ys, ys + h), P.dx().seg_avg_y(dom.x1, ys, ys + h)
        elif side == 2:
            val, dn = P.seg_avg_x(xs, xs + h, dom.y1), P.dy().seg_avg_x(xs, xs + h, dom.y1)
        else:
            val, dn = P.seg_avg_y(dom.x0, ys, ys + h), -P.dx().seg_avg_y(dom.x0, ys, ys + h)
        a1, a2 = D.bc_alpha(bc)
        out.append(np.broadcast_to(a1 * val + a2 * dn, (n,)))
    return np.concatenate(out)


# ---------------------------------------------------------------------------
# Sec. 4.1 ghost formulas
# ---------------------------------------------------------------------------
def test_ghost_coefficients_match_printed_formulas():
    """Dirichlet and Neumann ghost coefficients of Sec. 4.1 (golden file),
    with the garbled Dirichlet depth-2 datum read as 300."""
    h = 0.01
    for kind, depth, c3, c2, c1, c0, cg, div in _golden("ghost_coefficients.txt"):
        k = W.DIRICHLET if kind == "dirichlet" else W.NEUMANN
        G_ = ghost_coefficients(k, 0.0, 0.0, h)[int(depth) - 1]
        want = np.array([float(c0), float(c1), float(c2), float(c3)]) / float(div)
        np.testing.assert_allclose(G_[:4], want, rtol=0, atol=1e-12)
        datum_scale = 1.0 if k == W.DIRICHLET else 12.0 * h
        np.testing.assert_allclose(G_[4], float(cg) * datum_scale / float(div), rtol=1e-12)


@pytest.mark.parametrize("kind,a1,a2", [(W.DIRICHLET, 1, 0), (W.NEUMANN, 0, 1), (W.ROBIN, 1.0, 0.5),
                                        (W.ROBIN, 2.0, -0.3)])
def test_ghost_exact_on_quartics(kind, a1, a2):
    """Ghost averages reproduce the exact averages of any quartic; a quintic
    is not reproduced (so a wrong coefficient cannot hide)."""
    h = 0.037
    rng = np.random.default_rng(3)
    for deg, exact in ((4, True), (5, False)):
        c = rng.standard_normal(deg + 1)
        P = np.polynomial.Polynomial(c)      # in the physical distance x from the wall
        I = P.integ()
        dP = P.deriv()
        avg = lambda s0, s1: (I(s1 * h) - I(s0 * h)) / ((s1 - s0) * h)
        U = [avg(-k - 1, -k) for k in range(4)]
        g = (a1 * P(0.0) + a2 * dP(0.0)) if kind == W.ROBIN else (P(0.0) if kind == W.DIRICHLET else dP(0.0))
        Gc = ghost_coefficients(kind, a1, a2, h)
        for m in (1, 2):
            got = Gc[m - 1, :4] @ U + Gc[m - 1, 4] * g
            want = avg(m - 1, m)
            if exact:
                assert abs(got - want) < 1e-11 * (1 + abs(want))
            else:
                assert abs(got - want) > 1e-9


def test_corner_extrapolation_exact_on_quartics():
    E = extrapolation_coefficients()
    rng = np.random.default_rng(4)
    P = np.polynomial.Polynomial(rng.standard_normal(5))
    I = P.integ()
    avg = lambda s0, s1: (I(s1) - I(s0)) / (s1 - s0)
    U = [avg(-k - 1, -k) for k in range(5)]
    for m in (1, 2):
        assert abs(E[m - 1] @ U - avg(m - 1, m)) < 1e-11
    np.testing.assert_allclose(E[0], [5, -10, 10, -5, 1], atol=1e-11)


# ---------------------------------------------------------------------------
# SFV rows: exactness on polynomials (Eq. 4.7a,b and the ghosts)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("abc,bcs", [
    ((1.0, 0.0, 2.0), (W.BC(), W.BC(), W.BC(), W.BC())),
    ((1.0, 0.5, 2.0), (W.BC(), W.BC(W.NEUMANN, 0, 1), W.BC(), W.BC(W.ROBIN, 1.0, 0.5))),
    ((1.5, -0.8, 1.0), (W.BC(W.ROBIN, 1.0, 0.5),) * 4),
])
def test_sfv_rows_exact_on_quartics(abc, bcs):
    a, b, c = abc
    n = 12
    dom = W.Domain(box_bc=bcs)
    lev = G.build_level(dom, n, 0.1)
    d = D.discretize(lev, a, b, c)
    assert (d.kind == D.SFV).all(), "every cell of a box is an SFV cell"
    P = Poly2.random(4, 11)
    h = lev.h
    xs = h * np.arange(n)
    X0, Y0 = np.meshgrid(xs, xs)
    ue = P.rect_avg(X0, X0 + h, Y0, Y0 + h)
    fe = P.L(a, b, c).rect_avg(X0, X0 + h, Y0, Y0 + h)
    g = _box_wall_data(P, dom, n)
    bvec = D.rhs(d, fe, g)
    tau = (d.A @ ue.ravel() - bvec.ravel())
    assert np.abs(tau).max() < 1e-9 * (1.0 / h ** 2), np.abs(tau).max()


def test_sfv_interior_exact_on_quintics():
    a, b, c = 1.0, 0.0, 2.0
    n = 16
    dom = W.Domain()
    lev = G.build_level(dom, n, 0.1)
    d = D.discretize(lev, a, b, c)
    P = Poly2.random(5, 12)
    h = lev.h
    xs = h * np.arange(n)
    X0, Y0 = np.meshgrid(xs, xs)
    ue = P.rect_avg(X0, X0 + h, Y0, Y0 + h)
    fe = P.L(a, b, c).rect_avg(X0, X0 + h, Y0, Y0 + h)
    tau = (d.A @ ue.ravel()).reshape(n, n) - fe
    inner = tau[2:-2, 2:-2]
    assert np.abs(inner).max() < 1e-9 / h ** 2
    assert np.abs(tau).max() > 1e-6            # wall rows see the O(h^5) ghost error


# ---------------------------------------------------------------------------
# Table 3: regular-domain accuracy (closed-form inputs, direct solve)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [64, 128])
def test_table3_error_norms(n):
    rows = {int(r[0]): [float(v) for v in r[1:]] for r in _golden("table3_unit_square.txt")}
    P = W.problem_table3()
    lev = G.build_level(P.dom, n, 0.1)
    d = D.discretize(lev, P.a, P.b, P.c)
    f = D.cell_averages(lev, P.f)
    g = D.boundary_data(d, P.u)
    b = D.rhs(d, f, g)
    u = spl.spsolve(d.A.tocsc(), b.ravel()).reshape(n, n)
    ue = W.regular_cell_averages(P.u, P.dom, n)
    e = np.abs(u - ue)
    got = [e.max(), (e * lev.vol).sum(), math.sqrt((e * e * lev.vol).sum())]
    for gv, want in zip(got, rows[n]):
        assert float(f"{gv:.2e}") == want, (gv, want)


# ---------------------------------------------------------------------------
# Table 2: two-grid spectral radius (smoother, transfers, coarse operator)
# ---------------------------------------------------------------------------
def test_table2_two_grid_spectral_radius():
    P = W.problem_table3()
    n = 64
    H = M.build_hierarchy(P.dom, n, P.a, P.b, P.c, min_coarse=n // 2)
    assert H.nl == 2
    for nu1, nu2, want in _golden("table2_unit_square.txt"):
        op = M.two_grid_operator(H, int(nu1), int(nu2))
        v0 = np.random.default_rng(0).standard_normal(n * n)
        w = eigs(op, k=1, which="LM", return_eigenvectors=False, tol=1e-9, maxiter=20000, v0=v0)
        assert round(abs(w[0]), 3) == float(want), (nu1, nu2, abs(w[0]))


# ---------------------------------------------------------------------------
# Cut cells: closed-form geometry
# ---------------------------------------------------------------------------
def _level_moment(lev, p, q):
    """Integral of x^p y^q over the whole domain from the oracle's cells."""
    h = lev.h
    tot = 0.0
    for k in np.flatnonzero(lev.present.ravel()):
        px, py = lev.center(int(k))
        m = lev.moments(int(k))
        for a in range(p + 1):
            for b in range(q + 1):
                tot += (math.comb(p, a) * math.comb(q, b) * px ** (p - a) * py ** (q - b)
                        * h ** (a + b) * m[G.MIDX[(a, b)]] * h * h)
    return tot


@pytest.mark.parametrize("n", [32, 100])
def test_disk_complement_area_moments_perimeter(n):
    r = 0.2
    dom = W.problem_disk().dom
    lev = G.build_level(dom, n, 0.1)
    # closed forms for the unit square minus the disk of radius r at (1/2, 1/2)
    area = 1.0 - math.pi * r * r
    mx = 0.5 - 0.5 * math.pi * r * r
    mxx = 1.0 / 3.0 - (math.pi * r * r * 0.25 + math.pi * r ** 4 / 4.0)
    mxxyy = 1.0 / 9.0 - integrate.dblquad(lambda y, x: x * x * y * y, 0.3, 0.7,
                                          lambda x: 0.5 - math.sqrt(max(0, r * r - (x - .5) ** 2)),
                                          lambda x: 0.5 + math.sqrt(max(0, r * r - (x - .5) ** 2)),
                                          epsabs=1e-15, epsrel=1e-14)[0]
    assert abs(lev.vol.sum() - area) < 1e-13
    assert abs(_level_moment(lev, 1, 0) - mx) < 1e-13
    assert abs(_level_moment(lev, 2, 0) - mxx) < 1e-13
    assert abs(_level_moment(lev, 2, 2) - mxxyy) < 1e-12
    per = sum(w for cc in lev.cut.values() for (_, _, _, _, w, _) in cc.bnodes)
    assert abs(per - 2 * math.pi * r) < 1e-13
    vf = lev.vol[lev.present] / lev.h ** 2
    assert vf.min() >= 0.1 - 1e-14              # Alg. 1: no cell below epsilon h^2
    # merged control volumes point to a present cell
    own = lev.owner[(lev.owner >= 0) & ~lev.present]
    assert lev.present.ravel()[own].all()


def test_overlapping_circles_area():
    r = 0.15
    d = 0.2                                     # centre distance < 2r: overlap
    dom = W.Domain(holes=[W.Ellipse(0.4, 0.5, r, r), W.Ellipse(0.6, 0.5, r, r)],
                   hole_bc=[W.BC(), W.BC()])
    lens = 2 * r * r * math.acos(d / (2 * r)) - 0.5 * d * math.sqrt(4 * r * r - d * d)
    area = 1.0 - (2 * math.pi * r * r - lens)
    for n in (64, 90):
        lev = G.build_level(dom, n, 0.1)
        assert abs(lev.vol.sum() - area) < 1e-13


def test_ellipse_area():
    e = W.Ellipse(0.45, 0.52, 0.2, 0.11, 0.7)
    dom = W.Domain(holes=[e], hole_bc=[W.BC()])
    lev = G.build_level(dom, 77, 0.1)
    assert abs(lev.vol.sum() - (1 - math.pi * e.r1 * e.r2)) < 1e-13


def _moved_components(monkeypatch):
    moved = []
    attach = G._attach_component
    monkeypatch.setattr(G, "_attach_component",
                        lambda lev, k, pcs, cv: (moved.append(k), attach(lev, k, pcs, cv))[1])
    return moved


def test_components_moved_to_a_neighbour_keep_the_moments(monkeypatch):
    """Alg. 1, cells of several components: at N = 64 some cut cells of
    problem 4 of the batch workload hold two pieces of the domain (a narrow
    gap between two holes), the level still resolves, and every component
    joins some cell whole.  The area, first and second moments of the domain
    then equal the closed forms of the unit square minus disjoint rotated
    ellipses: a component dropped, or its moments shifted to the wrong
    centre, fails one of them."""
    P, n = W.problem_batch(4)
    moved = _moved_components(monkeypatch)
    lev = G.build_level(P.dom, n, 0.1)
    assert moved and lev.resolved, lev.reason
    want = {(0, 0): 1.0, (1, 0): 0.5, (0, 1): 0.5, (2, 0): 1 / 3, (1, 1): 0.25, (0, 2): 1 / 3}
    for e in P.dom.holes:
        a = math.pi * e.r1 * e.r2
        c, s = math.cos(e.theta), math.sin(e.theta)
        ixx = a / 4 * (e.r1 ** 2 * c * c + e.r2 ** 2 * s * s)
        iyy = a / 4 * (e.r1 ** 2 * s * s + e.r2 ** 2 * c * c)
        ixy = a / 4 * (e.r1 ** 2 - e.r2 ** 2) * c * s
        want[(0, 0)] -= a
        want[(1, 0)] -= a * e.cx
        want[(0, 1)] -= a * e.cy
        want[(2, 0)] -= a * e.cx ** 2 + ixx
        want[(1, 1)] -= a * e.cx * e.cy + ixy
        want[(0, 2)] -= a * e.cy ** 2 + iyy
    assert abs(lev.vol.sum() - want[(0, 0)]) < 1e-13
    for (p, q), v in want.items():
        assert abs(_level_moment(lev, p, q) - v) < 1e-13, (p, q)


def _waist_domain():
    """Two disks of radius 0.2 whose centres are 0.3999 apart: their union
    has a waist 0.0089 high at x = 0.49995, thinner than a cell at the grids
    below, so the cell holding it is split into the parts above and below."""
    return W.Domain(holes=[W.Ellipse(0.3, 0.507, 0.2, 0.2), W.Ellipse(0.6999, 0.507, 0.2, 0.2)],
                    hole_bc=[W.BC(), W.BC(W.NEUMANN, 0, 1)])


@pytest.mark.parametrize("n", [32, 48, 64])
def test_cell_split_by_a_waist_keeps_the_moments(monkeypatch, n):
    """Alg. 1, cells of several components, on a union of two disks that
    overlap by a sliver: the cells holding the waist have a part above and
    a part below it; one part stays, the other joins a neighbour, and the
    level resolves.  The area and the moments of the domain equal those of
    the square minus the union: two disks minus their lens, with the
    first moments from the union's symmetry and the second moments of the
    lens by adaptive quadrature."""
    dom = _waist_domain()
    moved = _moved_components(monkeypatch)
    lev = G.build_level(dom, n, 0.1)
    assert moved and lev.resolved, lev.reason
    r, c1, c2, cy = 0.2, 0.3, 0.6999, 0.507
    d = c2 - c1
    lens = 2 * r * r * math.acos(d / (2 * r)) - 0.5 * d * math.sqrt(4 * r * r - d * d)
    union = 2 * math.pi * r * r - lens
    xm = 0.5 * (c1 + c2)

    def lens_int(f):
        half = lambda x: min(math.sqrt(max(0.0, r * r - (x - c1) ** 2)), math.sqrt(max(0.0, r * r - (x - c2) ** 2)))
        return integrate.dblquad(lambda y, x: f(x, y), c2 - r, c1 + r, lambda x: cy - half(x),
                                 lambda x: cy + half(x), epsabs=1e-16, epsrel=1e-14)[0]

    disk_xx = sum(math.pi * r * r * (c * c + r * r / 4) for c in (c1, c2))
    disk_yy = 2 * math.pi * r * r * (cy * cy + r * r / 4)
    disk_xy = sum(math.pi * r * r * c * cy for c in (c1, c2))
    want = {(0, 0): 1.0 - union, (1, 0): 0.5 - union * xm, (0, 1): 0.5 - union * cy,
            (2, 0): 1 / 3 - (disk_xx - lens_int(lambda x, y: x * x)),
            (0, 2): 1 / 3 - (disk_yy - lens_int(lambda x, y: y * y)),
            (1, 1): 0.25 - (disk_xy - lens_int(lambda x, y: x * y))}
    assert abs(lev.vol.sum() - want[(0, 0)]) < 1e-13
    for (p, q), v in want.items():
        assert abs(_level_moment(lev, p, q) - v) < 1e-13, (p, q)


def test_components_moved_in_an_overlapping_union_keep_the_moments(monkeypatch):
    """The same step in a union of overlapping ellipses (union 15) at
    N = 128, where it moves components; at N = 150 no cell has several.
    The moments of the domain agree between the two grids within 1e-12 (the
    Gauss rules on the ellipse arcs leave a few 1e-13): the moved component
    has volume 1.7e-9, so dropping it, or shifting its moments by one cell,
    shows."""
    P = W.problem_ellipses(15)
    moved = _moved_components(monkeypatch)
    lev = G.build_level(P.dom, 128, 0.1)
    assert moved and lev.resolved, lev.reason
    del moved[:]
    other = G.build_level(P.dom, 150, 0.1)
    assert not moved
    for p, q in ((0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)):
        assert abs(_level_moment(lev, p, q) - _level_moment(other, p, q)) < 1e-12, (p, q)


# ---------------------------------------------------------------------------
# PLG rows: exactness on quartics with averages from adaptive quadrature
# ---------------------------------------------------------------------------
def _disk_cell_avg(P, i, j, h, r=0.2):
    """Average of P over control volume (i,j) minus the disk, by adaptive
    quadrature, and the volume."""
    x0, x1, y0, y1 = i * h, (i + 1) * h, j * h, (j + 1) * h

    def yint(x):
        dx = x - 0.5
        if abs(dx) >= r:
            return [(y0, y1)]
        lo, hi = 0.5 - math.sqrt(r * r - dx * dx), 0.5 + math.sqrt(r * r - dx * dx)
        out = []
        if y0 < lo:
            out.append((y0, min(y1, lo)))
        if y1 > hi:
            out.append((max(y0, hi), y1))
        return out

    def inner(x, fun):
        return sum(integrate.quad(lambda y: fun(x, y), a, b, epsabs=1e-16, epsrel=1e-14)[0]
                   for (a, b) in yint(x))
    pts = [0.5 - r, 0.5 + r]
    vol = integrate.quad(lambda x: inner(x, lambda x_, y_: 1.0), x0, x1, epsabs=1e-18,
                         epsrel=1e-14, points=[p for p in pts if x0 < p < x1] or None, limit=200)[0]
    tot = integrate.quad(lambda x: inner(x, lambda x_, y_: float(P(x_, y_))), x0, x1,
                         epsabs=1e-18, epsrel=1e-14,
                         points=[p for p in pts if x0 < p < x1] or None, limit=200)[0]
    return tot, vol


def _disk_arc_avg(fun, i, j, h, r=0.2):
    """Average over the circle's arc inside control volume (i,j) of fun(t)."""
    ts = np.linspace(0, 2 * math.pi, 200001)
    x = 0.5 + r * np.cos(ts)
    y = 0.5 + r * np.sin(ts)
    inside = (x >= i * h) & (x <= (i + 1) * h) & (y >= j * h) & (y <= (j + 1) * h)
    num = den = 0.0
    idx = np.flatnonzero(inside)
    if len(idx) == 0:
        return 0.0, 0.0
    # contiguous runs
    runs = np.split(idx, np.flatnonzero(np.diff(idx) > 1) + 1)

    def edge(t_in, t_out):
        for _ in range(80):
            tm = 0.5 * (t_in + t_out)
            xm, ym = 0.5 + r * math.cos(tm), 0.5 + r * math.sin(tm)
            if i * h <= xm <= (i + 1) * h and j * h <= ym <= (j + 1) * h:
                t_in = tm
            else:
                t_out = tm
        return t_in
    for run in runs:
        a = edge(ts[run[0]], ts[run[0] - 1])
        b = edge(ts[run[-1]], ts[min(run[-1] + 1, len(ts) - 1)])
        num += integrate.quad(lambda t: fun(t) * r, a, b, epsabs=1e-18, epsrel=1e-14)[0]
        den += r * (b - a)
    return num, den


def test_plg_rows_exact_on_quartics():
    """Sum beta_k <P>_k + beta_b <<N P>> = <L P>_i for a random quartic, with
    every average computed by adaptive quadrature on the exact geometry."""
    P_ = W.problem_disk()
    n = 32
    lev = G.build_level(P_.dom, n, 0.1)
    d = D.discretize(lev, P_.a, P_.b, P_.c)
    h = lev.h
    P = Poly2.random(4, 21)
    LP = P.L(P_.a, P_.b, P_.c)
    cache = {}

    def avg(fun, name, k):
        key = (name, k)
        if key not in cache:
            j, i = divmod(k, n)
            tot = vol = 0.0
            for kk in np.flatnonzero(lev.owner.ravel() == k):     # merged control volumes
                jj, ii = divmod(int(kk), n)
                t_, v_ = _disk_cell_avg(fun, ii, jj, h)
                tot += t_
                vol += v_
            cache[key] = tot / vol
        return cache[key]

    rows = [k for k in d.lattices if k in lev.cut][:6] + [k for k in d.lattices if k not in lev.cut][:3]
    assert rows
    for k in rows:
        s = sum(bk * avg(P, "u", kj) for bk, kj in zip(d.betas[k], d.lattices[k]))
        if k in d.bd_cells:
            # Neumann on the circle: outward normal of the domain points to the centre
            def dn(t):
                x, y = 0.5 + 0.2 * math.cos(t), 0.5 + 0.2 * math.sin(t)
                return float(-(P.dx()(x, y) * math.cos(t) + P.dy()(x, y) * math.sin(t)))
            num = den = 0.0
            for kk in np.flatnonzero(lev.owner.ravel() == k):
                jj, ii = divmod(int(kk), n)
                a_, b_ = _disk_arc_avg(dn, ii, jj, h)
                num += a_
                den += b_
            row = d.Nmat.getrow(k)
            s += row.data[0] * num / den
        want = avg(LP, "f", k)
        scale = np.abs(d.betas[k]).sum() * 10.0
        assert abs(s - want) < 1e-10 * scale, (divmod(k, n)[::-1], s, want)


# ---------------------------------------------------------------------------
# Convergence and the multigrid solver
# ---------------------------------------------------------------------------
@pytest.mark.slow
def test_disk_fourth_order_convergence():
    P = W.problem_disk()
    errs = []
    for n in (64, 128, 256):
        lev = G.build_level(P.dom, n, 0.1)
        d = D.discretize(lev, P.a, P.b, P.c)
        b = D.rhs(d, D.cell_averages(lev, P.f), D.boundary_data(d, P.u))
        u = spl.spsolve(d.A.tocsc(), b.ravel()).reshape(n, n)
        errs.append(np.abs(u - D.cell_averages(lev, P.u))[lev.present].max())
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) >= 3.7, rates


def _four_disk_errors(kind, n):
    P = W.problem_four_disks(kind)
    lev = G.build_level(P.dom, n, 0.08)
    d = D.discretize(lev, P.a, P.b, P.c)
    b = D.rhs(d, D.cell_averages(lev, P.f), D.boundary_data(d, P.u))
    u = spl.spsolve(d.A.tocsc(), b.ravel()).reshape(n, n)
    e = np.abs(u - D.cell_averages(lev, P.u))
    e[~lev.present] = 0.0
    return [e.max(), (e * lev.vol).sum(), math.sqrt((e * e * lev.vol).sum())]


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["D", "N"])
def test_four_disks_error_magnitudes(kind):
    """The square minus four overlapping disks (Sec. 6): the printed error
    norms pin the magnitude only, because the PLG lattices behind them are
    not given; with Dirichlet data on the disks the oracle's L1/L2 errors
    land within 1.5x of the printed ones and L-inf within 2x, with Neumann
    data within 8x.  Both converge at fourth order between h = 1/64 and
    1/128."""
    rows = {(r[0], int(r[1])): [float(v) for v in r[2:]]
            for r in _golden("four_disks_errors.txt")}
    k = W.DIRICHLET if kind == "D" else W.NEUMANN
    got = {n: _four_disk_errors(k, n) for n in (64, 128)}
    for n, errs in got.items():
        want = rows[(kind, n)]
        bounds = [2.0, 1.5, 1.5] if kind == "D" else [8.0, 8.0, 8.0]
        for g, w, f in zip(errs, want, bounds):
            assert w / f < g < w * f, (kind, n, errs, want)
    for q in range(3):
        assert math.log2(got[64][q] / got[128][q]) > 3.7, (kind, got)


@pytest.mark.parametrize("name", ["disk", "ellipses0", "four_disks"])
def test_irregular_cells_are_plg_and_covered_by_coarse_plg(name):
    """Sec. 5.3: every irregular (cut) cell is a PLG cell, and every fine PLG
    cell is covered by a coarse PLG cell.  A fine cell whose coarse parent
    control volume was merged away (Alg. 1) is covered by the coarse cut cell
    that absorbed it."""
    P = {"disk": W.problem_disk, "ellipses0": lambda: W.problem_ellipses(0),
         "four_disks": lambda: W.problem_four_disks(W.DIRICHLET)}[name]()
    H = M.build_hierarchy(P.dom, 64, P.a, P.b, P.c, min_coarse=16)
    assert H.nl >= 2
    for l, d in enumerate(H.levels):
        cut = (d.lev.ctype != G.REGULAR) & d.lev.present
        assert np.all(d.kind[cut] == D.PLG), (name, l)
        if l + 1 == H.nl:
            continue
        c = H.levels[l + 1]
        js, is_ = np.nonzero(d.kind == D.PLG)
        for j, i in zip(js, is_):
            pj, pi = j // 2, i // 2
            k = pj * c.n + pi if c.lev.present[pj, pi] else int(c.lev.owner[pj, pi])
            assert k >= 0 and c.kind.ravel()[k] == D.PLG, (name, l, i, j)


@pytest.mark.parametrize("n", [64, 128])
def test_block_bandwidth_near_one_curve(n):
    """Lemma 5.2: with the PLG cells of one smooth Jordan curve ordered as in
    Def. 5.1, A22 is a band of width at most 17 plus two corner blocks (the
    curve closes on itself), i.e. its cyclic bandwidth is at most 17.  The
    disk with b = 0 has no other block cells."""
    P = W.problem_disk()
    lev = G.build_level(P.dom, n, 0.1)
    d = D.discretize(lev, 1.0, 0.0, 2.0)
    order = d.plg_order
    m = len(order)
    pos = {k: i for i, k in enumerate(order)}
    A = d.A.tocsr()
    cbw = 0
    for k in order:
        for kk in A.indices[A.indptr[k]:A.indptr[k + 1]]:
            if kk in pos:
                dd = abs(pos[kk] - pos[k])
                cbw = max(cbw, min(dd, m - dd))
    assert 0 < cbw <= 17, cbw


@pytest.mark.parametrize("name,n,mc", [("box", 16, 4), ("disk", 32, 16)])
@pytest.mark.parametrize("gamma", [1, 2])
def test_cycles_converge_to_direct_solve(name, n, mc, gamma):
    P = W.problem_poisson_square() if name == "box" else W.problem_disk()
    H = M.build_hierarchy(P.dom, n, P.a, P.b, P.c, min_coarse=mc)
    d = H.levels[0]
    b = D.rhs(d, D.cell_averages(d.lev, P.f), D.boundary_data(d, P.u))
    ud = spl.spsolve(d.A.tocsc(), b.ravel()).reshape(n, n)
    r = M.solve(H, b, tol=1e-13, gamma=gamma, max_cycles=80)
    assert r.history[-1] < 1e-12
    assert np.abs(r.u - ud).max() < 1e-11 * np.abs(ud).max()
    # residual reduction per cycle stays well below 1
    h = r.history
    assert max(h[k + 1] / h[k] for k in range(1, len(h) - 1)) < 0.7


def test_block_smoother_zeroes_plg_residual_and_lu_is_exact():
    P = W.problem_disk()
    H = M.build_hierarchy(P.dom, 32, P.a, P.b, P.c, min_coarse=16)
    d, lu = H.levels[0], H.lus[0]
    A22 = d.A[lu.order][:, lu.order].toarray()
    t = np.random.default_rng(1).standard_normal(lu.m)
    np.testing.assert_allclose(lu.solve(t), np.linalg.solve(A22, t), rtol=0, atol=1e-12 * np.abs(t).max() * 1e3)
    rng = np.random.default_rng(2)
    u = rng.standard_normal((32, 32)) * d.lev.present
    b = rng.standard_normal((32, 32)) * d.lev.present
    u1 = M.smooth(H, 0, u, b)
    r = M.residual(d, u1, b)
    assert np.abs(r.ravel()[lu.order]).max() < 1e-9 * np.abs(r).max()


def test_variational_property():
    """I_{2h}^h = 2^D (I_h^{2h})^T on a box (Sec. 5.3, after Eq. 5.11)."""
    P = W.problem_poisson_square()
    H = M.build_hierarchy(P.dom, 8, P.a, P.b, P.c, min_coarse=4)
    n, nc = 8, 4
    R = np.column_stack([M.restrict(H, 0, np.eye(n * n)[k].reshape(n, n), zero_plg=False).ravel()
                         for k in range(n * n)])
    Pm = np.column_stack([M.interpolate(H, 0, np.eye(nc * nc)[k].reshape(nc, nc)).ravel()
                          for k in range(nc * nc)])
    np.testing.assert_array_equal(Pm, 4 * R.T)


def test_poisson_vcycle_rate_and_fmg_reduction():
    """V(3,3) on the Poisson unit-square problem down to 4 x 4 converges at
    about 0.4 per cycle; each FMG(3,3) cycle (Alg. 3) on the Table 3 problem
    reduces the residual more than 5 times (Sec. 6.5 reports 7.6; Table 8
    gives an averaged rate of 0.131)."""
    P = W.problem_poisson_square()
    H = M.build_hierarchy(P.dom, 64, P.a, P.b, P.c, min_coarse=4)
    d = H.levels[0]
    b = D.rhs(d, D.cell_averages(d.lev, P.f), D.boundary_data(d, P.u))
    r = M.solve(H, b, tol=1e-10)
    h = r.history
    assert max(h[k + 1] / h[k] for k in range(len(h) - 6, len(h) - 1)) < 0.42
    P = W.problem_table3()
    H = M.build_hierarchy(P.dom, 64, P.a, P.b, P.c, min_coarse=4)
    d = H.levels[0]
    b = D.rhs(d, D.cell_averages(d.lev, P.f), D.boundary_data(d, P.u))
    r = M.solve(H, b, tol=1e-10, method="fmg")
    h = r.history
    red = [h[k] / h[k + 1] for k in range(4)]
    assert min(red) > 5.0, red


def test_w_depth_cycle_shape():
    """The W-cycle truncated to its finest level (w_depth = 1: the finest
    level repeats its coarse-grid correction, coarser levels recurse once).
    It is the V-cycle of Alg. 2 when gamma = 1 and the full W-cycle when
    w_depth covers every level, keeps the exact solution fixed, and on the
    Poisson problem down to 4 x 4 (6 levels) converges like the W-cycle
    (0.292 against 0.288 per cycle) where the V-cycle degrades to 0.404;
    counting the truncation from the coarse end gives about 0.43."""
    P = W.problem_poisson_square()
    H = M.build_hierarchy(P.dom, 128, P.a, P.b, P.c, min_coarse=4)
    assert H.nl == 6
    d = H.levels[0]
    b = D.rhs(d, D.cell_averages(d.lev, P.f), D.boundary_data(d, P.u))
    u0 = np.random.default_rng(3).standard_normal(b.shape) * d.lev.present
    np.testing.assert_array_equal(M.cycle(H, 0, u0, b, 3, 3, 1, 1), M.cycle(H, 0, u0, b, 3, 3, 1))
    np.testing.assert_array_equal(M.cycle(H, 0, u0, b, 3, 3, 2, H.nl), M.cycle(H, 0, u0, b, 3, 3, 2))
    ustar = spl.spsolve(d.A.tocsc(), b.ravel()).reshape(b.shape)
    rates = {}
    for wd in (1, 0):
        r = M.solve(H, b, tol=1e-11, gamma=2, w_depth=wd)
        h = r.history
        rates[wd] = max(h[k + 1] / h[k] for k in range(len(h) - 5, len(h) - 1))
    r = M.solve(H, b, tol=1e-11, gamma=1)
    h = r.history
    rate_v = max(h[k + 1] / h[k] for k in range(len(h) - 5, len(h) - 1))
    assert rates[1] < 0.31 and rates[0] < 0.31, rates
    assert rate_v > 0.38, rate_v
    np.testing.assert_allclose(M.cycle(H, 0, ustar, b, 3, 3, 2, 1), ustar,
                               atol=1e-10 * np.abs(ustar).max())


# ---------------------------------------------------------------------------
# Multicolour Gauss-Seidel variant of the block smoother (outside the paper)
# ---------------------------------------------------------------------------
def _sfv_mask(H, l):
    d = H.levels[l]
    blk = np.zeros(d.n * d.n, dtype=bool)
    blk[H.lus[l].order] = True
    return (d.kind.ravel() == D.SFV) & ~blk


@pytest.mark.parametrize("name,n", [("table3", 24), ("disk", 32), ("four_disks", 32)])
def test_mcgs_colour_classes_do_not_couple(name, n):
    """No two SFV cells of one colour class are coupled by the operator, wall
    ghosts included (b = 0: 4 classes, b != 0: 15), so a class can be relaxed
    all at once and in place."""
    P = (W.problem_table3() if name == "table3" else W.problem_disk() if name == "disk"
         else W.problem_four_disks(W.NEUMANN))
    H = M.build_hierarchy(P.dom, n, P.a, P.b, P.c, min_coarse=n // 2, smoother="mcgs", omega=0.6)
    d = H.levels[0]
    col = M.colours(d).ravel()
    assert col.max() + 1 == (4 if P.b == 0 else 15)
    m = _sfv_mask(H, 0)
    A = d.A.tocoo()
    same = (col[A.row] == col[A.col]) & (A.row != A.col) & m[A.row] & m[A.col] & (A.data != 0)
    assert not same.any()


@pytest.mark.parametrize("name,n", [("table3", 24), ("disk", 32), ("box_cross", 20)])
def test_mcgs_sweep_is_the_colour_ordered_splitting(name, n):
    """One multicolour sweep equals, on the SFV unknowns, the splitting
    u + (D / omega I + L)^-1 (b - A u) with L the couplings from earlier to
    later colours (a block Gauss-Seidel step in colour order, solved here by
    scipy's sparse triangular solve), followed by the exact block solve."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    if name == "table3":
        P = W.problem_table3()
    elif name == "disk":
        P = W.problem_disk()
    else:
        u = W.u_expcos()
        dom = W.Domain(box_bc=(W.BC(), W.BC(W.NEUMANN, 0, 1), W.BC(), W.BC(W.ROBIN, 1.0, 0.5)))
        P = W.Problem("box_cross", dom, 1.0, 0.5, 2.0, u, W.apply_L(u, 1.0, 0.5, 2.0))
    om = 0.6
    H = M.build_hierarchy(P.dom, n, P.a, P.b, P.c, min_coarse=n // 2, smoother="mcgs", omega=om)
    d = H.levels[0]
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal((n, n)) * d.lev.present
    b0 = rng.standard_normal((n, n)) * d.lev.present
    got = M.smooth(H, 0, u0, b0).ravel()
    m = _sfv_mask(H, 0)
    col = M.colours(d).ravel()
    S = np.nonzero(m)[0]
    S = S[np.argsort(col[S], kind="stable")]               # SFV cells in colour order
    r0 = b0.ravel() - d.A @ u0.ravel()
    ASS = d.A[S][:, S].tocoo()
    low = col[S][ASS.row] > col[S][ASS.col]
    Lm = sp.csr_matrix((ASS.data[low], (ASS.row[low], ASS.col[low])), shape=(len(S), len(S)))
    Mat = (sp.identity(len(S)) * (d.diag / om) + Lm).tocsr()
    delta = spl.spsolve_triangular(Mat, r0[S], lower=True)
    want = u0.ravel().copy()
    want[S] += delta
    # then the exact block solve on the new SFV values (Eq. 5.8), as in smooth()
    rows = H.lus[0].order
    if len(rows):
        w1 = want.copy()
        w1[rows] = 0.0
        want[rows] = H.lus[0].solve(b0.ravel()[rows] - d.A[rows] @ w1)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_mcgs_two_grid_rate():
    """Two-grid spectral radius (Eq. 5.12) of the multicolour variant on the
    Table 3 problem at N = 64: with omega = 0.6 two pre- and post-sweeps
    reduce errors faster than the paper's Jacobi smoother with two (Table 2:
    0.513) and about as fast as Jacobi with three (0.378); undamped
    (omega = 1) the variant diverges, because the fourth-order stencil's far
    weights have the sign opposite to the centre."""
    P = W.problem_table3()
    n = 64
    v0 = np.random.default_rng(0).standard_normal(n * n)

    def rho(om, nu):
        H = M.build_hierarchy(P.dom, n, P.a, P.b, P.c, min_coarse=n // 2, smoother="mcgs", omega=om)
        op = M.two_grid_operator(H, nu, nu)
        w = eigs(op, k=1, which="LM", return_eigenvectors=False, tol=1e-7, maxiter=20000, v0=v0)
        return abs(w[0])

    r22 = rho(0.6, 2)
    assert 0.30 < r22 < 0.40, r22
    assert rho(1.0, 1) > 1.0


# ---------------------------------------------------------------------------
# Sec. 6.2: the square minus a flower (a boundary that is not an ellipse)
# ---------------------------------------------------------------------------
def test_flower_error_magnitudes():
    """The oracle's direct solve of the flower problem (Poisson, Dirichlet on
    the square, Neumann on r = 0.25 + 0.05 cos 6 theta, eps = 0.02) at
    h = 1/40, 1/80, 1/160 has L-inf, L1 and L2 errors within 2.5x of the
    printed Table 4 (3.64e-7 / 2.29e-8 / 1.29e-9 in L-inf against 5.42e-7 /
    1.72e-8 / 1.29e-9) and converges at fourth order; magnitude only, since
    the lattices behind the table are not given."""
    P = W.problem_flower()
    printed = {int(r[0]): [float(v) for v in r[1:]] for r in _golden("flower_errors.txt")}
    errs = {}
    for n in (40, 80, 160):
        lev = G.build_level(P.dom, n, 0.02)
        assert lev.resolved
        d = D.discretize(lev, P.a, P.b, P.c)
        b = D.rhs(d, D.cell_averages(lev, P.f), D.boundary_data(d, P.u))
        u = spl.spsolve(d.A.tocsc(), b.ravel()).reshape(n, n)
        e = np.abs(u - D.cell_averages(lev, P.u))
        e[~lev.present] = 0.0
        errs[n] = np.array([e.max(), (e * lev.vol).sum(), math.sqrt((e * e * lev.vol).sum())])
        for got, want in zip(errs[n], printed[n]):
            assert want / 2.5 < got < want * 2.5, (n, errs[n], printed[n])
    rate = np.log2(errs[80] / errs[160])
    assert np.all(rate > 3.5), rate


def test_flower_two_grid_spectral_radius():
    """Table 2, flower row, at N = 80 (two grids, eps = 0.02): with two and
    three sweeps the spectral radius of TG (Eq. 5.12) equals the printed 0.414
    and 0.283 to all three digits; with fewer sweeps it is within 10 % below
    the printed values (1.014 / 0.672 / 0.474 against 1.069 / 0.698 / 0.483:
    the slowest mode of one sweep lives at the cut cells, whose lattices
    differ from the paper's)."""
    P = W.problem_flower()
    n = 80
    H = M.build_hierarchy(P.dom, n, P.a, P.b, P.c, eps=0.02, min_coarse=n // 2)
    assert H.nl == 2
    for nu1, nu2, want in _golden("table2_flower.txt"):
        op = M.two_grid_operator(H, int(nu1), int(nu2))
        v0 = np.random.default_rng(0).standard_normal(n * n)
        w = abs(eigs(op, k=1, which="LM", return_eigenvectors=False, tol=1e-9, maxiter=20000, v0=v0)[0])
        if int(nu1) >= 2 and int(nu2) >= 2:
            assert round(w, 3) == float(want), (nu1, nu2, w)
        else:
            assert 0.9 * float(want) < w <= float(want) + 1e-3, (nu1, nu2, w)


# ---------------------------------------------------------------------------
# Sec. 6.1, the rotated square: the cross-derivative term and PLG rows on a
# boundary that is not aligned with the grid
# ---------------------------------------------------------------------------
def _rotated_norms(hinv):
    P = W.problem_rotated_square()
    n = int(round(1.5 * hinv))          # the box has side 1.5
    lev = G.build_level(P.dom, n, 0.1)
    assert lev.resolved
    assert abs(lev.vol.sum() - 1.0) < 1e-12      # the area of Omega_r
    d = D.discretize(lev, P.a, P.b, P.c)
    b = D.rhs(d, D.cell_averages(lev, P.f), D.boundary_data(d, P.u))
    u = spl.spsolve(d.A.tocsc(), b.ravel()).reshape(n, n)
    e = np.abs(u - D.cell_averages(lev, P.u))
    e[~lev.present] = 0.0
    return np.array([e.max(), (e * lev.vol).sum(), math.sqrt((e * e * lev.vol).sum())])


def test_rotated_square_error_norms():
    """Table 3, lower half: at h = 1/128 the oracle's L-inf, L1 and L2 errors
    on Omega_r are within 5 % of the printed 8.85e-9, 2.95e-9, 3.72e-9
    (8.64e-9, 2.94e-9, 3.67e-9); at h = 1/64 the L1 and L2 errors are within
    15 % (5.07e-8, 6.37e-8) and the L-inf error within 10x (9.2e-7 against
    1.35e-7: one cell of a coarse lattice); fourth order in L1 and L2."""
    printed = {int(r[0]): np.array([float(v) for v in r[1:]]) for r in _golden("table3_rotated_square.txt")}
    e64, e128 = _rotated_norms(64), _rotated_norms(128)
    assert np.all(np.abs(e128 / printed[128] - 1.0) < 0.05), (e128, printed[128])
    assert np.all(np.abs(e64[1:] / printed[64][1:] - 1.0) < 0.15), (e64, printed[64])
    assert printed[64][0] / 10 < e64[0] < printed[64][0] * 10
    rate = np.log2(e64[1:] / e128[1:])
    assert np.all(rate > 3.9), rate


def test_rotated_square_two_grid_spectral_radius():
    """Table 2, rotated-square row, at h = 1/64 (two grids): the oracle's
    spectral radii of TG (Eq. 5.12) are the printed ones to within one unit
    in the third digit (1.109 / 0.744 / 0.523 / 0.421 / 0.275 against
    1.110 / 0.745 / 0.523 / 0.421 / 0.275)."""
    P = W.problem_rotated_square()
    n = 96
    H = M.build_hierarchy(P.dom, n, P.a, P.b, P.c, min_coarse=n // 2)
    assert H.nl == 2
    for nu1, nu2, want in _golden("table2_rotated_square.txt"):
        op = M.two_grid_operator(H, int(nu1), int(nu2))
        v0 = np.random.default_rng(0).standard_normal(n * n)
        w = abs(eigs(op, k=1, which="LM", return_eigenvectors=False, tol=1e-6, maxiter=20000, v0=v0)[0])
        assert abs(w - float(want)) <= 1.5e-3, (nu1, nu2, w)


# ---------------------------------------------------------------------------
# PLG fits and lattices against independent computations
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["disk", "ellipses0"])
def test_boundary_fits_are_the_closed_form_of_lemma_4_4(name):
    """For every PLG cell with boundary data, beta is the minimiser of
    ||beta||_{W^-1} under M beta = phi with W^-1 = diag(w), w_k = max(|j_k -
    i|, 1/2), w_b = 1/2 (Eq. 4.17-4.18): equal to the closed form W M^T (M W
    M^T)^-1 phi of Lemma 4.4, computed here by a normal-equations solve (the
    oracle uses a scaled least-squares solve), and no null-space move of M
    makes the W^-1 norm smaller."""
    P = W.problem_disk() if name == "disk" else W.problem_ellipses(0)
    n = 64
    lev = G.build_level(P.dom, n, 0.1)
    d = D.discretize(lev, P.a, P.b, P.c)
    rng = np.random.default_rng(9)
    checked = 0
    for k in d.bd_cells:
        lat = d.lattices[k]
        j0, i0 = divmod(k, n)
        M = np.column_stack([D.sample_column(lev, k, kj) for kj in lat] + [D._boundary_column(lev, k)])
        phi = D._L_column(lev, k, P.a, P.b, P.c)
        w = np.array([max(math.hypot(kj % n - i0, kj // n - j0), 0.5) for kj in lat] + [0.5])
        Wd = 1.0 / w
        want = Wd * (M.T @ np.linalg.solve((M * Wd[None, :]) @ M.T, phi))
        got = np.array(list(d.betas[k]) + [d.Nmat[k, 4 * n + d.bd_cells.index(k)]])
        assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max(), k
        # minimality: any null-space direction z of M increases the W^-1 norm
        ns = np.linalg.svd(M)[2][M.shape[0]:]
        base = np.sum(w * want ** 2)
        for z in ns:
            for t in (1e-3, -1e-3):
                cand = want + t * np.abs(want).max() * z
                assert np.sum(w * cand ** 2) > base
        checked += 1
        if checked >= 40:
            break
    assert checked >= 20


def _lattice_cost(lev, ki, cells, orient):
    n = lev.n
    j0, i0 = divmod(ki, n)
    tot = 0
    for kj in cells:
        jj, ii = divmod(kj, n)
        cut = lev.ctype[jj, ii] != G.REGULAR and kj != ki
        tot += (ii - i0) ** 2 + (jj - j0) ** 2 + (D.CUT_PENALTY if cut else 0)
    return tot


@pytest.mark.parametrize("name", ["disk", "flower"])
def test_lattice_is_the_cheapest_five_line_set_by_brute_force(name):
    """The lattice rule (a reading of Def. 4.3) restated as an exhaustive
    search: over both orientations and every assignment of the counts
    5, 4, 3, 2, 1 to distinct lines of the 9 x 9 box, each line taking its
    cheapest present cells, the least total cost.  The oracle's dynamic
    programme must reach that cost, with five lines of those counts."""
    from itertools import permutations
    if name == "disk":
        P, eps = W.problem_disk(), 0.1
    else:
        P, eps = W.problem_flower(), 0.02
    n = 64
    lev = G.build_level(P.dom, n, eps)
    d = D.discretize(lev, P.a, P.b, P.c)
    plg = sorted(d.lattices)[::max(1, len(d.lattices) // 25)]
    R = D.PLG_RADIUS
    for ki in plg:
        j0, i0 = divmod(ki, n)
        best = None
        for orient in (0, 1):
            lines = {}
            for v in range(-R, R + 1):
                cs = []
                for u in range(-R, R + 1):
                    di, dj = (u, v) if orient == 0 else (v, u)
                    i, j = i0 + di, j0 + dj
                    if 0 <= i < n and 0 <= j < n and lev.present[j, i]:
                        cut = lev.ctype[j, i] != G.REGULAR and (di, dj) != (0, 0)
                        cs.append(u * u + v * v + (D.CUT_PENALTY if cut else 0))
                lines[v] = sorted(cs)
            for pick in permutations(range(-R, R + 1), 5):
                if any(len(lines[v]) < c for v, c in zip(pick, (5, 4, 3, 2, 1))):
                    continue
                cost = sum(sum(lines[v][:c]) for v, c in zip(pick, (5, 4, 3, 2, 1)))
                best = cost if best is None else min(best, cost)
        lat = d.lattices[ki]
        if best is None:      # no lattice in the 9 x 9 box: the oracle searched a larger one
            continue
        rows = sorted(collections_counter(kj // n for kj in lat).values())
        cols = sorted(collections_counter(kj % n for kj in lat).values())
        orient = 0 if rows == [1, 2, 3, 4, 5] else 1
        assert rows == [1, 2, 3, 4, 5] or cols == [1, 2, 3, 4, 5], ki
        if _lattice_cost(lev, ki, lat, orient) != best:
            # only an alternative lattice taken for the sign: the cheapest lattice's row
            # then has a coefficient of its own cell that is not negative
            first = D.choose_lattice(lev, ki)
            beta, _ = D.fit_beta(lev, ki, first, P.a, P.b, P.c, ki in d.bd_cells)
            assert D.row_diagonal(ki, first, beta) >= 0.0, ki
            assert D.row_diagonal(ki, lat, d.betas[ki]) < 0.0, ki


def collections_counter(it):
    from collections import Counter
    return Counter(it)


def _brute_lattice_cost(lev, ki, R):
    """The least cost of a five-line set with counts 5, 4, 3, 2, 1 in the box
    of half-width R around cell ki, over both orientations and every
    assignment of the counts to distinct lines (each line taking its
    cheapest present cells); None if the box holds no such set."""
    from itertools import permutations
    n = lev.n
    j0, i0 = divmod(ki, n)
    best = None
    for orient in (0, 1):
        lines = {}
        for v in range(-R, R + 1):
            cs = []
            for u in range(-R, R + 1):
                di, dj = (u, v) if orient == 0 else (v, u)
                i, j = i0 + di, j0 + dj
                if 0 <= i < n and 0 <= j < n and lev.present[j, i]:
                    cut = lev.ctype[j, i] != G.REGULAR and (di, dj) != (0, 0)
                    cs.append(u * u + v * v + (D.CUT_PENALTY if cut else 0))
            lines[v] = sorted(cs)
        usable = [v for v in lines if lines[v]]
        for pick in permutations(usable, 5):
            if any(len(lines[v]) < c for v, c in zip(pick, (5, 4, 3, 2, 1))):
                continue
            cost = sum(sum(lines[v][:c]) for v, c in zip(pick, (5, 4, 3, 2, 1)))
            best = cost if best is None else min(best, cost)
    return best


@pytest.mark.parametrize("name,n", [("disk", 64), ("disk", 128), ("four_disks", 64), ("flower", 80),
                                    ("ellipses0", 128), ("ellipses1", 128), ("ellipses2", 128),
                                    ("ellipses3", 128)])
def test_plg_rows_have_the_sign_of_the_sfv_centre_weight(name, n):
    """On the validation domains every PLG row of the finest level gives its
    own cell a negative coefficient, the sign of the SFV centre weight
    -5(a + c)/(2 h^2) of Eq. 4.7, of between a fifth and five times that
    weight (measured: 0.29 to 3.04).  The lattice rule is not given by the
    paper; this checks its rows against the regular stencil rather than
    against itself.  It does not hold everywhere: on some random unions and
    batch domains a few rows per level keep a non-negative coefficient that
    no alternative lattice mends."""
    if name == "disk":
        P, eps = W.problem_disk(), 0.1
    elif name == "four_disks":
        P, eps = W.problem_four_disks(W.NEUMANN), 0.08
    elif name == "flower":
        P, eps = W.problem_flower(), 0.02
    else:
        P, eps = W.problem_ellipses(int(name[8:])), 0.1
    lev = G.build_level(P.dom, n, eps)
    d = D.discretize(lev, P.a, P.b, P.c)
    centre = -5.0 * (P.a + P.c) / (2.0 * lev.h ** 2)
    assert d.lattices
    for k, lat in d.lattices.items():
        own = D.row_diagonal(k, lat, d.betas[k])
        assert own < 0.0, (k, own)
        assert 0.2 < own / centre < 5.0, (k, own / centre)


def test_far_lattices_at_wedge_tips_are_the_cheapest_by_brute_force():
    """Near the tip of a thin wedge between two overlapping ellipses (union
    52 at 256^2) the 13 x 13 box holds no five-line set, and the rule's
    search goes on to larger boxes.  For every such cell the
    exhaustive search finds no set in the 9 x 9 to 13 x 13 boxes either, the
    oracle's lattice lies in the first larger box that holds one and has the
    least cost there, and the cell's row has a negative own coefficient."""
    P = W.problem_ellipses(52)
    n = 256
    lev = G.build_level(P.dom, n, 0.1)
    d = D.discretize(lev, P.a, P.b, P.c)
    far = {}
    for ki, lat in d.lattices.items():
        j0, i0 = divmod(ki, n)
        ext = max(max(abs(kj % n - i0), abs(kj // n - j0)) for kj in lat)
        if ext > D.PLG_RADIUS_MAX:
            far[ki] = ext
    assert far
    for ki, ext in sorted(far.items()):
        for R in range(D.PLG_RADIUS, ext):
            assert _brute_lattice_cost(lev, ki, R) is None, (ki, R)
        lat = d.lattices[ki]
        rows = sorted(collections_counter(kj // n for kj in lat).values())
        orient = 0 if rows == [1, 2, 3, 4, 5] else 1
        assert _lattice_cost(lev, ki, lat, orient) == _brute_lattice_cost(lev, ki, ext), ki
        assert D.row_diagonal(ki, lat, d.betas[ki]) < 0.0, ki


def test_alternative_lattices_mend_a_diverging_union(monkeypatch):
    """Alternative lattices on ellipse union 30 at 128^2 (three overlapping ellipses): with the
    cheapest lattice alone, PLG rows of its 64^2 and 32^2 levels have a
    coefficient of their own cell that is not negative, and the W(4,4)
    iteration diverges.  With the alternatives every PLG row of every level
    has a negative own coefficient, and the iteration reaches 1e-10 in at
    most 20 cycles."""
    P = W.problem_ellipses(30)

    def run():
        H = M.build_hierarchy(P.dom, 128, P.a, P.b, P.c, min_coarse=32)
        d = H.levels[0]
        b = D.rhs(d, D.cell_averages(d.lev, P.f), D.boundary_data(d, P.u))
        r = M.solve(H, b, tol=1e-10, gamma=2, w_depth=1, nu1=4, nu2=4, max_cycles=20)
        own = [D.row_diagonal(k, lat, lv.betas[k]) for lv in H.levels for k, lat in lv.lattices.items()]
        return r.history[-1], max(own)

    res, worst = run()
    assert res < 1e-10 and worst < 0.0
    with monkeypatch.context() as mp:
        mp.setattr(D, "lattice_candidates", lambda lev, k: [])
        res0, worst0 = run()
    assert worst0 >= 0.0 and not res0 < 1e3, (res0, worst0)
