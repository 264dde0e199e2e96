"""Library checks that need no GPU: the shared library loads and exports every
entry point of include/ccmg.h, and its host-side setup (geometry, Alg. 1,
Def. 4.1, PLG fits) agrees with the oracle's tables."""
import os
import re

import numpy as np
import pytest

import __graft_entry__
from oracle import discretize as D
from oracle import geometry as G
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    from paper_2601_02975_gb300 import _lib
    return _lib


def test_exports_every_declared_symbol(lib):
    text = open(os.path.join(ROOT, "include", "ccmg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(cc_[a-z_0-9]+)\s*\(", text))
    assert len(names) >= 20
    L = lib.lib()
    for name in sorted(names):
        assert hasattr(L, name), name
    assert names == set(lib._SIGS), names ^ set(lib._SIGS)


def _host(P, n, **kw):
    from paper_2601_02975_gb300 import Hierarchy, default_options
    return Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n, default_options(host_only=1, **kw))


@pytest.mark.parametrize("name,n", [("disk", 32), ("disk", 64), ("ellipses0", 64),
                                    ("ellipses3", 96), ("box_cross", 24), ("four_disks_N", 64),
                                    ("ellipses0", 256), ("waist", 48)])
def test_setup_tables_match_oracle(lib, name, n):
    """The finest level's cell types, volumes, kinds, lattices, fits and
    boundary coefficients equal the oracle's.  "waist": two disks overlapping
    by a sliver, whose waist splits a cell into two components (Alg. 1)."""
    if name == "waist":
        u = W.u_expcos()
        dom = W.Domain(holes=[W.Ellipse(0.3, 0.507, 0.2, 0.2), W.Ellipse(0.6999, 0.507, 0.2, 0.2)],
                       hole_bc=[W.BC(), W.BC(W.NEUMANN, 0, 1)])
        P = W.Problem("waist", dom, 1.0, 0.3, 1.5, u, W.apply_L(u, 1.0, 0.3, 1.5))
    elif name == "disk":
        P = W.problem_disk()
    elif name == "four_disks_N":
        P = W.problem_four_disks(W.NEUMANN)
    elif name.startswith("ellipses"):
        P = W.problem_ellipses(int(name[-1]))
    else:
        P = W.Problem("box_cross", W.Domain(box_bc=(W.BC(), W.BC(W.NEUMANN, 0, 1), W.BC(),
                                                     W.BC(W.ROBIN, 1.0, 0.5))),
                      1.0, 0.5, 2.0, W.u_expcos(), W.apply_L(W.u_expcos(), 1.0, 0.5, 2.0))
    H = _host(P, n, min_coarse_n=n)
    lev = G.build_level(P.dom, n, 0.1)
    d = D.discretize(lev, P.a, P.b, P.c)
    typ, kind, vol = H.cell_types()
    np.testing.assert_array_equal(kind, d.kind)
    np.testing.assert_array_equal(typ, lev.ctype)
    assert np.abs(vol - lev.vol).max() < 1e-15
    _, lat, beta = H.level_tables(0)
    plg = sorted(d.lattices)
    assert len(plg) == len(lat)
    for r, k in enumerate(plg):
        np.testing.assert_array_equal(lat[r], d.lattices[k])
        want = np.array(list(d.betas[k]))
        scale = np.abs(want).max()
        assert np.abs(beta[r, :15] - want).max() < 1e-11 * scale
        if k in d.bd_cells:
            bb = d.Nmat[k, 4 * n + d.bd_cells.index(k)]
            assert abs(beta[r, 15] - bb) < 1e-11 * max(1.0, abs(bb))
    assert H.info.n_bd == len(d.bd_cells)
    H.close()


def test_quadrature_rules(lib):
    """The exported rules integrate polynomials like the oracle's geometry."""
    P = W.problem_ellipses(0)
    n = 64
    H = _host(P, n, min_coarse_n=n)
    q = H.quadrature_nodes()
    lev = G.build_level(P.dom, n, 0.1)
    w = np.add.reduceat(q["vnode"][:, 2], q["vptr"][:-1])
    np.testing.assert_allclose(w, 1.0, atol=1e-12)
    poly = lambda x, y: (x - 0.3) ** 4 - 2 * (x - 0.5) * (y - 0.4) ** 3 + y
    want = D.cell_averages(lev, poly)
    vn = q["vnode"]
    got = np.add.reduceat(poly(vn[:, 0], vn[:, 1]) * vn[:, 2], q["vptr"][:-1])
    assert np.abs(got - want.ravel()[q["cell"]]).max() < 1e-12
    bw = np.add.reduceat(q["bnode"][:, 4], q["bptr"][:-1])
    np.testing.assert_allclose(bw, 1.0, atol=1e-12)
    H.close()


@pytest.mark.parametrize("case", ["not_elliptic", "too_small", "hole_outside", "bad_bc_count"])
def test_setup_rejects_bad_arguments(lib, case):
    from paper_2601_02975_gb300 import CCError, Hierarchy, default_options
    P = W.problem_disk()
    a, b, c, n = P.a, P.b, P.c, 32
    dom = P.dom
    bcs = list(dom.box_bc) + list(dom.hole_bc)
    if case == "not_elliptic":
        b = 3.0
    elif case == "too_small":
        n = 2
    elif case == "hole_outside":
        dom = W.Domain(holes=[W.Ellipse(0.95, 0.5, 0.2, 0.2)], hole_bc=[W.BC()])
        bcs = list(dom.box_bc) + list(dom.hole_bc)
    else:
        bcs = bcs[:3]
    with pytest.raises(CCError) as ei:
        Hierarchy(dom, a, b, c, bcs, n, default_options(host_only=1))
    assert ei.value.status in (1, 2)


def test_rejected_setup_says_which_step(lib):
    """A problem the setup rejects names the step in cc_last_error_string and
    in the Python error: ellipse union 58 at 2048^2 has cells near a wedge
    tip with no five-line set up to 25 x 25 (the far search of the lattice
    rule ends there), and union 52 at 256^2, whose cells need boxes of
    15 x 15, sets up."""
    from paper_2601_02975_gb300 import CCError
    P = W.problem_ellipses(58)
    with pytest.raises(CCError) as ei:
        _host(P, 2048, min_coarse_n=32)
    assert ei.value.status == 3
    assert "no poised lattice" in str(ei.value)
    assert lib.lib().cc_last_error_string().decode() == "no poised lattice for a PLG cell"
    P = W.problem_ellipses(52)
    H = _host(P, 256, min_coarse_n=32)
    assert H.info.n_levels >= 2
    H.close()


def test_new_options_are_checked(lib):
    """hole_cells, serve_slots, w_depth, fmg_cycle and krylov are validated
    by cc_setup (krylov: 0..32, with a V or W cycle); cc_serve_budget rejects
    a negative cap."""
    from paper_2601_02975_gb300 import CCError, Hierarchy, default_options, serve_budget
    P = W.problem_disk()
    for kw in ({"hole_cells": 0.0}, {"hole_cells": -1.0}, {"serve_slots": 0}, {"w_depth": -1},
               {"fmg_cycle": 3}, {"krylov": -1}, {"krylov": 33, "precision": 1},
               {"krylov": 8, "precision": 1, "cycle": 3}):
        with pytest.raises(CCError) as ei:
            Hierarchy.from_domain(P.dom, P.a, P.b, P.c, 32, default_options(host_only=1, **kw))
        assert ei.value.status == 1, kw
    with pytest.raises(CCError):
        serve_budget(-1)
    serve_budget(0)
    for prec in (0, 1):
        H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, 32,
                                  default_options(host_only=1, krylov=32, precision=prec, cycle=2))
        H.close()


def test_hole_cells_sets_the_depth(lib):
    """The coarse-level hole resolution decides where coarsening stops, the
    same way in the library and in the oracle: the disk (r = 0.2) keeps 16^2
    with 2 cells (0.2 >= 2/16) and stops at 32^2 with 3.5 cells."""
    from paper_2601_02975_gb300 import Hierarchy, default_options
    from oracle import multigrid as M
    P = W.problem_disk()
    for hc, want in ((2.0, [64, 32, 16]), (3.5, [64, 32])):
        H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, 64,
                                  default_options(host_only=1, min_coarse_n=8, hole_cells=hc))
        assert list(H.info.level_n[:H.info.n_levels]) == want
        levels = [64]
        n = 64
        while n // 2 >= 8 and 0.2 >= hc / (n // 2):
            n //= 2
            levels.append(n)
        assert levels == want
    O = M.build_hierarchy(P.dom, 32, P.a, P.b, P.c, min_coarse=8, hole_cells=3.5)
    assert [d.n for d in O.levels] == [32]


def test_batch_generator_properties():
    """The batch workload generator keeps its stated ranges: N a power of two
    in 64..1024, 1-8 holes with semi-axes in [0.03, 0.15] whose bounding
    circles keep 0.02 from the box and from one another, a, c in [0.5, 2],
    b^2 < 3ac, Dirichlet box, g = 0; and it is seeded."""
    import math
    seen = set()
    for k in range(40):
        P, n = W.problem_batch(k)
        assert n in (64, 128, 256, 512, 1024)
        seen.add(n)
        hs = P.dom.holes
        assert 1 <= len(hs) <= 8
        for i, e in enumerate(hs):
            R = max(e.r1, e.r2)
            assert 0.03 <= min(e.r1, e.r2) and R <= 0.15
            assert min(e.cx, e.cy, 1 - e.cx, 1 - e.cy) - R >= 0.02
            for o in hs[:i]:
                assert math.hypot(e.cx - o.cx, e.cy - o.cy) - R - max(o.r1, o.r2) >= 0.02
        assert 0.5 <= P.a <= 2 and 0.5 <= P.c <= 2 and P.b * P.b < 3 * P.a * P.c
        assert all(bc.kind == W.DIRICHLET for bc in P.dom.box_bc)
        assert not P.exact and len(P.u.terms) == 0
        P2, n2 = W.problem_batch(k)
        assert n2 == n and P2.dom.holes == hs and P2.a == P.a
    assert len(seen) >= 4


def test_large_block_inverse_is_exact(lib):
    """The 2380-cell block of the 512^2 disk level is inverted with the
    threaded Gauss-Jordan elimination: the normwise backward error of the
    exact block solve, measured at setup, stays at rounding level."""
    P = W.problem_disk()
    H = _host(P, 512, min_coarse_n=32)
    assert H.info.n_block > 2000
    assert H.info.block_error < 1e-14, H.info.block_error
    H.close()


def test_default_options_match_the_header(lib):
    """cc_default_options fills the defaults that include/ccmg.h documents, read
    back through the binding's copy of the struct (a layout mismatch between
    the two would show as wrong values here)."""
    from paper_2601_02975_gb300 import default_options
    o = default_options()
    want = {"eps": 0.1, "nu1": 3, "nu2": 3, "omega": 0.5, "cycle": 1, "min_coarse_n": 4,
            "precision": 0, "max_cycles": 100, "use_graphs": 1, "host_only": 0, "fmg_cycle": 1,
            "w_depth": 0, "serve_slots": 4, "cache": 0, "hole_cells": 2.0, "krylov": 0}
    got = {k: getattr(o, k) for k in want}
    assert got == want, got
    o = default_options(krylov=7, hole_cells=3.5)
    assert (o.krylov, o.hole_cells, o.cache) == (7, 3.5, 0)


@pytest.mark.parametrize("name,n,mc", [("disk", 128, 16), ("four_disks_D", 128, 16),
                                       ("batch8", 256, 32), ("ellipses30", 256, 32),
                                       ("batch4", 64, 8), ("ellipses15", 128, 32),
                                       ("ellipses52", 256, 32)])
def test_coarse_level_tables_match_oracle(lib, name, n, mc):
    """Every level of the hierarchy (Eq. 5.9: each coarse level discretised
    on its own grid) has the same cell kinds, lattices and PLG coefficients
    in the library and in the oracle, and both stop coarsening at the same
    level.  Problem 8 of the batch workload is the one whose coarsest level
    has PLG rows with a positive diagonal that no alternative lattice mends:
    both sides build the same rows.  Ellipse union 30 has such rows on its
    64^2 and 32^2 levels that alternative lattices do mend: both sides
    pick the same alternatives.  Problem 4 of the batch and union 15 have
    finest-level cut cells of two components (Alg. 1): both sides keep the
    same one, move the other to the same neighbour, and build the same
    cells, volumes and rows.  Union 52 has cells near a wedge tip whose
    13 x 13 box holds no lattice: both sides find the same one in a larger
    box."""
    from oracle import multigrid as M
    if name == "disk":
        P = W.problem_disk()
    elif name == "four_disks_D":
        P = W.problem_four_disks(W.DIRICHLET)
    elif name.startswith("ellipses"):
        P = W.problem_ellipses(int(name[8:]))
    else:
        P, n2 = W.problem_batch(int(name[5:]))
        assert n2 == n
    H = _host(P, n, min_coarse_n=mc)
    O = M.build_hierarchy(P.dom, n, P.a, P.b, P.c, min_coarse=mc)
    assert H.info.n_levels == O.nl
    typ, _, vol = H.cell_types()
    np.testing.assert_array_equal(typ, O.levels[0].lev.ctype)
    assert np.abs(vol - O.levels[0].lev.vol).max() < 1e-15
    for l, d in enumerate(O.levels):
        kind, lat, beta = H.level_tables(l)
        np.testing.assert_array_equal(kind, d.kind)
        plg = sorted(d.lattices)
        assert len(plg) == len(lat), l
        for r, k in enumerate(plg):
            np.testing.assert_array_equal(lat[r], d.lattices[k])
            want = np.array(list(d.betas[k]))
            assert np.abs(beta[r, :15] - want).max() < 1e-11 * np.abs(want).max(), (l, k)
    H.close()


@pytest.mark.parametrize("n", [40, 80])
def test_flower_tables_match_oracle(lib, n):
    """The flower of Sec. 6.2 (a polar curve, eps = 0.02): the library's cell
    types, volumes, lattices and fit coefficients equal the oracle's,
    including at the tips and valleys that lie on grid lines (touched, not
    crossed)."""
    P = W.problem_flower()
    H = _host(P, n, min_coarse_n=n, eps=0.02)
    lev = G.build_level(P.dom, n, 0.02)
    d = D.discretize(lev, P.a, P.b, P.c)
    typ, kind, vol = H.cell_types()
    np.testing.assert_array_equal(kind, d.kind)
    np.testing.assert_array_equal(typ, lev.ctype)
    assert np.abs(vol - lev.vol).max() < 1e-15
    _, lat, beta = H.level_tables(0)
    plg = sorted(d.lattices)
    assert len(plg) == len(lat)
    for r, k in enumerate(plg):
        np.testing.assert_array_equal(lat[r], d.lattices[k])
        want = np.array(list(d.betas[k]))
        assert np.abs(beta[r, :15] - want).max() < 1e-11 * np.abs(want).max()
    assert H.info.n_bd == len(d.bd_cells)
    H.close()


@pytest.mark.parametrize("hinv", [64, 128])
def test_rotated_square_tables_match_oracle(lib, hinv):
    """The rotated square of Sec. 6.1 (the hole outside a rotated rectangle,
    corners on grid lines): the library's cell types, volumes, lattices and
    fit coefficients equal the oracle's."""
    P = W.problem_rotated_square()
    n = int(1.5 * hinv)
    H = _host(P, n, min_coarse_n=n)
    lev = G.build_level(P.dom, n, 0.1)
    d = D.discretize(lev, P.a, P.b, P.c)
    typ, kind, vol = H.cell_types()
    np.testing.assert_array_equal(kind, d.kind)
    np.testing.assert_array_equal(typ, lev.ctype)
    assert np.abs(vol - lev.vol).max() < 1e-15
    _, lat, beta = H.level_tables(0)
    plg = sorted(d.lattices)
    assert len(plg) == len(lat)
    for r, k in enumerate(plg):
        np.testing.assert_array_equal(lat[r], d.lattices[k])
        want = np.array(list(d.betas[k]))
        assert np.abs(beta[r, :15] - want).max() < 1e-11 * np.abs(want).max()
    assert H.info.n_bd == len(d.bd_cells)
    H.close()
