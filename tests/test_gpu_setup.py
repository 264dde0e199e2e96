"""The per-cell setup steps on the GPU (cc_options.device_setup): the
classification of the cells no curve crosses (Sec. 3.1), the kinds of
Def. 4.1, the poised lattices (Def. 4.3), the fits (Eq. 4.14, 4.17-4.18)
and the curve-order samples of Def. 5.1.

The device kernels and the host threads run the same per-cell functions with
IEEE operations only and no fused multiply-adds, so every table must equal
the host path's bit for bit, on every level (union 15 and 32 include cut
cells of two components, whose second component the host moves to a
neighbour in both paths; union 52 has a cell whose lattice only the host's
far search finds, after the device's search of the 9 x 9 to 13 x 13
boxes); the device tables are also
compared with the oracle's directly (lattices exactly, fits to rounding).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
from oracle import discretize as D  # noqa: E402
from oracle import geometry as G  # noqa: E402
from paper_2601_02975_gb300 import Hierarchy, default_options  # noqa: E402
import workloads as W  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _problem(name):
    if name == "disk":
        return W.problem_disk(), {}
    if name.startswith("ellipses"):
        return W.problem_ellipses(int(name[8:])), {}
    if name == "four_disks":
        return W.problem_four_disks(W.NEUMANN), {}
    if name == "flower":
        return W.problem_flower(), {"eps": 0.02}
    if name == "rotated":
        return W.problem_rotated_square(), {}
    if name == "box_cross":
        u = W.u_expcos()
        dom = W.Domain(box_bc=(W.BC(), W.BC(W.NEUMANN, 0, 1), W.BC(), W.BC(W.ROBIN, 1.0, 0.5)))
        return W.Problem("box_cross", dom, 1.0, 0.5, 2.0, u, W.apply_L(u, 1.0, 0.5, 2.0)), {}
    raise KeyError(name)


def _both(name, n, mc, **opt):
    """The same problem set up on the device and on host threads.  Launch
    shapes are not tuned: a timed choice of chunk size could differ between
    the two and change the rounding of the block solves (tuning has its own
    tests)."""
    P, extra = _problem(name)
    hs = []
    for dev in (1, 0):
        hs.append(Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                                        default_options(min_coarse_n=mc, device_setup=dev, autotune=0,
                                                        **extra, **opt)))
    return P, extra, hs[0], hs[1]


@pytest.mark.parametrize("name,n,mc", [("disk", 256, 16), ("ellipses0", 256, 32),
                                       ("ellipses3", 512, 64), ("four_disks", 256, 32),
                                       ("flower", 256, 32), ("rotated", 192, 24),
                                       ("box_cross", 128, 8), ("disk", 1024, 32),
                                       ("ellipses15", 128, 32), ("ellipses32", 256, 32),
                                       ("ellipses52", 256, 32)])
def test_device_tables_equal_host_tables(name, n, mc):
    P, _, Hd, Hh = _both(name, n, mc)
    assert Hd.info.n_levels == Hh.info.n_levels
    assert Hd.info.setup_kernel_ms > 0 and Hh.info.setup_kernel_ms == 0
    for a, b in zip(Hd.cell_types(), Hh.cell_types()):
        np.testing.assert_array_equal(a, b)
    for lev in range(Hd.info.n_levels):
        kd, ld, bd = Hd.level_tables(lev)
        kh, lh, bh = Hh.level_tables(lev)
        np.testing.assert_array_equal(kd, kh)
        np.testing.assert_array_equal(ld, lh)
        # the same bits, not just the same values
        np.testing.assert_array_equal(bd.view(np.uint64), bh.view(np.uint64))
        np.testing.assert_array_equal(Hd.level_block(lev), Hh.level_block(lev))
    assert Hd.info.block_error == Hh.info.block_error
    Hd.close()
    Hh.close()


@pytest.mark.parametrize("name,n", [("ellipses0", 128), ("flower", 128), ("rotated", 96)])
def test_device_tables_match_oracle(name, n):
    """The device-built finest level against the oracle's tables: the same
    types, kinds and lattices, fits within 1e-11 of the largest weight."""
    P, extra = _problem(name)
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                              default_options(min_coarse_n=n // 2, device_setup=1, **extra))
    lev = G.build_level(P.dom, n, extra.get("eps", 0.1))
    d = D.discretize(lev, P.a, P.b, P.c)
    typ, kind, vol = H.cell_types()
    np.testing.assert_array_equal(typ, lev.ctype)
    np.testing.assert_array_equal(kind, d.kind)
    assert np.abs(vol - lev.vol).max() < 1e-15
    _, lat, beta = H.level_tables(0)
    plg = sorted(d.lattices)
    assert len(plg) == len(lat)
    for r, k in enumerate(plg):
        np.testing.assert_array_equal(lat[r], d.lattices[k])
        want = np.array(list(d.betas[k]))
        assert np.abs(beta[r, :15] - want).max() < 1e-11 * np.abs(want).max()
    H.close()


def test_device_setup_solve_equals_host_setup_solve():
    """Equal tables give equal solves: the mixed-precision solve of the
    ellipse-union problem from both setups, bit for bit."""
    from paper_2601_02975_gb300 import inputs as I
    P, _, Hd, Hh = _both("ellipses1", 256, 32, cycle=2, precision=1, nu1=4, nu2=4, w_depth=1)
    outs = []
    for H in (Hd, Hh):
        f, g, _ = I.problem_inputs(H, P)
        ft = torch.tensor(f.ravel(), dtype=torch.float64, device=DEV)
        gt = torch.tensor(g, dtype=torch.float64, device=DEV)
        u = torch.zeros_like(ft)
        r = H.solve(ft, gt, u, 1e-10)
        torch.cuda.synchronize()
        assert r.status == 0
        outs.append((u.cpu().numpy(), r.cycles))
    assert outs[0][1] == outs[1][1]
    np.testing.assert_array_equal(outs[0][0].view(np.uint64), outs[1][0].view(np.uint64))
    Hd.close()
    Hh.close()
