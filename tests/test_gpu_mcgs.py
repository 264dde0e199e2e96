"""The multicolour Gauss-Seidel variant of the block smoother (outside the
paper) on the GPU, against the oracle's variant: each step of one sweep,
whole cycles in FP64 and mixed-precision solves.  The colour classes are
relaxed in place, one launch each; see oracle.multigrid.colours."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
from oracle import discretize as D  # noqa: E402
from oracle import multigrid as M  # noqa: E402
from paper_2601_02975_gb300 import SMOOTHER_MCGS, Hierarchy, default_options  # noqa: E402
from paper_2601_02975_gb300 import inputs as I  # noqa: E402
import workloads as W  # noqa: E402

DEV = "cuda:0"
OMEGA = 0.6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _problem(name):
    if name == "table3":
        return W.problem_table3()
    if name == "disk":
        return W.problem_disk()
    if name == "ellipses0":
        return W.problem_ellipses(0)
    return W.problem_four_disks(W.NEUMANN)


def _pair(name, n, mc, **opt):
    P = _problem(name)
    kw = dict(eps=0.08) if name == "four_disks" else {}
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                              default_options(min_coarse_n=mc, smoother=SMOOTHER_MCGS, omega=OMEGA,
                                              **kw, **opt))
    O = M.build_hierarchy(P.dom, n, P.a, P.b, P.c, min_coarse=mc, smoother="mcgs", omega=OMEGA, **kw)
    assert H.info.n_levels == O.nl
    return P, H, O


def _t(x):
    return torch.tensor(np.ascontiguousarray(x).ravel(), dtype=torch.float64, device=DEV)


def _np(t, n):
    return t.cpu().numpy().reshape(n, n)


@pytest.mark.parametrize("name,n,mc", [("table3", 48, 6), ("disk", 64, 16), ("ellipses0", 64, 16),
                                       ("four_disks", 64, 16)])
def test_mcgs_sweep_parity(name, n, mc):
    """One multicolour sweep (every class in place, then the exact block
    solve) on every level but the coarsest, random inputs, FP64: the oracle's
    sweep to 1e-12 relative."""
    P, H, O = _pair(name, n, mc)
    for l in range(O.nl - 1):
        d = O.levels[l]
        rng = np.random.default_rng(40 + l)
        u = rng.standard_normal((d.n, d.n)) * d.lev.present
        b = rng.standard_normal((d.n, d.n)) * d.lev.present
        ut = _t(u)
        H.smooth(l, ut, _t(b))
        uo = M.smooth(O, l, u, b)
        assert np.abs(_np(ut, d.n) - uo).max() < 1e-12 * np.abs(uo).max() * 10, l


@pytest.mark.parametrize("name,n,mc", [("table3", 48, 6), ("disk", 64, 16), ("ellipses0", 64, 16)])
def test_mcgs_cycle_parity_fp64(name, n, mc):
    """FP64 W(2,2) cycles with the multicolour smoother match the oracle's
    iterates to 1e-11 relative max-norm after every cycle."""
    P, H, O = _pair(name, n, mc, cycle=2, nu1=2, nu2=2)
    f, g, _ = I.problem_inputs(H, P)
    b = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    H.assemble_rhs(_t(f), _t(g), b)
    d = O.levels[0]
    bo = D.rhs(d, D.cell_averages(d.lev, P.f), D.boundary_data(d, P.u))
    u = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    uo = np.zeros((n, n))
    for k in range(5):
        H.cycle(u, b)
        uo = M.cycle(O, 0, uo, bo, 2, 2, 2)
        err = np.abs(_np(u, n) - uo).max() / np.abs(uo).max()
        assert err < 1e-11, (k, err)


@pytest.mark.parametrize("name,n,mc", [("disk", 128, 16), ("ellipses0", 128, 16)])
def test_mcgs_solve_mixed(name, n, mc):
    """The mixed-precision solve with the multicolour smoother (FP32 W(2,2)
    cycles in FP64 refinement) reaches 1e-10 in about the oracle's number of
    cycles, with an error against the exact cell averages within 1.1x of the
    oracle's solve."""
    P, H, O = _pair(name, n, mc, cycle=2, nu1=2, nu2=2, precision=1)
    f, g, ue = I.problem_inputs(H, P)
    d = O.levels[0]
    bo = D.rhs(d, D.cell_averages(d.lev, P.f), D.boundary_data(d, P.u))
    ro = M.solve(O, bo, tol=1e-10, nu1=2, nu2=2, gamma=2)
    err_o = np.abs(ro.u - D.cell_averages(d.lev, P.u))[d.lev.present].max()
    u = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    r = H.solve(_t(f), _t(g), u, 1e-10)
    assert r.status == 0 and r.rel_res < 1e-10
    assert abs(r.cycles - len(ro.history)) <= 2, (r.cycles, len(ro.history))
    err = np.abs(_np(u, n) - ue)[d.lev.present].max()
    assert err <= 1.1 * err_o + 1e-14, (err, err_o)
