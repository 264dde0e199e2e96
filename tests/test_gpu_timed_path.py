"""GPU parity of the kernels on the timed path against the FP64 oracle.

The bench solves the 1024^2 disk (and the ellipse unions at 2048^2 and 4096^2)
with FP32 cycles inside FP64 refinement.  On those grids the cycle runs
kernels that the small parity cases of test_gpu_parity.py do not reach:

  - the chunked exact block solve (Eq. 5.8) of blocks above 1024 cells, in
    FP64 and in FP32;
  - the streamed FP32 Jacobi sweep of grids of 256^2 and more (Eq. 5.7);
  - the FP32 dense block solve and FP32 restriction / interpolation of the
    coarser levels.

Here each is compared with the oracle on the same problem: one FP64 sweep
element by element, one FP32 cycle against the oracle's FP64 cycle, and whole
mixed-precision solves whose error against the exact cell averages must be
within 1.1x of the oracle's direct solve of the same system.
"""
import functools

import numpy as np
import pytest
import scipy.sparse.linalg as spl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
from oracle import discretize as D  # noqa: E402
from oracle import geometry as G  # noqa: E402
from oracle import multigrid as M  # noqa: E402
from paper_2601_02975_gb300 import Hierarchy, default_options  # noqa: E402
from paper_2601_02975_gb300 import inputs as I  # noqa: E402
import workloads as W  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _problem(name):
    return W.problem_disk() if name == "disk" else W.problem_ellipses(0)


def _t(x):
    return torch.tensor(np.ascontiguousarray(x).ravel(), dtype=torch.float64, device=DEV)


def _np(t, n):
    return t.cpu().numpy().reshape(n, n)


@functools.lru_cache(maxsize=None)
def _oracle_finest(name, n):
    """The oracle's finest level alone (geometry, discretisation, the A22
    factorisation of Def. 5.3): enough for its block smoother."""
    P = _problem(name)
    d = D.discretize(G.build_level(P.dom, n, 0.1), P.a, P.b, P.c)
    return M.Hierarchy([d], [M.A22LU(d)], None)


@functools.lru_cache(maxsize=None)
def _oracle_hierarchy(name, n, mc):
    P = _problem(name)
    return M.build_hierarchy(P.dom, n, P.a, P.b, P.c, min_coarse=mc)


@functools.lru_cache(maxsize=None)
def _oracle_direct(name, n, mc):
    """The oracle's direct solve of its own system, and its max-norm error
    against the exact cell averages."""
    P = _problem(name)
    O = _oracle_hierarchy(name, n, mc)
    d = O.levels[0]
    b = D.rhs(d, D.cell_averages(d.lev, P.f), D.boundary_data(d, P.u))
    ud = spl.spsolve(d.A.tocsc(), b.ravel()).reshape(n, n)
    err = np.abs(ud - D.cell_averages(d.lev, P.u))[d.lev.present].max()
    return b, ud, err


@pytest.mark.slow
@pytest.mark.parametrize("name,n", [("ellipses0", 512), ("disk", 1024)])
def test_chunked_block_sweep_matches_oracle(name, n):
    """One FP64 block-smoother sweep (Def. 5.6) on the finest level of the
    512^2 ellipse union (a block of 2789 cells) and of the bench's 1024^2
    disk (4680 cells), where the block is solved by the two chunked launches,
    against the oracle's sweep with its sequential banded LU (Def. 5.3), on
    random u and b: 1e-11 relative max-norm."""
    P = _problem(name)
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n, default_options(min_coarse_n=32))
    assert H.info.block_chunks[0] > 0, "the finest block must take the chunked solve"
    O = _oracle_finest(name, n)
    d = O.levels[0]
    assert O.lus[0].m == H.info.block_m[0]
    rng = np.random.default_rng(1234)
    u = rng.standard_normal((n, n)) * d.lev.present
    b = rng.standard_normal((n, n)) * d.lev.present / d.h ** 2
    ut = _t(u)
    H.smooth(0, ut, _t(b))
    uo = M.smooth(O, 0, u, b)
    got = _np(ut, n)
    err = np.abs(got - uo).max() / np.abs(uo).max()
    assert err < 1e-11, err
    # the exactly solved rows have zero residual after the sweep (Sec. 5.2)
    r = M.residual(d, got, b).ravel()[O.lus[0].order]
    assert np.abs(r).max() < 1e-9 * np.abs(b).max(), np.abs(r).max()


@pytest.mark.slow
@pytest.mark.parametrize("name", ["disk", "ellipses0"])
def test_fp32_cycle_matches_oracle_cycle(name):
    """One FP32 cycle of the mixed mode (cc_cycle on a mixed handle: streamed
    FP32 sweeps, FP32 chunked and dense block solves, FP32 restriction and
    interpolation, the FP64 bottom solve) on the 512^2 grid against the
    oracle's FP64 cycle from the same u and b: the same iterate up to FP32
    rounding.  Bound, from the arithmetic: each exact block solve in FP32
    returns its rows with a relative error up to about cond(A22) eps32
    (eps32 = 2^-24), the finest level solves its block nu1 + nu2 = 8 times in
    the cycle, and the Jacobi updates and transfers add a few eps32 more; so
    the cycle's iterate may differ from the FP64 one by
    4 (nu1 + nu2) cond(A22) eps32 relative (max-norm), cond(A22) computed here
    from the oracle's block (a few hundred).  A wrong FP32 kernel misses it
    by orders of magnitude (one mis-solved chunk gives about 1e-1)."""
    n, mc, nu = 512, 32, 4
    P = _problem(name)
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                              default_options(min_coarse_n=mc, cycle=2, w_depth=1, nu1=nu,
                                              nu2=nu, precision=1))
    O = _oracle_hierarchy(name, n, mc)
    assert H.info.n_levels == O.nl
    assert H.info.block_chunks[0] > 0 and H.info.block_chunks[1] > 0
    b, _, _ = _oracle_direct(name, n, mc)
    u0 = np.zeros((n, n))
    ut = _t(u0)
    H.cycle(ut, _t(b))
    uo = M.cycle(O, 0, u0, b, nu, nu, 2, 1)
    present = O.levels[0].lev.present
    got = _np(ut, n)
    err = np.abs(got - uo)[present].max() / np.abs(uo)[present].max()
    order = O.lus[0].order
    cond = np.linalg.cond(O.levels[0].A[order][:, order].toarray())
    bound = 4 * (2 * nu) * cond * 2.0 ** -24
    print(f"{name}: FP32 cycle vs oracle {err:.3e}, cond(A22) {cond:.0f}, bound {bound:.2e}")
    assert err < bound, (err, bound)


@pytest.mark.slow
@pytest.mark.parametrize("name,n", [("disk", 256), ("ellipses0", 256), ("disk", 512),
                                    ("ellipses0", 512)])
def test_mixed_solve_error_within_oracle(name, n):
    """The mixed-precision solve as the bench runs it (FP32 W(4,4) cycles,
    gamma = 2 on the finest level only, inside FP64 refinement) at 256^2 and
    512^2, where the streamed sweep and the chunked FP32 block solves run: it
    reaches the relative residual tol, and its max-norm error against the
    exact cell averages is within 1.1x of the oracle's direct solve of the
    same system (its discretisation error).  tol is small enough for the
    algebraic error to sit below the discretisation error: 1e-13 on the disk,
    whose right-hand side carries boundary data scaled by 1/h^2, 1e-12 on the
    ellipse union."""
    mc, nu = 32, 4
    P = _problem(name)
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                              default_options(min_coarse_n=mc, cycle=2, w_depth=1, nu1=nu,
                                              nu2=nu, precision=1, max_cycles=60))
    _, _, err_o = _oracle_direct(name, n, mc)
    f, g, ue = I.problem_inputs(H, P)
    u = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    tol = 1e-13 if name == "disk" else 1e-12
    r = H.solve(_t(f), _t(g), u, tol)
    assert r.status == 0 and r.rel_res < tol, (r.status, r.cycles, r.rel_res)
    present = H.cell_types()[0] != 0
    err = np.abs(_np(u, n) - ue)[present].max()
    print(f"{name} {n}: mixed error {err:.3e}, oracle direct {err_o:.3e}, {r.cycles} cycles")
    assert err <= 1.1 * err_o + 1e-14, (err, err_o)
