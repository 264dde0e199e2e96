"""The device-resident solve loop (cc_options.device_loop): a solve's
iterations (Alg. 3's outer loop around the cycles of Alg. 2) run inside one
CUDA graph launch, a conditional WHILE node repeating the iteration while a
one-thread kernel finds the relative residual above the tolerance.

The loop makes the same decisions as the host loop from the same numbers,
so every outcome must match the host loop's exactly: the solution bit for
bit, the status, the cycle count and the final relative residual.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
from paper_2601_02975_gb300 import Hierarchy, default_options, lib  # noqa: E402
from paper_2601_02975_gb300 import inputs as I  # noqa: E402
import workloads as W  # noqa: E402
from paper_2601_02975_gb300._lib import cc_result  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _problem(name):
    if name == "disk":
        return W.problem_disk()
    if name.startswith("ellipses"):
        return W.problem_ellipses(int(name[-1]))
    if name == "box_cross":
        u = W.u_expcos()
        dom = W.Domain(box_bc=(W.BC(), W.BC(W.NEUMANN, 0, 1), W.BC(), W.BC(W.ROBIN, 1.0, 0.5)))
        return W.Problem("box_cross", dom, 1.0, 0.5, 2.0, u, W.apply_L(u, 1.0, 0.5, 2.0))
    if name.startswith("batch"):
        return W.problem_batch(int(name[len("batch"):]))[0]
    raise KeyError(name)


def _solve(H, f, g, u, tol):
    """cc_solve without raising on a non-converged or diverged outcome."""
    r = cc_result()
    st = lib().cc_solve(H.h, f.data_ptr(), g.data_ptr(), u.data_ptr(), tol, None, C.byref(r))
    torch.cuda.synchronize()
    return st, r


CASES = [
    ("disk", 256, 32, 1e-13, dict(cycle=2, precision=1, w_depth=1, nu1=4, nu2=4)),   # the headline setting
    ("ellipses0", 128, 16, 1e-10, dict(cycle=1, precision=0)),                      # FP64 V(3,3)
    ("disk", 128, 16, 1e-10, dict(cycle=3, precision=1)),                           # FMG, mixed
    ("box_cross", 64, 8, 1e-13, dict(cycle=2, precision=0, max_cycles=3)),          # stops at max_cycles
    ("batch8", 256, 32, 1e-10, dict(cycle=2, precision=1, w_depth=1, nu1=4, nu2=4, max_cycles=40)),  # diverges
]


@pytest.mark.parametrize("name,n,mc,tol,opt", CASES)
def test_device_loop_equals_host_loop(name, n, mc, tol, opt):
    P = _problem(name)
    out = []
    f = g = None
    for loop in (1, 0):
        H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                                  default_options(min_coarse_n=mc, device_loop=loop, **opt))
        if f is None:
            fh, gh, _ = I.problem_inputs(H, P)
            f = torch.tensor(fh.ravel(), dtype=torch.float64, device=DEV)
            g = torch.tensor(gh, dtype=torch.float64, device=DEV)
        u = torch.zeros(n * n, dtype=torch.float64, device=DEV)
        st, r = _solve(H, f, g, u, tol)
        # a second solve on the same handle replays the same graph
        u2 = torch.zeros(n * n, dtype=torch.float64, device=DEV)
        st2, r2 = _solve(H, f, g, u2, tol)
        assert (st2, r2.status, r2.cycles, r2.rel_res) == (st, r.status, r.cycles, r.rel_res)
        assert torch.equal(u, u2)
        out.append((st, r.status, r.cycles, r.rel_res, u.cpu().numpy()))
        assert r.kernels > 0
        H.close()
    (sd, rd, cd, reld, ud), (sh, rh, ch, relh, uh) = out
    assert (sd, rd, cd) == (sh, rh, ch)
    assert reld == relh
    np.testing.assert_array_equal(ud.view(np.uint64), uh.view(np.uint64))
    if name == "batch8":
        assert rd == 6                      # CC_ERR_DIVERGED
    elif "max_cycles" in opt:
        assert rd == 5 and cd == opt["max_cycles"]   # CC_ERR_NOT_CONVERGED
    else:
        assert rd == 0 and reld < tol


def test_device_loop_zero_cycles_when_the_guess_is_converged():
    """Starting from a converged solution the loop body never runs: status OK,
    0 cycles, the guess returned unchanged."""
    P = _problem("disk")
    n = 128
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n,
                              default_options(min_coarse_n=16, cycle=2, precision=1))
    fh, gh, _ = I.problem_inputs(H, P)
    f = torch.tensor(fh.ravel(), dtype=torch.float64, device=DEV)
    g = torch.tensor(gh, dtype=torch.float64, device=DEV)
    u = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    st, r = _solve(H, f, g, u, 1e-12)
    assert st == 0 and r.cycles > 0
    u0 = u.clone()
    st, r = _solve(H, f, g, u, 1e-6)
    assert st == 0 and r.cycles == 0 and r.rel_res < 1e-6
    assert torch.equal(u, u0)
    H.close()
