"""cc_smooth_noalloc, the sweep for callers that must not allocate device
memory at call time (for example inside stream capture), against cc_smooth.

The two entry points run the same kernels on the same inputs; the
allocation-free one keeps its temporaries in the library's one file-scope
device array instead of the handle's buffers.  Two calls in a row check
that what the first call leaves in that array does not leak into the
second.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
from paper_2601_02975_gb300 import CCError, Hierarchy, default_options  # noqa: E402
import workloads as W  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def hier():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    P = W.problem_disk()
    # 256^2: the finest level's exact block (1256 cells) takes the chunked
    # solve, whose temporaries live in the scratch array; the 128^2 level's
    # block (668 cells) the one-launch dense solve
    return Hierarchy.from_domain(P.dom, P.a, P.b, P.c, 256, default_options(min_coarse_n=16))


@pytest.mark.parametrize("level", [0, 1])
def test_noalloc_sweep_matches_cc_smooth(hier, level):
    H = hier
    n = H.info.level_n[level]
    # level 0 takes the chunked branch, level 1 the dense one
    assert (H.info.block_chunks[level] > 0) == (level == 0), list(H.info.block_chunks[:2])
    typ = None
    if level == 0:
        typ = H.cell_types()[0].ravel() != 0
    rng = np.random.default_rng(100 + level)
    for call in range(2):                       # two calls in a row
        u0 = rng.standard_normal(n * n)
        b0 = rng.standard_normal(n * n)
        if typ is not None:
            u0 *= typ
            b0 *= typ
        ref = torch.tensor(u0, dtype=torch.float64, device=DEV)
        got = ref.clone()
        bt = torch.tensor(b0, dtype=torch.float64, device=DEV)
        H.smooth(level, ref, bt)
        H.smooth_noalloc(level, got, bt)
        torch.cuda.synchronize()
        r = ref.cpu().numpy()
        g = got.cpu().numpy()
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max(), (level, call)


def test_noalloc_rejects_levels_beyond_the_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    P = W.problem_disk()       # 1024^2 cells plus about 4700 block cells: over 2^20
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, 1024, default_options(min_coarse_n=16))
    n = 1024
    u = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    b = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    with pytest.raises(CCError) as ei:
        H.smooth_noalloc(0, u, b)
    assert ei.value.status == 1 and "scratch" in str(ei.value)
    H.smooth_noalloc(1, u[: 512 * 512], b[: 512 * 512])     # 512^2 fits
    torch.cuda.synchronize()


def test_noalloc_multicolour_sweep_matches_cc_smooth():
    """The same on a handle with the multicolour smoother (its classes relaxed
    in place on a copy of u in the scratch array), levels 0 and 1 (the
    chunked and the dense block), two calls in a row each."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2601_02975_gb300 import SMOOTHER_MCGS
    P = W.problem_disk()
    H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, 256,
                              default_options(min_coarse_n=16, smoother=SMOOTHER_MCGS, omega=0.6))
    for level in (0, 1):
        n = H.info.level_n[level]
        rng = np.random.default_rng(200 + level)
        for call in range(2):
            u0 = rng.standard_normal(n * n)
            b0 = rng.standard_normal(n * n)
            ref = torch.tensor(u0, dtype=torch.float64, device=DEV)
            got = ref.clone()
            bt = torch.tensor(b0, dtype=torch.float64, device=DEV)
            H.smooth(level, ref, bt)
            H.smooth_noalloc(level, got, bt)
            torch.cuda.synchronize()
            typ = H.cell_types()[0].ravel() != 0 if level == 0 else None
            r = ref.cpu().numpy()
            g = got.cpu().numpy()
            if typ is not None:
                r, g = r[typ], g[typ]
            assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max(), (level, call)
