"""The launch shapes cc_setup times on the device (cc_options.autotune): the
CTA count of the streamed FP32 sweep and the chunk size of each chunked
exact block of up to 8192 cells.

The sweep's result does not depend on its CTA count, so an FP32 cycle on a
domain without an exact block (Poisson on the unit square) must be the same
bits with and without tuning.  A tuned chunk size changes the rounding of
the block solve only: the tuned mixed solve of the disk problem must reach
the tolerance in about as many cycles, with an error against the exact
solution within 1.1x of the untuned one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
from paper_2601_02975_gb300 import Hierarchy, default_options  # noqa: E402
from paper_2601_02975_gb300 import inputs as I  # noqa: E402
import workloads as W  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _opts(tune, **kw):
    return default_options(min_coarse_n=32, cycle=2, precision=1, w_depth=1, nu1=4, nu2=4,
                           autotune=tune, **kw)


def test_tuned_sweep_gives_the_same_bits():
    P = W.problem_poisson_square()
    n = 1024
    outs = []
    for tune in (1, 0):
        H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n, _opts(tune))
        info = H.info
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        nt = (n // 32) * (n // 32)
        for lev in range(info.n_levels):
            ln = info.level_n[lev]
            g = info.sweep_ctas[lev]
            if ln >= 256:
                tiles = (ln // 32) * (ln // 32)
                assert g > 0 and (g % sms == 0 or g == tiles), (lev, g)
            else:
                assert g == 0
        assert 0 < info.sweep_ctas[0] <= nt
        rng = np.random.default_rng(5)
        u = torch.tensor(rng.standard_normal(n * n), dtype=torch.float64, device=DEV)
        b = torch.tensor(rng.standard_normal(n * n), dtype=torch.float64, device=DEV)
        for _ in range(2):
            H.cycle(u, b)
        torch.cuda.synchronize()
        outs.append(u.cpu().numpy())
        H.close()
    np.testing.assert_array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))


def test_tuned_chunk_size_solves_like_the_model_choice():
    P = W.problem_disk()
    n = 1024
    res = []
    for tune in (1, 0):
        H = Hierarchy.from_domain(P.dom, P.a, P.b, P.c, n, _opts(tune))
        rows = list(H.info.block_chunk_rows[:H.info.n_levels])
        assert rows[0] in (48, 64, 80, 96, 112, 128, 160, 192, 224, 256), rows
        f, g, ue = I.problem_inputs(H, P)
        present = H.cell_types()[0] != 0
        ft = torch.tensor(f.ravel(), dtype=torch.float64, device=DEV)
        gt = torch.tensor(g, dtype=torch.float64, device=DEV)
        u = torch.zeros(n * n, dtype=torch.float64, device=DEV)
        r = H.solve(ft, gt, u, 1e-13)
        torch.cuda.synchronize()
        assert r.status == 0
        err = float(np.abs(u.cpu().numpy().reshape(n, n) - ue)[present].max())
        res.append((r.cycles, err, rows))
        H.close()
    (ct, et, _), (c0, e0, _) = res
    assert abs(ct - c0) <= 1, res
    assert et <= 1.1 * e0 + 1e-14, res
