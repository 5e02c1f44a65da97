"""Failure detection on the GPU without a fault: a bounded device wait that
nothing will satisfy (the cooperative kernels' grid barrier, the tensor-core
kernels' mbarrier) gives up after the context's limit, the host reads
FRACLAP_ERR_TIMEOUT, and the same context then computes a correct result."""
import time

import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_times_out_and_context_survives(which):
    import paper_1911_11906_gb300 as F
    ctx = F.Context(wait_timeout_s=0.2)
    t0 = time.perf_counter()
    ctx.wait_selftest(which)
    with pytest.raises(F.FraclapError) as ei:
        ctx.sync()
    assert ei.value.code == -4
    assert time.perf_counter() - t0 < 30.0
    ctx.sync()  # the status was read and cleared
    # the context (and its grid-barrier state) still works: a small solve
    p = I.square_problem(12, n_poly=1, alphas=(1.0, 2.0))
    mask = torch.from_numpy(p.mask).cuda()
    Fd = torch.from_numpy(np.asfortranarray(p.F)).cuda()
    lam, V, U = F.solve(mask, p.h, Fd, p.pair_f, p.pair_alpha, ctx=ctx)
    _, _, U_o = O.solve(p.mask, p.h, p.F, p.pair_f, p.pair_alpha)
    Ug = U.cpu().numpy()
    for j in range(U_o.shape[1]):
        assert np.linalg.norm(Ug[:, j] - U_o[:, j]) <= 1e-10 * np.linalg.norm(U_o[:, j])


def test_wait_selftest_rejects_unknown_kind():
    import paper_1911_11906_gb300 as F
    ctx = F.Context()
    with pytest.raises(F.FraclapError) as ei:
        ctx.wait_selftest(2)
    assert ei.value.code == -1
