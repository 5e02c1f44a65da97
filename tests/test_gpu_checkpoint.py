"""A decomposition computed on the GPU, written to a checkpoint and read
back onto the GPU, gives bit-identical solves (the "compute the eigenpairs
once, reuse them" use of Sec. II)."""
import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_checkpoint_round_trip_on_the_gpu(tmp_path):
    import paper_1911_11906_gb300 as F
    p = I.ellipse_problem(24, seed=12)
    ctx = F.Context()
    mask = torch.from_numpy(p.mask).cuda()
    asm = F.fd_assemble(mask, p.h, ctx=ctx)
    lam, V = F.eig_full(asm["A"], ctx=ctx)
    Fd = torch.from_numpy(np.ascontiguousarray(p.F.T)).cuda().t()
    U = F.frac_apply(V, lam, Fd, p.pair_f, p.pair_alpha, ctx=ctx)
    path = str(tmp_path / "ellipse24.fraclap")
    F.save_decomposition(path, lam, V, mask=p.mask, h=p.h)
    lam2, V2 = F.load_decomposition(path, mask=mask, h=p.h)
    assert lam2.is_cuda and V2.is_cuda and V2.stride() == (1, p.n)
    assert torch.equal(lam2, lam) and torch.equal(V2, V)
    U2 = F.frac_apply(V2, lam2, Fd, p.pair_f, p.pair_alpha, ctx=ctx)
    assert torch.equal(U2, U)
    # and the reloaded pairs still solve the problem: alpha = 2 against the oracle's direct solve
    _, A = O.assemble(p.mask, p.h)
    Uh = U2.cpu().numpy()
    for j in np.nonzero(p.pair_alpha == 2.0)[0][:3]:
        ref = O.band_solve(A, p.F[:, p.pair_f[j]])
        assert np.linalg.norm(Uh[:, j] - ref) <= 1e-10 * np.linalg.norm(ref)
