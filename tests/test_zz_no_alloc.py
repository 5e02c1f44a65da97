"""frac_apply_noalloc: the spectral apply for callers that cannot allocate
device memory (code running inside another framework's memory pool, or
latency-critical loops that cannot afford cudaMalloc's implicit device
synchronisation).  Its scratch is a fixed array inside the library, shared
by every call, so this test checks that two calls in a row, each through the
C ABI, reproduce the allocating frac_apply entry point and the oracle's
apply on different inputs (nothing stale from the first call may leak into
the second), and that a
problem too large for the array is refused without launching anything.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_DOUBLES = 1 << 21  # FRACLAP_NOALLOC_MAX_DOUBLES in include/fraclap.h


def _colmajor(a):
    a = np.asfortranarray(a, dtype=np.float64)
    return torch.from_numpy(a.T.copy()).cuda().t()


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _noalloc(lib, V, lam, F, pf, pa, U, status):
    n, m, k = V.shape[0], F.shape[1], pf.numel()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.frac_apply_noalloc(_p(V), V.stride(1), _p(lam), n, _p(F), F.stride(1), m, _p(pf), _p(pa), k,
                                  _p(U), U.stride(1), _p(status), st)


def _case(m_grid, seed):
    p = I.ellipse_problem(m_grid, n_forcings=5, alphas=(0.0, 0.5, 1.3, 2.0, -1.0), seed=seed)
    _, A = O.assemble(p.mask, p.h)
    lam, V = O.eig_full(A.dense())
    return p, lam, V


def test_noalloc_matches_frac_apply_on_two_calls():
    import paper_1911_11906_gb300 as F
    lib = F.load_library()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for grid, seed in ((22, 31), (27, 32)):   # two calls in a row, different sizes and data
        p, lam, V = _case(grid, seed)
        Vd, ld = _colmajor(V), torch.from_numpy(lam).cuda()
        Fd = _colmajor(p.F)
        pf = torch.from_numpy(p.pair_f.astype(np.int32)).cuda()
        pa = torch.from_numpy(p.pair_alpha).cuda()
        ref = F.frac_apply(Vd, ld, Fd, pf, pa).cpu().numpy()
        U = F._binding.empty_colmajor(p.n, pf.numel())
        U.fill_(float("nan"))
        rc = _noalloc(lib, Vd, ld, Fd, pf, pa, U, status)
        torch.cuda.synchronize()
        assert rc == 0
        assert int(status.item()) == 0
        got = U.cpu().numpy()
        for j in range(ref.shape[1]):
            assert np.linalg.norm(got[:, j] - ref[:, j]) <= 1e-13 * np.linalg.norm(ref[:, j])
        # and the oracle's apply of the same (V, lambda): the definition of the result
        U_o = O.frac_apply(V, lam, p.F, p.pair_f, p.pair_alpha)
        for j in range(U_o.shape[1]):
            assert np.linalg.norm(got[:, j] - U_o[:, j]) <= 1e-12 * np.linalg.norm(U_o[:, j])


def test_noalloc_refuses_oversized_problems():
    import paper_1911_11906_gb300 as F
    lib = F.load_library()
    n, m, k = 4096, 512, 512          # n * (m + k) = 2^22, twice the array
    V = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.frac_apply_noalloc(_p(V), n, _p(V), n, _p(V), n, m, _p(V), _p(V), k, _p(V), n, None, st)
    assert rc == -7   # FRACLAP_ERR_UNSUPPORTED, nothing launched
    torch.cuda.synchronize()
