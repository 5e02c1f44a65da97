"""GPU parity of the eigen-decomposition stages against the FP64 CPU oracle.

Intermediate results of the reduction are not unique (reflector signs,
the band), so the stages are compared through invariants: the tridiagonal
matrix has the oracle's eigenvalues, the accumulated Q is orthogonal and
Q^T A Q reproduces T; the divide-and-conquer solver is compared with the
oracle's implicit-QR solver on the same (d, e); eig_full is compared on
eigenvalues, residual, orthogonality and on spectral projectors.
"""
import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I
from conftest import square_closed_form

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _F():
    import paper_1911_11906_gb300 as F
    return F


def _colmajor(a):
    a = np.asfortranarray(a, dtype=np.float64)
    return torch.from_numpy(a.T.copy()).cuda().t()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _tridiag_cases():
    rng = np.random.default_rng(11)
    cases = []
    for n in (1, 2, 3, 5, 31, 32, 33, 64, 100, 257, 1000):
        cases.append((f"random{n}", rng.standard_normal(n), rng.standard_normal(max(n - 1, 0))))
    cases.append(("lap1d", np.full(300, 2.0), np.full(299, -1.0)))
    cases.append(("glued", np.ones(200), np.full(199, 1e-10)))
    cases.append(("zero_coupling", np.arange(150.0), np.zeros(149)))
    cases.append(("wilkinson", np.abs(np.arange(-60, 61)).astype(float), np.ones(120)))
    # many close poles in every merge: rotations within and across the
    # deflation pass's 32-position groups
    cases.append(("wilkinson401", np.abs(np.arange(-200, 201)).astype(float), np.ones(400)))
    cases.append(("clusters1000", np.floor(np.arange(1000) / 7.0) + 1e-13 * rng.standard_normal(1000),
                  1e-9 * rng.standard_normal(999)))
    p = I.ellipse_problem(30, seed=9)
    _, A = O.assemble(p.mask, p.h)
    d, e, _ = O.tridiagonalize(A.dense(), want_q=False)
    cases.append(("ellipse30", d, e))
    return cases


@pytest.mark.parametrize("name,d,e", _tridiag_cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_tridiag_dc_vs_oracle(name, d, e):
    F = _F()
    n = d.size
    lam_o, _ = O.tridiag_eig(d, e, want_vectors=False)
    lam, Z = F.tridiag_eig(_cuda(d), _cuda(e))
    lam, Z = lam.cpu().numpy(), Z.cpu().numpy()
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1) if n > 1 else np.diag(d)
    nrm = max(np.abs(lam_o).max(), 1e-300)
    assert np.max(np.abs(lam - lam_o)) <= 1e-13 * nrm * max(1, np.log2(n))
    assert np.all(np.diff(lam) >= 0)
    assert np.linalg.norm(T @ Z - Z * lam) <= 1e-14 * n * max(np.linalg.norm(T), 1e-300)
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) <= 1e-13 * max(1, np.sqrt(n))


@pytest.mark.parametrize("b", [4, 16, 32, 64])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 65, 130, 301])
def test_tridiagonalize_invariants(n, b):
    F = _F()
    ctx = F.Context(band_width=b)
    rng = np.random.default_rng(n * 7 + b)
    B = rng.standard_normal((n, n))
    A = B + B.T
    d, e, Q = F.tridiagonalize(_colmajor(A), ctx=ctx)
    d, e, Q = d.cpu().numpy(), e.cpu().numpy(), Q.cpu().numpy()
    T = np.diag(d) + (np.diag(e, 1) + np.diag(e, -1) if n > 1 else 0)
    nrm = np.linalg.norm(A)
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 1e-14 * max(n, 4)
    assert np.linalg.norm(Q @ T @ Q.T - A) <= 1e-14 * n * nrm
    lam_A, _ = O.eig_full(A)
    lam_T, _ = O.tridiag_eig(d, e, want_vectors=False)
    assert np.max(np.abs(lam_A - lam_T)) <= 1e-13 * np.abs(lam_A).max() * max(1, np.sqrt(n))


def _check_decomposition(A, lam_o, lam, V, tol_lam=1e-11):
    n = A.shape[0]
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(lam - lam_o) / np.abs(lam_o)) <= tol_lam
    resid = np.linalg.norm(A @ V - V * lam) / (np.linalg.norm(A) * n)
    assert resid <= 1e-13
    assert np.max(np.abs(V.T @ V - np.eye(n))) <= 1e-12


@pytest.mark.parametrize("route", ["fp64", "mixed"])
@pytest.mark.parametrize("m", [1, 2, 3, 5, 9, 23])
def test_eig_full_small_squares(m, route):
    """Both routes on the smallest grids (n = 1, 4, 9, ...): one-tile and
    one-panel cases of every kernel, against the closed form and the oracle."""
    F = _F()
    p = I.square_problem(m, n_poly=0)
    _, A = O.assemble(p.mask, p.h)
    D = A.dense()
    if route == "fp64":
        lam, V = F.eig_full(_colmajor(D))
    else:
        lam, V = F.eig_full_mixed(_colmajor(D), *_csr_cuda(A), refine_iters=6)
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    ref = square_closed_form(m, 2)
    lam_o, _ = O.eig_full(D)
    _check_decomposition(D, lam_o, lam, V)
    assert np.max(np.abs(lam - ref) / ref) <= 1e-11


@pytest.mark.parametrize("seed,b,q2", [(3, 32, 0), (4, 8, 0), (5, 64, 0), (5, 64, 16), (6, 64, 4)])
def test_eig_full_masked_vs_oracle(seed, b, q2):
    F = _F()
    p = I.ellipse_problem(36, seed=seed)
    _, A = O.assemble(p.mask, p.h)
    D = A.dense()
    lam_o, V_o = O.eig_full(D)
    ctx = F.Context(band_width=b)
    ctx.set_schedule("q2_parts", q2)  # FP64 stage-2 back-transformation with 8 (default, and for 4) or 16 parts
    lam, V = F.eig_full(_colmajor(D), ctx=ctx)
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    _check_decomposition(D, lam_o, lam, V)
    # solutions agree (eigenvectors are not compared column by column)
    U_o = O.frac_apply(V_o, lam_o, p.F, p.pair_f, p.pair_alpha)
    U = O.frac_apply(V, lam, p.F, p.pair_f, p.pair_alpha)
    err = max(np.linalg.norm(U[:, j] - U_o[:, j]) / np.linalg.norm(U_o[:, j]) for j in range(U.shape[1]))
    assert err <= 1e-10


def _csr_cuda(A):
    return (torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.col).cuda(), torch.from_numpy(A.val).cuda())


@pytest.mark.parametrize("tc,tile_n,q2,cluster", [(0, 256, 0, 1), (1, 128, 0, 1), (0, 128, 8, 1), (0, 128, 16, 1),
                                                  (0, 256, 4, 1), (0, 256, 0, 2), (0, 128, 0, 2), (0, 192, 8, 1)])
@pytest.mark.parametrize("which,b,iters", [("square23", 32, 6), ("ellipse36", 32, 6), ("ellipse36", 64, 6),
                                            ("ellipse64", 32, 6), ("ellipse48", 16, 6), ("square9", 8, 6),
                                            ("cube6", 32, 6)])
def test_eig_full_mixed_refined_vs_oracle(which, b, iters, tc, tile_n, q2, cluster):
    """FP32 stages (FMA kernel, or three TF32 products on the tensor cores
    with tc = 1) + Ogita-Aishima refinement (slice products on 128- or
    256-column tiles, alone or in clusters sharing the B tile, lower
    triangle only) reach the FP64 tolerances."""
    F = _F()
    if which.startswith("square"):
        p = I.square_problem(int(which[6:]))
    elif which.startswith("cube"):
        m = int(which[4:])
        p = I.holed_cube_problem(m, n_holes=0, n_forcings=3)
    else:
        p = I.ellipse_problem(int(which[7:]), seed=17)
    _, A = O.assemble(p.mask, p.h)
    D = A.dense()
    lam_o, V_o = O.eig_full(D)
    ctx = F.Context(band_width=b)
    ctx.set_schedule("fp32_stages_tc", tc)
    ctx.set_schedule("ozaki_tile_n", tile_n)
    ctx.set_schedule("q2_parts", q2)
    ctx.set_schedule("ozaki_cluster", cluster)
    lam, V = F.eig_full_mixed(_colmajor(D), *_csr_cuda(A), refine_iters=iters, ctx=ctx)
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    _check_decomposition(D, lam_o, lam, V)
    stats = ctx.refine_stats()
    assert 1 <= len(stats) <= iters
    assert stats[-1]["norm2_R"] <= 3e-9 or len(stats) == iters
    U_o = O.frac_apply(V_o, lam_o, p.F, p.pair_f, p.pair_alpha)
    U = O.frac_apply(V, lam, p.F, p.pair_f, p.pair_alpha)
    err = max(np.linalg.norm(U[:, j] - U_o[:, j]) / np.linalg.norm(U_o[:, j]) for j in range(U.shape[1]))
    assert err <= 1e-10


@pytest.mark.parametrize("tc", [0, 1])
def test_eig_full_mixed_without_refinement_is_fp32_accurate(tc):
    F = _F()
    p = I.ellipse_problem(30, seed=3)
    _, A = O.assemble(p.mask, p.h)
    D = A.dense()
    lam_o, _ = O.eig_full(D)
    ctx = F.Context()
    ctx.set_schedule("fp32_stages_tc", tc)
    lam, V = F.eig_full_mixed(_colmajor(D), *_csr_cuda(A), refine_iters=0, ctx=ctx)
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    assert np.max(np.abs(lam - lam_o)) <= 1e-4 * lam_o[-1]
    assert np.max(np.abs(V.T @ V - np.eye(A.n))) <= 1e-4
