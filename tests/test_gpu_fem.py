"""GPU parity of the generalised problem K phi = theta M phi (Sec. II eq.
discrete_laplace with bilinear / trilinear finite elements) against the
oracle: the assembly (CSR structure and values compared exactly, dense
copies), the eigenpairs of the pencil (eigenvalues, M-orthonormality,
residuals, the closed-form spectra of the square and the cube) and the apply
in the M-inner product (the oracle's apply on the oracle's pencil, alpha = 0
returning f, alpha = 2 solving K u = M f)."""
import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _F():
    import paper_1911_11906_gb300 as F
    return F


def _mu(m):
    """1-D generalised eigenvalues of the linear elements: (6/h^2)(1 - cos(j pi h)) / (2 + cos(j pi h))."""
    h = 1.0 / (m + 1)
    c = np.cos(np.arange(1, m + 1) * np.pi * h)
    return (6.0 / h ** 2) * (1 - c) / (2 + c)


def _closed(m, dim):
    mu = _mu(m)
    tot = np.zeros((m,) * dim)
    for d in range(dim):
        shape = [1] * dim
        shape[d] = m
        tot = tot + mu.reshape(shape)
    return np.sort(tot.ravel())


def _masks():
    return {"square9": (np.ones((9, 9), np.uint8), 0.1),
            "ellipse40": (lambda p: (p.mask, p.h))(I.ellipse_problem(40, n_ellipses=4, seed=7)),
            "cube5": (np.ones((5, 5, 5), np.uint8), 1.0 / 6),
            "holed": (lambda p: (p.mask, p.h))(I.holed_cube_problem(10, n_holes=2, n_forcings=1, seed=5)),
            "strip": (np.ones((1, 12), np.uint8), 1.0 / 13)}


@pytest.mark.parametrize("name", ["square9", "ellipse40", "cube5", "holed", "strip"])
def test_fem_assembly_matches_oracle(name):
    """CSR row pointer, columns, both value arrays and the dof numbering equal
    the oracle's exactly; the dense copies hold the same entries."""
    F = _F()
    mask, h = _masks()[name]
    idx_o, K_o, M_o = O.assemble_fem(mask, h)
    asm = F.fem_assemble(torch.from_numpy(mask).cuda(), h)
    assert asm["n"] == K_o.n
    assert np.array_equal(asm["idx"].cpu().numpy().ravel(), idx_o)
    assert np.array_equal(asm["rowptr"].cpu().numpy(), K_o.rowptr)
    assert np.array_equal(asm["col"].cpu().numpy(), K_o.col)
    assert np.array_equal(asm["valK"].cpu().numpy(), K_o.val)
    assert np.array_equal(asm["valM"].cpu().numpy(), M_o.val)
    assert np.array_equal(asm["K"].cpu().numpy(), K_o.dense())
    assert np.array_equal(asm["M"].cpu().numpy(), M_o.dense())


def test_fem_assembly_empty_and_single_node():
    F = _F()
    empty = F.fem_assemble(torch.zeros((4, 5), dtype=torch.uint8, device="cuda"), 0.2)
    assert empty["n"] == 0
    one = np.zeros((3, 3), np.uint8)
    one[1, 1] = 1
    h = 0.25
    asm = F.fem_assemble(torch.from_numpy(one).cuda(), h)
    _, K_o, M_o = O.assemble_fem(one, h)
    assert asm["n"] == 1 and float(asm["valK"][0]) == K_o.val[0] and float(asm["valM"][0]) == M_o.val[0]
    # one node: four cells, K = 4 (2/3) = 8/3 and M = 4 (h/3)^2, so theta = 6 / h^2
    theta, Phi = F.eig_pencil(asm["K"], asm["rowptr"], asm["col"], asm["valM"])
    assert abs(float(theta[0]) - 6.0 / h ** 2) <= 1e-13 * 6.0 / h ** 2
    assert abs(float(Phi[0, 0]) ** 2 * float(asm["valM"][0]) - 1.0) <= 1e-14


def _pencil(F, mask, h):
    asm = F.fem_assemble(torch.from_numpy(mask).cuda(), h)
    theta, Phi = F.eig_pencil(asm["K"], asm["rowptr"], asm["col"], asm["valM"])
    return asm, theta, Phi


@pytest.mark.parametrize("dim,m", [(2, 12), (2, 31), (3, 6)])
def test_pencil_closed_form(dim, m):
    """Square / cube: theta = sum_d mu_{j_d}; Phi^T M Phi = I; K Phi = M Phi Theta."""
    F = _F()
    mask = np.ones((m,) * dim, np.uint8)
    h = 1.0 / (m + 1)
    asm, theta, Phi = _pencil(F, mask, h)
    th = theta.cpu().numpy()
    ref = _closed(m, dim)
    assert np.max(np.abs(th - ref) / ref) <= 1e-11
    Kd, Md = asm["K"], asm["M"]
    G = Phi.t() @ (Md @ Phi)
    G.diagonal().sub_(1.0)
    assert float(G.abs().max()) <= 1e-12
    R = Kd @ Phi - (Md @ Phi) * theta
    assert float(R.abs().max()) <= 1e-12 * float(theta[-1]) * float(Md.abs().max())


@pytest.mark.parametrize("name", ["ellipse40", "holed"])
def test_pencil_and_mass_apply_match_oracle(name):
    """Masked domains: eigenvalues against the oracle's pencil solver (1e-11),
    and the solutions of the M-inner-product apply against the oracle's apply
    on the oracle's pencil (1e-10), for polynomial forcings and several
    orders; alpha = 0 returns f and alpha = 2 solves K u = M f (oracle's
    banded direct solve)."""
    F = _F()
    mask, h = _masks()[name]
    _, K_o, M_o = O.assemble_fem(mask, h)
    th_o, Phi_o = O.eig_pencil(K_o.dense(), M_o.dense())
    asm, theta, Phi = _pencil(F, mask, h)
    th = theta.cpu().numpy()
    assert np.max(np.abs(th - th_o) / th_o) <= 1e-11
    n = K_o.n
    rng = np.random.default_rng(n)
    Fm = rng.standard_normal((n, 3))
    pf = np.array([0, 1, 2, 0, 1, 2, 0], np.int32)
    pa = np.array([0.5, 1.0, 1.5, 2.0, 0.0, -2.0, 0.25])
    U_o = O.frac_apply_mass(Phi_o, th_o, M_o, Fm, pf, pa)
    Fd = torch.from_numpy(np.ascontiguousarray(Fm.T)).cuda().t()
    U = F.frac_apply_mass(Phi, theta, asm["rowptr"], asm["col"], asm["valM"], Fd, pf, pa).cpu().numpy()
    err = np.linalg.norm(U - U_o, axis=0) / np.linalg.norm(U_o, axis=0)
    assert err.max() <= 1e-10, err
    assert np.linalg.norm(U[:, 4] - Fm[:, 1]) <= 1e-12 * np.linalg.norm(Fm[:, 1])
    ref2 = O.band_solve(K_o, O.spmv(M_o, Fm[:, 0]))
    assert np.linalg.norm(U[:, 3] - ref2) <= 1e-10 * np.linalg.norm(ref2)


def test_mass_apply_rejects_bad_pairs_and_keeps_context_usable():
    F = _F()
    mask, h = _masks()["square9"]
    asm, theta, Phi = _pencil(F, mask, h)
    Fd = torch.ones(asm["n"], 1, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FraclapError):
        F.frac_apply_mass(Phi, theta, asm["rowptr"], asm["col"], asm["valM"], Fd, [3], [1.0])
    U = F.frac_apply_mass(Phi, theta, asm["rowptr"], asm["col"], asm["valM"], Fd, [0], [0.0])
    assert float((U - Fd).abs().max()) <= 1e-12
