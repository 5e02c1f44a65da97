"""Pins of the oracle's finite-element generalised problem (Sec. II, eq.
discrete_laplace: K phi = theta M phi with K_ij = <grad e_i, grad e_j> and
M_ij = <e_i, e_j>), bilinear/trilinear elements on the grid cells: hand-derived
matrices, the tensor-product structure of the full grid, closed-form spectra
of the square and the cube, scipy's generalised eigensolver, inertia counts,
and the apply in the M-inner product (alpha = 0, 2, -2, the sine mode, O(h^2)
convergence to the continuum solution)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    text = [ln for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and not ln.startswith("#")]
    dim, nx, ny, nz, h = text[0].split()
    dim, nx, ny, nz, h = int(dim), int(nx), int(ny), int(nz), float(h)
    nm = ny * nz
    mask = np.array([[int(v) for v in r.split()] for r in text[1:1 + nm]], np.uint8)
    mask = mask.reshape((nz, ny, nx) if dim == 3 else (ny, nx))
    rest = text[1 + nm:]
    ki, mi = rest.index("K\n"), rest.index("M\n")
    K = np.array([[float(v) for v in r.split()] for r in rest[ki + 1:mi]])
    M = np.array([[float(v) for v in r.split()] for r in rest[mi + 1:]])
    return mask, h, K, M


def _mu(m):
    """1-D generalised eigenvalues of the linear elements (stiffness over mass
    of the discrete sine j): (6/h^2)(1 - cos(j pi h)) / (2 + cos(j pi h))."""
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


def test_fem_matches_hand_derived_matrices():
    mask, h, K3, M36 = _read("fem_2d_3x2.txt")
    _, K, M = O.assemble_fem(mask, h)
    np.testing.assert_allclose(K.dense() * 3, K3, rtol=0, atol=1e-13)
    np.testing.assert_allclose(M.dense() * 36 / h ** 2, M36, rtol=0, atol=1e-13)
    mask, h, K12, M216 = _read("fem_3d_2x2x2.txt")
    _, K, M = O.assemble_fem(mask, h)
    np.testing.assert_allclose(K.dense() * 12 / h, K12, rtol=0, atol=1e-12)
    np.testing.assert_allclose(M.dense() * 216 / h ** 3, M216, rtol=0, atol=1e-12)
    for A in (K, M):
        for i in range(A.n):
            assert np.all(np.diff(A.col[A.rowptr[i]:A.rowptr[i + 1]]) > 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_single_node(dim):
    """One dof: K = dim (2/h)(2h/3)^(dim-1), M = (2h/3)^dim, theta = K/M = 3 dim/h^2."""
    h = 0.25
    mask = np.ones((1,) * dim, np.uint8)
    _, K, M = O.assemble_fem(mask, h)
    k = dim * (2 / h) * (2 * h / 3) ** (dim - 1)
    m = (2 * h / 3) ** dim
    assert abs(K.val[0] - k) <= 1e-15 * k and abs(M.val[0] - m) <= 1e-15 * m
    th, _ = O.eig_pencil(K.dense(), M.dense())
    assert abs(th[0] - 3.0 * dim / h ** 2) <= 1e-14 * th[0]


@pytest.mark.parametrize("dim,m", [(2, 7), (3, 4)])
def test_full_grid_is_the_tensor_product(dim, m):
    """On the full grid K = sum_d (K1 on axis d, M1 on the others), M = M1 x
    ... x M1 with the 1-D linear-element matrices K1 = tridiag(-1, 2, -1)/h and
    M1 = h tridiag(1, 4, 1)/6."""
    h = 1.0 / (m + 1)
    e = np.ones(m - 1)
    K1 = (np.diag(2 * np.ones(m)) - np.diag(e, 1) - np.diag(e, -1)) / h
    M1 = h * (np.diag(4 * np.ones(m)) + np.diag(e, 1) + np.diag(e, -1)) / 6

    def kron_all(mats):
        out = mats[0]
        for a in mats[1:]:
            out = np.kron(out, a)
        return out

    # dof index = x + m y (+ m^2 z): the slowest axis is the leftmost Kronecker factor
    Kref = sum(kron_all([K1 if d == ax else M1 for d in range(dim)]) for ax in range(dim))
    Mref = kron_all([M1] * dim)
    _, K, M = O.assemble_fem(np.ones((m,) * dim, np.uint8), h)
    np.testing.assert_allclose(K.dense(), Kref, rtol=0, atol=1e-12 * np.abs(Kref).max())
    np.testing.assert_allclose(M.dense(), Mref, rtol=0, atol=1e-14 * np.abs(Mref).max())


def test_masked_is_principal_submatrix_and_row_sums():
    p = I.ellipse_problem(20, seed=31)
    _, K, M = O.assemble_fem(p.mask, p.h)
    _, Kf, Mf = O.assemble_fem(np.ones_like(p.mask), p.h)
    keep = np.nonzero(p.mask.reshape(-1))[0]
    np.testing.assert_array_equal(K.dense(), Kf.dense()[np.ix_(keep, keep)])
    np.testing.assert_array_equal(M.dense(), Mf.dense()[np.ix_(keep, keep)])
    # rows whose 3 x 3 box lies inside the mask: constants are in the kernel of the
    # gradient (K row sum 0) and the hats sum to one (M row sum = int e_i = h^2)
    Kd, Md = K.dense(), M.dense()
    m = p.mask.astype(bool)
    full = np.zeros_like(m)
    full[1:-1, 1:-1] = np.all([m[1 + dy:m.shape[0] - 1 + dy, 1 + dx:m.shape[1] - 1 + dx]
                               for dy in (-1, 0, 1) for dx in (-1, 0, 1)], axis=0)
    rows = np.nonzero(full.reshape(-1)[keep])[0]
    assert rows.size > 20
    assert np.abs(Kd[rows].sum(axis=1)).max() <= 1e-12
    assert np.abs(Md[rows].sum(axis=1) - p.h ** 2).max() <= 1e-16


@pytest.mark.parametrize("dim,m", [(2, 12), (2, 23), (3, 5)])
def test_pencil_closed_form(dim, m):
    """Square/cube: the discrete sines are generalised eigenvectors with
    theta = sum_d mu_{j_d}, mu_j = (6/h^2)(1 - cos(j pi h))/(2 + cos(j pi h))."""
    p = I.square_problem(m, n_poly=0) if dim == 2 else None
    mask = np.ones((m,) * dim, np.uint8)
    h = 1.0 / (m + 1)
    _, K, M = O.assemble_fem(mask, h)
    th, Phi = O.eig_pencil(K.dense(), M.dense())
    ref = _closed(m, dim)
    assert np.max(np.abs(th - ref) / ref) <= 1e-12
    n = K.n
    assert np.abs(Phi.T @ M.dense() @ Phi - np.eye(n)).max() <= 1e-12
    R = K.dense() @ Phi - M.dense() @ Phi * th
    assert np.abs(R).max() <= 1e-12 * th[-1] * np.abs(M.dense()).max()
    if p is not None:
        assert p.n == n


def test_pencil_matches_scipy_and_inertia():
    sl = pytest.importorskip("scipy.linalg")
    p = I.ellipse_problem(22, seed=5)
    _, K, M = O.assemble_fem(p.mask, p.h)
    th, Phi = O.eig_pencil(K.dense(), M.dense())
    ref = sl.eigh(K.dense(), M.dense(), eigvals_only=True)
    assert np.max(np.abs(th - ref) / ref) <= 1e-12
    rng = np.random.default_rng(2)
    for sigma in rng.uniform(0, th[-1] * 1.05, size=20):
        if np.min(np.abs(th - sigma)) < 1e-6 * sigma:
            continue
        assert O.count_below_pencil(K, M, sigma) == int(np.sum(th < sigma))
    with pytest.raises(ValueError):
        O.count_below_pencil(K, O.assemble(p.mask, p.h)[1], 1.0)


@pytest.fixture(scope="module")
def fem_masked():
    p = I.ellipse_problem(20, seed=31)
    _, K, M = O.assemble_fem(p.mask, p.h)
    th, Phi = O.eig_pencil(K.dense(), M.dense())
    return p, K, M, th, Phi


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_apply_mass_special_orders(fem_masked):
    """alpha = 0: the M-orthonormal expansion of f is f; alpha = 2: K u = M f;
    alpha = -2: M u = K f."""
    p, K, M, th, Phi = fem_masked
    k = p.F.shape[1]
    U = O.frac_apply_mass(Phi, th, M, p.F, np.arange(k), np.zeros(k))
    assert _rel(U, p.F) <= 1e-12
    for c in range(3):
        u2 = O.frac_apply_mass(Phi, th, M, p.F[:, c:c + 1], [0, 0], [2.0, -2.0])
        ref2 = O.band_solve(K, O.spmv(M, p.F[:, c]))
        assert _rel(u2[:, 0], ref2) <= 1e-12
        assert _rel(O.spmv(M, u2[:, 1]), O.spmv(K, p.F[:, c])) <= 1e-12


def test_apply_mass_sine_mode_and_planted_mistakes():
    """f = sin(pi x) sin(pi y) is a generalised eigenvector of theta_11 =
    2 mu_1, so u = theta_11^{-alpha/2} f; wrong mass, transposed Phi and
    shifted eigenvalues must fail that."""
    m = 16
    p = I.square_problem(m, n_poly=0)
    _, K, M = O.assemble_fem(p.mask, p.h)
    th, Phi = O.eig_pencil(K.dense(), M.dense())
    t11 = 2 * _mu(m)[0]
    alphas = [0.5, 1.0, 1.5, 2.0]
    f = p.F[:, :1]

    def err(U):
        return max(_rel(U[:, j], t11 ** (-a / 2) * f[:, 0]) for j, a in enumerate(alphas))

    assert err(O.frac_apply_mass(Phi, th, M, f, [0] * 4, alphas)) <= 1e-12
    ident = O.CSR(M.n, M.rowptr, M.col, np.where(M.col == np.repeat(np.arange(M.n), np.diff(M.rowptr)), 1.0, 0.0))
    assert err(O.frac_apply_mass(Phi, th, ident, f, [0] * 4, alphas)) > 1e-3
    assert err(O.frac_apply_mass(np.asfortranarray(Phi.T), th, M, f, [0] * 4, alphas)) > 1e-3
    assert err(O.frac_apply_mass(Phi, np.roll(th, 1), M, f, [0] * 4, alphas)) > 1e-3
    with pytest.raises(RuntimeError):
        O.frac_apply_mass(Phi, th, M, f, [1], [1.0])


@pytest.mark.parametrize("alpha", np.linspace(0.0, 2.0, 11))
def test_apply_mass_continuum_convergence(alpha):
    """Sec. V eqs. (poisson_f, poisson_u) with bilinear elements: the nodal
    solution for f = 2 sin(pi x) sin(pi y) converges at O(h^2) to
    2 (2 pi^2)^{-alpha/2} sin(pi x) sin(pi y) for the 11 orders used there."""
    errs = []
    for m in (7, 15, 31):
        p = I.square_problem(m, n_poly=0)
        _, K, M = O.assemble_fem(p.mask, p.h)
        th, Phi = O.eig_pencil(K.dense(), M.dense())
        u = O.frac_apply_mass(Phi, th, M, 2.0 * p.F[:, :1], [0], [alpha])[:, 0]
        exact = 2.0 * (2 * np.pi ** 2) ** (-alpha / 2) * p.F[:, 0]
        errs.append(np.max(np.abs(u - exact)))
    if alpha == 0.0:
        assert max(errs) <= 1e-12
    else:
        assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
