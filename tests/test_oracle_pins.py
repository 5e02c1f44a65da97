"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test names the passage of arXiv:1911.11906 (or the mathematics) that
fixes the expected value: closed-form spectra of the Dirichlet Laplacian on
the square/cube/strip, hand-derived stencil matrices, special orders of the
spectral apply, Sylvester inertia, interlacing, trace/Frobenius identities,
and a second independent eigensolver (cyclic Jacobi) on small matrices.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I
from conftest import square_closed_form

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    dim, nx, ny, nz = (int(v) for v in rows[0][:4])
    h = float(rows[0][4])
    nmask = ny * nz
    mask = np.array([[int(v) for v in r] for r in rows[1:1 + nmask]], np.uint8)
    mask = mask.reshape((nz, ny, nx) if dim == 3 else (ny, nx))
    A = np.array([[float(v) for v in r] for r in rows[1 + nmask:]])
    return mask, h, A


# --------------------------------------------------------------------------
# Assembly: Sec. II eq. (discrete_laplace), nodal FD reading
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["assemble_2d_3x2.txt", "assemble_3d_2x2x2.txt"])
def test_assembly_matches_hand_derived_matrix(name):
    mask, h, Aref = _read_golden(name)
    idx, A = O.assemble(mask, h)
    assert A.n == Aref.shape[0]
    np.testing.assert_array_equal(A.dense(), Aref)
    # dof numbering: row-major over kept nodes
    flat = mask.reshape(-1)
    assert list(idx[flat == 1]) == list(range(A.n))
    assert np.all(idx[flat == 0] == -1)
    # columns strictly ascending within each row (canonical CSR)
    for i in range(A.n):
        c = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_assembly_edge_count_identity():
    p = I.ellipse_problem(24, seed=77)
    _, A = O.assemble(p.mask, p.h)
    m = p.mask.astype(int)
    edges = int((m[:, 1:] & m[:, :-1]).sum() + (m[1:, :] & m[:-1, :]).sum())
    assert A.nnz == A.n + 2 * edges
    D = A.dense()
    np.testing.assert_array_equal(D, D.T)


def test_empty_and_single_node_masks():
    idx, A = O.assemble(np.zeros((4, 5), np.uint8), 0.25)
    assert A.n == 0 and A.nnz == 0 and np.all(idx == -1)
    mask = np.zeros((3, 3), np.uint8)
    mask[1, 1] = 1
    _, A = O.assemble(mask, 0.25)
    lam, V = O.eig_full(A.dense())
    assert lam[0] == 4.0 / 0.25 ** 2 and abs(abs(V[0, 0]) - 1.0) == 0.0


def test_two_node_brute_force():
    mask = np.zeros((3, 4), np.uint8)
    mask[1, 1:3] = 1
    h = 0.2
    _, A = O.assemble(mask, h)
    lam, _ = O.eig_full(A.dense())
    np.testing.assert_allclose(lam, [3.0 / h ** 2, 5.0 / h ** 2], rtol=1e-15)


# --------------------------------------------------------------------------
# Closed-form spectra (the discrete Fourier modes of Sec. V on the square/cube)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m", [1, 5, 12, 20])
def test_square_closed_form(m):
    p = I.square_problem(m, n_poly=0)
    _, A = O.assemble(p.mask, p.h)
    lam, V = O.eig_full(A.dense())
    ref = square_closed_form(m, 2)
    assert np.max(np.abs(lam - ref) / ref) <= 1e-13


def test_square48_closed_form(square48):
    p, A, lam, V = square48
    ref = square_closed_form(48, 2)
    # backward-stable bound: |error| <= c(n) eps ||A||_2, c(n) = 4 sqrt(n)
    assert np.max(np.abs(lam - ref)) <= 4 * np.sqrt(lam.size) * np.finfo(float).eps * ref[-1]
    assert np.max(np.abs(lam - ref) / ref) <= 5e-12
    # lambda_11 = (8/h^2) sin^2(pi h / 2) ~ 19.73 at h = 1/49
    assert abs(lam[0] - 8.0 / p.h ** 2 * np.sin(np.pi * p.h / 2) ** 2) <= 5e-12 * lam[0]
    assert abs(lam[0] - 19.732) < 1e-3


@pytest.mark.parametrize("m", [3, 6])
def test_cube_closed_form(m):
    h = 1.0 / (m + 1)
    mask = np.ones((m, m, m), np.uint8)
    _, A = O.assemble(mask, h)
    lam, _ = O.eig_full(A.dense())
    ref = square_closed_form(m, 3)
    assert np.max(np.abs(lam - ref) / ref) <= 1e-13


def test_strip_closed_form_fig2():
    """A one-row strip: the 1-D modes of Fig. 2 shifted by the 2/h^2 that the
    2-D stencil adds for the two missing vertical neighbours."""
    m = 20
    h = 1.0 / (m + 1)
    mask = np.ones((1, m), np.uint8)
    _, A = O.assemble(mask, h)
    lam, _ = O.eig_full(A.dense())
    k = np.arange(1, m + 1)
    ref = 2.0 / h ** 2 + 4.0 / h ** 2 * np.sin(k * np.pi * h / 2) ** 2
    np.testing.assert_allclose(lam, ref, rtol=1e-14)


# --------------------------------------------------------------------------
# Independent second route: cyclic Jacobi on small matrices
# --------------------------------------------------------------------------
def test_jacobi_closed_form():
    p = I.square_problem(6, n_poly=0)
    _, A = O.assemble(p.mask, p.h)
    lam, V = O.eig_jacobi(A.dense())
    ref = square_closed_form(6, 2)
    assert np.max(np.abs(lam - ref) / ref) <= 1e-13
    D = A.dense()
    assert np.linalg.norm(D @ V - V * lam) <= 1e-13 * np.linalg.norm(D)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 33, 64])
def test_householder_ql_agrees_with_jacobi(n):
    rng = np.random.default_rng(100 + n)
    B = rng.standard_normal((n, n))
    A = np.asfortranarray(B + B.T)
    l1, V1 = O.eig_full(A)
    l2, V2 = O.eig_jacobi(A)
    nrm = np.linalg.norm(A, 2)
    assert np.max(np.abs(l1 - l2)) <= 1e-13 * nrm
    # random matrices have simple spectra: compare spectral projectors
    for i in range(n):
        P1 = np.outer(V1[:, i], V1[:, i])
        P2 = np.outer(V2[:, i], V2[:, i])
        gap = np.min(np.abs(np.delete(l1, i) - l1[i])) if n > 1 else nrm
        assert np.max(np.abs(P1 - P2)) <= 1e-12 * nrm / gap + 1e-14


def test_masked_small_grid_ql_vs_jacobi():
    p = I.ellipse_problem(10, n_ellipses=3, seed=5)
    _, A = O.assemble(p.mask, p.h)
    D = A.dense()
    l1, _ = O.eig_full(D)
    l2, _ = O.eig_jacobi(D)
    assert np.max(np.abs(l1 - l2) / l2) <= 1e-13


# --------------------------------------------------------------------------
# Tridiagonal stage
# --------------------------------------------------------------------------
def test_tridiagonal_closed_form():
    n = 50
    d = np.full(n, 2.0)
    e = np.full(n - 1, -1.0)
    lam, Z = O.tridiag_eig(d, e)
    k = np.arange(1, n + 1)
    ref = 2.0 - 2.0 * np.cos(k * np.pi / (n + 1))
    np.testing.assert_allclose(lam, ref, rtol=1e-13, atol=1e-15)
    # the eigenvectors are the discrete sines
    s = np.sin(np.outer(np.arange(1, n + 1), k) * np.pi / (n + 1))
    s /= np.linalg.norm(s, axis=0)
    assert np.max(np.abs(np.abs(Z.T @ s) - np.eye(n))) <= 1e-12


def test_tridiagonal_vs_jacobi_and_values_only():
    rng = np.random.default_rng(7)
    n = 40
    d = rng.standard_normal(n)
    e = rng.standard_normal(n - 1)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    l1, Z = O.tridiag_eig(d, e)
    l2, _ = O.eig_jacobi(T)
    l3, _ = O.tridiag_eig(d, e, want_vectors=False)
    assert np.max(np.abs(l1 - l2)) <= 1e-13 * np.abs(l2).max()
    np.testing.assert_array_equal(l1, l3)
    assert np.linalg.norm(T @ Z - Z * l1) <= 1e-13 * np.linalg.norm(T)


def test_tridiagonal_iteration_cap_reports_failure():
    d = np.arange(10, dtype=float)
    e = np.ones(9)
    with pytest.raises(RuntimeError):
        O.tridiag_eig(d, e, max_steps=1)


def test_householder_reduction_properties():
    p = I.ellipse_problem(12, n_ellipses=4, seed=11)
    _, A = O.assemble(p.mask, p.h)
    D = A.dense()
    d, e, Q = O.tridiagonalize(D)
    n = A.n
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    nrm = np.linalg.norm(D)
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 1e-14 * n
    assert np.linalg.norm(Q @ T @ Q.T - D) <= 1e-14 * n * nrm


# --------------------------------------------------------------------------
# Invariants on irregular masks
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def masked():
    p = I.ellipse_problem(24, seed=1234)
    _, A = O.assemble(p.mask, p.h)
    lam, V = O.eig_full(A.dense())
    return p, A, lam, V


def test_trace_and_frobenius(masked):
    p, A, lam, _ = masked
    m = p.mask.astype(int)
    edges = int((m[:, 1:] & m[:, :-1]).sum() + (m[1:, :] & m[:-1, :]).sum())
    h = p.h
    assert abs(lam.sum() - 4 * A.n / h ** 2) <= 1e-12 * 4 * A.n / h ** 2
    fro2 = (16 * A.n + 2 * edges) / h ** 4
    assert abs((lam ** 2).sum() - fro2) <= 1e-12 * fro2


def test_gershgorin_and_interlacing(masked):
    p, A, lam, _ = masked
    h = p.h
    assert lam[0] > 0 and lam[-1] <= 8 / h ** 2 * (1 + 1e-14)
    full = square_closed_form(p.mask.shape[0], 2)
    N, n = full.size, A.n
    tol = 1e-12 * full[-1]
    assert np.all(full[:n] <= lam + tol)
    assert np.all(lam <= full[N - n:] + tol)


def test_inertia_counts_match_spectrum(masked):
    """Sec. III-D-2: negative pivots of LDL^T(A - sigma I) = #{lambda < sigma}."""
    p, A, lam, _ = masked
    rng = np.random.default_rng(3)
    for sigma in rng.uniform(0, 8 / p.h ** 2, size=25):
        gap = np.min(np.abs(lam - sigma))
        if gap < 1e-6 * sigma:
            continue
        assert O.count_below(A, sigma) == int(np.sum(lam < sigma))


def test_inertia_counts_closed_form():
    m = 16
    p = I.square_problem(m, n_poly=0)
    _, A = O.assemble(p.mask, p.h)
    ref = square_closed_form(m, 2)
    for sigma in np.linspace(1.0, ref[-1] * 1.01, 37):
        if np.min(np.abs(ref - sigma)) < 1e-6 * sigma:
            continue
        assert O.count_below(A, sigma) == int(np.sum(ref < sigma))


# --------------------------------------------------------------------------
# Spectral apply: Sec. II eq. (poisson_solution) and its discrete sums
# --------------------------------------------------------------------------
def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_apply_alpha0_returns_forcing(masked):
    """alpha = 0: v is g, the eigen-expansion of f, which is f (Fig. 1, Sec. II)."""
    p, A, lam, V = masked
    U = O.frac_apply(V, lam, p.F, np.arange(p.F.shape[1], dtype=np.int32), np.zeros(p.F.shape[1]))
    assert _rel(U, p.F) <= 1e-13


def test_apply_alpha2_is_direct_solve(masked):
    """alpha = 2: the integer-order Poisson problem A u = f (Fig. 1)."""
    p, A, lam, V = masked
    for c in range(3):
        u = O.frac_apply(V, lam, p.F[:, c:c + 1], [0], [2.0])[:, 0]
        assert _rel(u, O.band_solve(A, p.F[:, c])) <= 1e-12


def test_apply_negative_orders_are_stencil_powers(masked):
    """alpha = -2 and -4: the forward operator of eq. (spectral_definition)."""
    p, A, lam, V = masked
    f = p.F[:, 0]
    Af = O.spmv(A, f)
    u = O.frac_apply(V, lam, f[:, None], [0, 0], [-2.0, -4.0])
    assert _rel(u[:, 0], Af) <= 1e-12
    assert _rel(u[:, 1], O.spmv(A, Af)) <= 1e-12


def test_apply_semigroup(masked):
    p, A, lam, V = masked
    f = p.F[:, 1]
    u1 = O.frac_apply(V, lam, f[:, None], [0], [0.7])[:, 0]
    u2 = O.frac_apply(V, lam, u1[:, None], [0], [0.6])[:, 0]
    u3 = O.frac_apply(V, lam, f[:, None], [0], [1.3])[:, 0]
    assert _rel(u2, u3) <= 1e-12


def _sine_mode_error(U, p, lam11, alphas):
    f = p.F[:, 0]
    return max(_rel(U[:, j], lam11 ** (-a / 2) * f) for j, a in enumerate(alphas))


def test_apply_sine_mode_square48(square48):
    """f = sin(pi x) sin(pi y) is the exact discrete eigenvector of lambda_11,
    so u = lambda_11^{-alpha/2} f (discrete form of eqs. poisson_f/poisson_u)."""
    p, A, lam, V = square48
    alphas = [0.5, 1.0, 1.5, 2.0]
    lam11 = 8.0 / p.h ** 2 * np.sin(np.pi * p.h / 2) ** 2
    U = O.frac_apply(V, lam, p.F[:, :1], [0] * 4, alphas)
    # error budget: lambda_11 carries ~1e-12 relative error (kappa * eps), times alpha/2
    assert _sine_mode_error(U, p, lam11, alphas) <= 5e-12


def test_pins_catch_planted_mistakes(square48):
    """Mistakes planted in oracle outputs must trip the pins above."""
    p, A, lam, V = square48
    alphas = [0.5, 1.0, 1.5, 2.0]
    lam11 = 8.0 / p.h ** 2 * np.sin(np.pi * p.h / 2) ** 2
    # wrong sign of the exponent
    U = O.frac_apply(V, lam, p.F[:, :1], [0] * 4, [-a for a in alphas])
    assert _sine_mode_error(U, p, lam11, alphas) > 1e-3
    # a transposed operand: V^T instead of V
    U = O.frac_apply(np.asfortranarray(V.T), lam, p.F[:, :1], [0] * 4, alphas)
    assert _sine_mode_error(U, p, lam11, alphas) > 1e-3
    # eigenvalues off by one index
    U = O.frac_apply(V, np.roll(lam, 1), p.F[:, :1], [0] * 4, alphas)
    assert _sine_mode_error(U, p, lam11, alphas) > 1e-3
    # a dropped stencil term changes the trace identity
    ref = square_closed_form(48, 2)
    assert np.max(np.abs((lam - 1.0 / p.h ** 2) - ref) / ref) > 1e-3


@pytest.mark.parametrize("alpha", np.linspace(0.0, 2.0, 11))
def test_continuum_convergence_e8(alpha):
    """Sec. V eqs. (poisson_f, poisson_u): f = 2 sin(pi x) sin(pi y) has
    u = 2 (2 pi^2)^{-alpha/2} sin(pi x) sin(pi y); the FD solution converges
    at O(h^2) for the 11 orders used there."""
    errs = []
    for m in (7, 15, 31):
        p = I.square_problem(m, n_poly=0)
        _, A = O.assemble(p.mask, p.h)
        lam, V = O.eig_full(A.dense())
        f = 2.0 * p.F[:, 0]
        u = O.frac_apply(V, lam, f[:, None], [0], [alpha])[:, 0]
        exact = 2.0 * (2 * np.pi ** 2) ** (-alpha / 2) * p.F[:, 0]
        errs.append(np.max(np.abs(u - exact)))
    if alpha == 0.0:
        assert max(errs) <= 1e-13
    else:
        assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


# --------------------------------------------------------------------------
# Fractional diffusion: Sec. II eq. (diffusion_solution)
# --------------------------------------------------------------------------
def test_diffusion_time_zero_and_alpha0(masked):
    """t = 0 returns the initial state; alpha = 0 decays every mode alike,
    u(t) = exp(-mu t) u0."""
    p, A, lam, V = masked
    k = p.F.shape[1]
    U = O.frac_diffusion(V, lam, p.F, np.arange(k), np.full(k, 1.3), np.zeros(k), mu=2.0)
    assert _rel(U, p.F) <= 1e-13
    U = O.frac_diffusion(V, lam, p.F[:, :1], [0], [0.0], [0.3], mu=2.0)[:, 0]
    assert _rel(U, np.exp(-0.6) * p.F[:, 0]) <= 1e-13


@pytest.mark.parametrize("mu,t", [(1.0, 1e-4), (2.5, 1e-3)])
def test_diffusion_alpha2_is_matrix_exponential(masked, mu, t):
    """alpha = 2: the heat equation, u(t) = expm(-mu t A) u0 (scipy's Pade
    scaling and squaring on the dense matrix, no eigenvectors involved).  t is
    small enough that the top of the spectrum has not decayed away."""
    sl = pytest.importorskip("scipy.linalg")
    p, A, lam, V = masked
    E = sl.expm(-mu * t * A.dense())
    for c in range(3):
        u = O.frac_diffusion(V, lam, p.F[:, c:c + 1], [0], [2.0], [t], mu=mu)[:, 0]
        assert _rel(u, E @ p.F[:, c]) <= 1e-12


def test_diffusion_alpha4_and_alpha1_match_matrix_functions(masked):
    """alpha = 4: expm(-mu t A^2); alpha = 1: expm(-mu t sqrtm(A)) with scipy's
    Schur-based square root."""
    sl = pytest.importorskip("scipy.linalg")
    p, A, lam, V = masked
    D = A.dense()
    f = p.F[:, 2]
    u = O.frac_diffusion(V, lam, f[:, None], [0, 0], [4.0, 1.0], [2e-8, 1e-2], mu=1.5)
    assert _rel(u[:, 0], sl.expm(-1.5 * 2e-8 * (D @ D)) @ f) <= 1e-11
    R = np.real(sl.sqrtm(D))
    assert _rel(u[:, 1], sl.expm(-1.5 * 1e-2 * R) @ f) <= 1e-10


def test_diffusion_semigroup(masked):
    """Evolving to t1 and then by t2 equals evolving to t1 + t2."""
    p, A, lam, V = masked
    f = p.F[:, 1]
    u1 = O.frac_diffusion(V, lam, f[:, None], [0], [1.2], [3e-3], mu=0.8)
    u2 = O.frac_diffusion(V, lam, u1, [0], [1.2], [5e-3], mu=0.8)[:, 0]
    u3 = O.frac_diffusion(V, lam, f[:, None], [0], [1.2], [8e-3], mu=0.8)[:, 0]
    assert _rel(u2, u3) <= 1e-12


def _decay_error(U, p, lam11, alphas, t, mu):
    u0 = 2.0 * p.F[:, 0]
    return max(_rel(U[:, j], np.exp(-mu * lam11 ** (a / 2) * t) * u0) for j, a in enumerate(alphas))


DIFF_ALPHAS = list(np.linspace(0.0, 2.0, 11))


@pytest.mark.parametrize("mu", [1.0, 2.5])
def test_diffusion_sine_mode_square48(square48, mu):
    """u0 = 2 sin(pi x) sin(pi y) is the exact discrete eigenvector of
    lambda_11, so u(t) = exp(-mu lambda_11^{alpha/2} t) u0 (discrete form of
    eqs. diffusion_ics/diffusion_sols at the paper's t = 0.4 and 11 orders)."""
    p, A, lam, V = square48
    lam11 = 8.0 / p.h ** 2 * np.sin(np.pi * p.h / 2) ** 2
    k = len(DIFF_ALPHAS)
    U = O.frac_diffusion(V, lam, 2.0 * p.F[:, :1], [0] * k, DIFF_ALPHAS, [0.4] * k, mu=mu)
    # lambda_11 carries ~1e-12 relative error; the exponent mu lambda^{alpha/2} t <= 20 amplifies it
    assert _decay_error(U, p, lam11, DIFF_ALPHAS, 0.4, mu) <= 5e-11


def test_diffusion_pins_catch_planted_mistakes(square48, masked):
    """Mistakes planted in the oracle's inputs must trip the diffusion pins."""
    p, A, lam, V = square48
    lam11 = 8.0 / p.h ** 2 * np.sin(np.pi * p.h / 2) ** 2
    k = len(DIFF_ALPHAS)
    u0 = 2.0 * p.F[:, :1]
    err = lambda U, mu=2.5: _decay_error(U, p, lam11, DIFF_ALPHAS, 0.4, mu)
    # growth instead of decay (sign of the exponent)
    assert err(O.frac_diffusion(V, lam, u0, [0] * k, DIFF_ALPHAS, [-0.4] * k, mu=2.5)) > 1e-3
    # mu dropped
    assert err(O.frac_diffusion(V, lam, u0, [0] * k, DIFF_ALPHAS, [0.4] * k, mu=1.0)) > 1e-3
    # lambda^alpha instead of lambda^{alpha/2}
    assert err(O.frac_diffusion(V, lam, u0, [0] * k, [2 * a for a in DIFF_ALPHAS], [0.4] * k, mu=2.5)) > 1e-3
    # eigenvalues off by one index
    assert err(O.frac_diffusion(V, np.roll(lam, 1), u0, [0] * k, DIFF_ALPHAS, [0.4] * k, mu=2.5)) > 1e-3
    # a transposed operand on a general initial state: caught by the matrix exponential
    sl = pytest.importorskip("scipy.linalg")
    pm, Am, lm, Vm = masked
    f = pm.F[:, 0]
    ref = sl.expm(-1e-4 * Am.dense()) @ f
    bad = O.frac_diffusion(np.asfortranarray(Vm.T), lm, f[:, None], [0], [2.0], [1e-4])[:, 0]
    assert _rel(bad, ref) > 1e-3


def test_diffusion_rejects_bad_pairs(masked):
    p, A, lam, V = masked
    with pytest.raises(RuntimeError):
        O.frac_diffusion(V, lam, p.F[:, :1], [1], [1.0], [0.1])
    with pytest.raises(ValueError):
        O.frac_diffusion(V, lam, p.F[:, :1], [0, 0], [1.0], [0.1, 0.2])


@pytest.mark.parametrize("alpha", DIFF_ALPHAS)
def test_diffusion_continuum_convergence(alpha):
    """Sec. V eqs. (diffusion_ics, diffusion_sols): u0 = 2 sin(pi x) sin(pi y)
    has u = 2 exp(-mu (2 pi^2)^{alpha/2} t) sin(pi x) sin(pi y); at the
    paper's t = 0.4, mu = 1 the FD solution converges at O(h^2)."""
    errs = []
    for m in (7, 15, 31):
        p = I.square_problem(m, n_poly=0)
        _, A = O.assemble(p.mask, p.h)
        lam, V = O.eig_full(A.dense())
        u0 = 2.0 * p.F[:, 0]
        u = O.frac_diffusion(V, lam, u0[:, None], [0], [alpha], [0.4], mu=1.0)[:, 0]
        exact = 2.0 * np.exp(-(2 * np.pi ** 2) ** (alpha / 2) * 0.4) * p.F[:, 0]
        errs.append(np.max(np.abs(u - exact)))
    if alpha == 0.0:
        assert max(errs) <= 1e-13
    else:
        assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
