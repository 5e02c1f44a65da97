"""GPU parity of frac_diffusion, the fractional diffusion solution
u(t) = V diag(exp(-mu lambda^{alpha/2} t)) V^T u0 (Sec. II, eq.
diffusion_solution), against the FP64 CPU oracle; every call goes through
the C ABI.  The decomposition is the oracle's where the apply alone is under
test, and the GPU's own (both routes) where the whole path is."""
import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALPHAS = (0.0, 0.5, 1.3, 2.0, 3.5, -1.0)
TIMES = (0.0, 1e-3, 0.05, 0.4, -1e-4)


def _F():
    import paper_1911_11906_gb300 as F
    return F


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _colmajor(a):
    a = np.asfortranarray(a, dtype=np.float64)
    return torch.from_numpy(a.T.copy()).cuda().t()


@pytest.fixture(scope="module")
def masked44():
    """n = 1238: nine 128-row tiles and a ragged tail of 86 rows."""
    p = I.ellipse_problem(44, seed=9)
    _, A = O.assemble(p.mask, p.h)
    lam, V = O.eig_full(A.dense())
    return p, A, lam, V


def _pairs(m, alphas=ALPHAS):
    pf, pa, pt = [], [], []
    for f in range(m):
        for a in alphas:
            for t in TIMES:
                if t < 0 and a > 1:  # backward in time the top modes grow past the double range
                    continue
                pf.append(f)
                pa.append(a)
                pt.append(t)
    return np.array(pf, np.int32), np.array(pa), np.array(pt)


def _check_columns(U, U_o, tol):
    """Element by element, relative to each column's largest entry."""
    scale = np.maximum(np.max(np.abs(U_o), axis=0), 1e-300)
    assert np.max(np.abs(U - U_o) / scale) <= tol


# FP64 products (and 7 slices, FP64 level): two length-n dot products per
# entry, each within n eps of the sum of magnitudes, bounded here by the
# column's largest entry: 4 n eps = 5.5e-13 at n = 1238.  5 slices carry 40
# bits: 2 n 2^-40 = 2.3e-9 on the same scale.
@pytest.mark.parametrize("slices,tol", [(0, 4 * 1238 * 2.0 ** -53), (7, 4 * 1238 * 2.0 ** -53),
                                        (5, 2 * 1238 * 2.0 ** -40)])
def test_diffusion_matches_oracle(masked44, slices, tol):
    F = _F()
    p, A, lam, V = masked44
    assert p.n == 1238
    U0 = p.F[:, :6]
    pf, pa, pt = _pairs(U0.shape[1])
    U_o = O.frac_diffusion(V, lam, U0, pf, pa, pt, mu=1.7)
    ctx = F.Context()
    ctx.set_apply_slices(slices)
    U = F.frac_diffusion(_colmajor(V), _cuda(lam), _colmajor(U0), pf, pa, pt, mu=1.7, ctx=ctx).cpu().numpy()
    _check_columns(U, U_o, tol)


@pytest.mark.parametrize("route", ["fp64", "mixed"])
def test_diffusion_whole_path_closed_form(square48, route):
    """The whole path on the GPU (assembly, eigenpairs, diffusion) on the
    48 x 48 square: u0 = 2 sin(pi x) sin(pi y) is the discrete eigenvector of
    lambda_11, so u(t) = exp(-mu lambda_11^{alpha/2} t) u0 at the paper's
    t = 0.4 and 11 orders; and every other initial state against the
    oracle's own decomposition and diffusion."""
    F = _F()
    p, A, lam_o, V_o = square48
    ctx = F.Context(band_width=64 if route == "mixed" else 32)
    asm = F.fd_assemble(_cuda(p.mask), p.h, ctx=ctx)
    if route == "mixed":
        lam, V = F.eig_full_mixed(asm["A"], asm["rowptr"], asm["col"], asm["val"], refine_iters=6, ctx=ctx)
    else:
        lam, V = F.eig_full(asm["A"], ctx=ctx)
    lam11 = 8.0 / p.h ** 2 * np.sin(np.pi * p.h / 2) ** 2

    def tol(mu, a, t):
        # eigenvalues within 1e-11 relative on each side; the dominant mode's
        # exponent x = mu t lambda_11^{alpha/2} turns a relative error d of
        # lambda into (alpha/2) x d of u
        return 1e-11 + (abs(a) / 2) * abs(mu * t * lam11 ** (a / 2)) * 2e-11

    alphas = np.linspace(0.0, 2.0, 11)
    k = len(alphas)
    u0 = 2.0 * p.F[:, :1]
    for mu in (1.0, 2.5):
        U = F.frac_diffusion(V, lam, _colmajor(u0), [0] * k, alphas, [0.4] * k, mu=mu, ctx=ctx).cpu().numpy()
        for j, a in enumerate(alphas):
            ref = np.exp(-mu * lam11 ** (a / 2) * 0.4) * u0[:, 0]
            assert np.linalg.norm(U[:, j] - ref) <= tol(mu, a, 0.4) * np.linalg.norm(ref), (mu, a)
    # orders up to 2: the smooth initial states are dominated by the lowest modes
    pf, pa, pt = _pairs(p.F.shape[1], [a for a in ALPHAS if a <= 2.0])
    U_o = O.frac_diffusion(V_o, lam_o, p.F, pf, pa, pt, mu=0.9)
    U = F.frac_diffusion(V, lam, _colmajor(p.F), pf, pa, pt, mu=0.9, ctx=ctx).cpu().numpy()
    # the solution is unique even where eigenvectors are not: compare u only
    for j in range(U.shape[1]):
        assert np.linalg.norm(U[:, j] - U_o[:, j]) <= tol(0.9, pa[j], pt[j]) * np.linalg.norm(U_o[:, j]), j


def test_diffusion_edge_cases(masked44):
    F = _F()
    p, A, lam, V = masked44
    Vd, ld = _colmajor(V), _cuda(lam)
    U0 = _colmajor(p.F[:, :3])
    # t = 0 returns the initial state, alpha = 0 decays by exp(-mu t), repeated states
    U = F.frac_diffusion(Vd, ld, U0, [0, 1, 1, 2], [1.5, 0.0, 0.0, 2.0], [0.0, 0.3, 0.0, 0.0], mu=2.0).cpu().numpy()
    for j, (c, s) in enumerate([(0, 1.0), (1, np.exp(-0.6)), (1, 1.0), (2, 1.0)]):
        ref = s * p.F[:, c]
        assert np.linalg.norm(U[:, j] - ref) <= 1e-13 * np.linalg.norm(ref), j
    # a large time decays every mode to (numerical) zero without overflow or NaN
    U = F.frac_diffusion(Vd, ld, U0, [0], [2.0], [1e4]).cpu().numpy()
    assert np.all(np.isfinite(U)) and np.max(np.abs(U)) == 0.0
    # no pairs: nothing to do
    assert F.frac_diffusion(Vd, ld, U0, [], [], []).shape == (p.n, 0)
    # a non-positive eigenvalue with alpha != 0 is reported; alpha = 0 never evaluates the power
    bad = lam.copy()
    bad[5] = 0.0
    with pytest.raises(F.FraclapError) as ei:
        F.frac_diffusion(Vd, _cuda(bad), U0, [0], [1.0], [0.1])
    assert ei.value.code == -2
    F.frac_diffusion(Vd, _cuda(bad), U0, [0], [0.0], [0.1])
    # a pair index outside the initial states is reported by the kernel's own check
    with pytest.raises(F.FraclapError) as ei:
        F.frac_diffusion(Vd, ld, U0, [3], [1.0], [0.1])
    assert ei.value.code == -1
    # a non-finite diffusion coefficient is refused before any launch
    with pytest.raises(F.FraclapError) as ei:
        F.frac_diffusion(Vd, ld, U0, [0], [1.0], [0.1], mu=float("inf"))
    assert ei.value.code == -1
    with pytest.raises(ValueError):
        F.frac_diffusion(Vd, ld, U0, [0, 1], [1.0], [0.1, 0.2])
