"""GPU parity of exact eigenvalue counting and spectrum slicing (Sec. III-D)
against the oracle: inertia counts of the banded LDL^T of A - sigma I and of
K - sigma M (shared-memory and global windows), Sturm counts and bisection
on the tridiagonal form, and the greedy partitioning.  Counts are integers
and are compared exactly; the GPU forms its pivots with the same operations
in the same order as the oracle, so the bisected eigenvalues and the
partition's split points are compared bit for bit too."""
import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _F():
    import paper_1911_11906_gb300 as F
    return F


def _csr_cuda(A, val=None):
    return (torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.col).cuda(),
            torch.from_numpy(A.val if val is None else val).cuda())


def _grid(name):
    """(mask, h) of a named test grid."""
    if name == "square24":
        return I.square_mask(24), 1.0 / 25
    if name == "ellipse40":
        p = I.ellipse_problem(40, n_ellipses=4, seed=7)
        return p.mask, p.h
    if name == "cube7":
        return I.square_mask(7, dim=3), 1.0 / 8
    if name == "strip":
        return np.ones((1, 40), dtype=np.uint8), 1.0 / 41
    raise ValueError(name)


def _shifts(lam, rng, extra=()):
    """Midpoints between neighbouring eigenvalues (clear of both), random
    points of the spectrum, and points outside it."""
    gaps = np.nonzero(np.diff(lam) > 1e-6 * lam[-1])[0]
    pick = rng.choice(gaps, size=min(24, gaps.size), replace=False)
    mids = 0.5 * (lam[pick] + lam[pick + 1])
    rnd = rng.uniform(lam[0] * 0.5, lam[-1] * 1.1, size=8)
    return np.concatenate([mids, rnd, [lam[0] * 0.25, lam[-1] * 2.0], list(extra)])


@pytest.mark.parametrize("grid", ["square24", "ellipse40", "cube7", "strip"])
def test_inertia_counts_match_oracle(grid):
    """Counts #{lambda < sigma} of the stencil matrix at many shifts, against
    the oracle's banded LDL^T, exactly; bandwidths from 1 (a 1-D strip) to a
    3-D plane."""
    F = _F()
    mask, h = _grid(grid)
    _, A = O.assemble(mask, h)
    lam, _ = O.eig_full(A.dense())
    sig = _shifts(lam, np.random.default_rng(A.n))
    rp, cl, vl = _csr_cuda(A)
    b = F.csr_half_bandwidth(rp, cl)
    assert b == max(int(i - A.col[q]) for i in range(A.n) for q in range(A.rowptr[i], A.rowptr[i + 1])
                    if A.col[q] <= i)
    got = F.inertia_counts(rp, cl, vl, sig).cpu().numpy()
    want = np.array([O.count_below(A, s) for s in sig])
    assert np.array_equal(got, want)
    # the counts also follow from the spectrum itself
    assert np.array_equal(got, np.searchsorted(lam, sig, side="left"))
    # a wider bandwidth than needed gives the same pivots
    assert np.array_equal(F.inertia_counts(rp, cl, vl, sig, half_bandwidth=b + 5).cpu().numpy(), want)


def test_inertia_counts_global_window():
    """A bandwidth above what one SM's shared memory holds (3-D plane of
    14 x 13 = 182 > 167) takes the global-memory window: same counts."""
    F = _F()
    m = np.ones((5, 13, 14), dtype=np.uint8)
    h = 1.0 / 15
    _, A = O.assemble(m, h)
    rp, cl, vl = _csr_cuda(A)
    assert F.csr_half_bandwidth(rp, cl) == 182
    lam, _ = O.eig_full(A.dense())
    sig = _shifts(lam, np.random.default_rng(3))[:20]
    got = F.inertia_counts(rp, cl, vl, sig).cpu().numpy()
    assert np.array_equal(got, np.array([O.count_below(A, s) for s in sig]))


def test_inertia_counts_zero_pivot_and_edges():
    """A shift equal to the first pivot (the diagonal value 4 / h^2 makes the
    first pivot exactly zero) gives -1; a 1 x 1 matrix; no shifts; a bandwidth
    below the true one is an argument error."""
    F = _F()
    p = I.square_problem(6)
    _, A = O.assemble(p.mask, p.h)
    rp, cl, vl = _csr_cuda(A)
    diag0 = float(A.val[A.rowptr[0]:A.rowptr[1]][A.col[A.rowptr[0]:A.rowptr[1]] == 0][0])
    got = F.inertia_counts(rp, cl, vl, [diag0, 1.0]).cpu().numpy()
    assert got[0] == -1 and got[1] == 0
    one = np.ones((1, 1), dtype=np.uint8)
    _, A1 = O.assemble(one, 0.5)
    r1, c1, v1 = _csr_cuda(A1)
    assert F.inertia_counts(r1, c1, v1, [15.9, 16.1]).cpu().numpy().tolist() == [0, 1]
    assert F.inertia_counts(rp, cl, vl, []).numel() == 0
    with pytest.raises(F.FraclapError) as ei:
        F.inertia_counts(rp, cl, vl, [1.0], half_bandwidth=2)
    assert ei.value.code == -1


@pytest.mark.parametrize("dim", [2, 3])
def test_pencil_counts_match_oracle(dim):
    """Counts of the generalised problem K phi = theta M phi (bilinear /
    trilinear elements): negative pivots of K - sigma M, against the oracle."""
    F = _F()
    if dim == 2:
        p = I.ellipse_problem(30, n_ellipses=3, seed=11)
        mask, h = p.mask, p.h
    else:
        mask, h = I.square_mask(6, dim=3), 1.0 / 7
    _, K, M = O.assemble_fem(mask, h)
    th, _ = O.eig_pencil(K.dense(), M.dense())
    sig = _shifts(th, np.random.default_rng(K.n + dim))
    rp, cl, vK = _csr_cuda(K)
    vM = torch.from_numpy(M.val).cuda()
    assert np.array_equal(M.rowptr, K.rowptr) and np.array_equal(M.col, K.col)
    got = F.inertia_counts(rp, cl, vK, sig, valM=vM).cpu().numpy()
    want = np.array([O.count_below_pencil(K, M, s) for s in sig])
    assert np.array_equal(got, want)
    assert np.array_equal(got, np.searchsorted(th, sig, side="left"))


def test_sturm_counts_and_bisection_match_oracle():
    """On the tridiagonal form of a masked grid's matrix (the oracle's own
    reduction) and on a random tridiagonal: Sturm counts equal the oracle's,
    bisected eigenvalues equal the oracle's bit for bit, for the whole
    spectrum and for a slice of it."""
    F = _F()
    p = I.ellipse_problem(36, n_ellipses=5, seed=2)
    _, A = O.assemble(p.mask, p.h)
    d, e, _ = O.tridiagonalize(A.dense(), want_q=False)
    rng = np.random.default_rng(17)
    cases = [(d, e), (rng.standard_normal(300), rng.standard_normal(299)),
             (np.full(50, 2.0), np.full(49, -1.0)), (np.array([3.0]), np.zeros(0))]
    for dd, ee in cases:
        n = dd.size
        dg, eg = torch.from_numpy(dd).cuda(), torch.from_numpy(ee).cuda()
        lam_o = O.bisect(dd, ee, 0, n - 1)
        sig = np.concatenate([lam_o - 1e-9 * (1 + abs(lam_o)), lam_o + 1e-9 * (1 + abs(lam_o)),
                              rng.uniform(lam_o[0] - 1, lam_o[-1] + 1, size=10)])
        got = F.sturm_counts(dg, eg, sig).cpu().numpy()
        assert np.array_equal(got, np.array([O.sturm_count(dd, ee, s) for s in sig]))
        lam = F.bisect(dg, eg, 0, n - 1).cpu().numpy()
        assert np.array_equal(lam, lam_o)
        k0, k1 = n // 3, max(n // 3, n // 2)
        assert np.array_equal(F.bisect(dg, eg, k0, k1).cpu().numpy(), O.bisect(dd, ee, k0, k1))
    # the 1-D Laplacian: closed form 2 - 2 cos(k pi / (n + 1))
    lam = F.bisect(torch.full((50,), 2.0, dtype=torch.float64, device="cuda"),
                   torch.full((49,), -1.0, dtype=torch.float64, device="cuda"), 0, 49).cpu().numpy()
    exact = 2 - 2 * np.cos(np.arange(1, 51) * np.pi / 51)
    assert np.max(np.abs(lam - exact)) <= 4 * 2.2e-16 * 4


def test_bisection_of_the_gpu_tridiagonal_form():
    """The spectrum-slicing route on the GPU alone: the two-stage reduction
    to T, then bisection of a slice of indices: the same eigenvalues as the
    oracle's full decomposition of A (1e-11 relative)."""
    F = _F()
    p = I.ellipse_problem(48, n_ellipses=6, seed=1000)
    _, A = O.assemble(p.mask, p.h)
    lam_o, _ = O.eig_full(A.dense())
    Ad = torch.from_numpy(np.ascontiguousarray(A.dense().T)).cuda().t()
    d, e, _ = F.tridiagonalize(Ad, want_q=False)
    k0, k1 = A.n // 4, A.n // 4 + 99
    lam = F.bisect(d, e, k0, k1).cpu().numpy()
    assert np.max(np.abs(lam - lam_o[k0:k1 + 1]) / lam_o[k0:k1 + 1]) <= 1e-11


@pytest.mark.parametrize("grid,P,n_b", [("square48", 7, 0), ("ellipse64", 11, 2), ("square48", 1, 0)])
def test_partition_spectrum_matches_oracle(grid, P, n_b):
    """The greedy partitioning of Sec. III-D on GPU counts reproduces the
    oracle's partitioner on the oracle's counts exactly (split points, loads,
    history), and balances the loads.  (With rho = 8 / h^2, an even P puts
    the first split of the middle at 4 / h^2, the diagonal value, where the
    first pivot of the factorisation without pivoting is exactly zero; both
    sides then report the shift instead of a count.)"""
    F = _F()
    p = I.square_problem(48) if grid == "square48" else I.ellipse_problem(64, n_ellipses=6, seed=1000)
    _, A = O.assemble(p.mask, p.h)
    rho = 8.0 / p.h ** 2
    rp, cl, vl = _csr_cuda(A)
    s_g, l_g, h_g = F.partition_spectrum(rp, cl, vl, rho, P, n_a=7, n_b=n_b, n_c=10)
    s_o, l_o, h_o = O.greedy_partition(lambda x: O.count_below(A, x), A.n, rho, P, n_a=7, n_b=n_b, n_c=10)
    assert np.array_equal(s_g, s_o)
    assert np.array_equal(l_g, l_o)
    assert list(h_g) == list(h_o)
    assert l_g.sum() == A.n
    if P > 1:
        assert l_g.max() <= 1.3 * A.n / P


def test_partition_reports_a_zero_pivot_shift():
    """A split on the diagonal value (rho = 8 / h^2, P = 2: the split 4 / h^2)
    makes the first pivot exactly zero: the partitioner reports it as an
    error, as the oracle's count does, and the context stays usable."""
    F = _F()
    p = I.square_problem(12)
    _, A = O.assemble(p.mask, p.h)
    rp, cl, vl = _csr_cuda(A)
    with pytest.raises(F.FraclapError) as ei:
        F.partition_spectrum(rp, cl, vl, 8.0 / p.h ** 2, 2, n_a=1)
    assert ei.value.code == -2
    with pytest.raises(RuntimeError):
        O.count_below(A, 4.0 / p.h ** 2)
    s, l, _ = F.partition_spectrum(rp, cl, vl, 8.0 / p.h ** 2, 3, n_a=2)
    assert l.sum() == A.n
