"""Pins of the oracle's inertia counting on the tridiagonal form, bisection,
and the greedy spectrum partitioner (Sec. III-D-2 exact counting and Sec.
III-D "greedy partitioning")."""
import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I

EPS = 2.0 ** -52


def _laplace_1d(n):
    d, e = 2.0 * np.ones(n), -np.ones(n - 1)
    ref = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    return d, e, ref


def _random_tridiagonal(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n), rng.standard_normal(n - 1)


def test_sturm_count_closed_form_between_eigenvalues():
    d, e, ref = _laplace_1d(50)
    mids = np.concatenate([[ref[0] / 2], (ref[1:] + ref[:-1]) / 2, [ref[-1] + 1.0]])
    for k, s in enumerate(mids):
        assert O.sturm_count(d, e, s) == k


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (17, 2), (200, 3)])
def test_sturm_count_matches_the_spectrum(n, seed):
    d, e = _random_tridiagonal(n, seed)
    lam, _ = O.tridiag_eig(d, e, want_vectors=False)
    rng = np.random.default_rng(seed + 100)
    for s in rng.uniform(lam[0] - 1, lam[-1] + 1, size=40):
        if np.min(np.abs(lam - s)) < 1e-9:
            continue
        assert O.sturm_count(d, e, s) == int(np.sum(lam < s))


def test_sturm_count_is_the_inertia_of_the_dense_matrix():
    """T = Q^T A Q is congruent to A: its counts are those of the banded
    LDL^T of A - sigma I (Sylvester's law of inertia)."""
    p = I.ellipse_problem(20, seed=8)
    _, A = O.assemble(p.mask, p.h)
    d, e, _ = O.tridiagonalize(A.dense(), want_q=False)
    lam, _ = O.eig_full(A.dense())
    rng = np.random.default_rng(4)
    for s in rng.uniform(0, 8 / p.h ** 2, size=25):
        if np.min(np.abs(lam - s)) < 1e-6 * s:
            continue
        assert O.sturm_count(d, e, s) == O.count_below(A, s)


def test_bisection_closed_form_and_subsets():
    d, e, ref = _laplace_1d(64)
    lam = O.bisect(d, e, 0, 63)
    assert np.max(np.abs(lam - ref)) <= 4 * EPS * 4.0
    sub = O.bisect(d, e, 10, 20)
    np.testing.assert_array_equal(sub, lam[10:21])
    # a diagonal matrix: the sorted diagonal
    dd = np.array([3.0, -1.0, 2.5, 7.0, 0.0])
    np.testing.assert_allclose(O.bisect(dd, np.zeros(4), 0, 4), np.sort(dd), rtol=0, atol=1e-14)
    assert abs(O.bisect(np.array([1.5]), np.zeros(0), 0, 0)[0] - 1.5) <= 1e-15
    with pytest.raises(RuntimeError):
        O.bisect(d, e, 5, 64)


@pytest.mark.parametrize("n,seed", [(33, 7), (300, 8)])
def test_bisection_matches_implicit_qr(n, seed):
    d, e = _random_tridiagonal(n, seed)
    lam, _ = O.tridiag_eig(d, e, want_vectors=False)
    norm = np.abs(d).max() + 2 * np.abs(e).max()
    got = O.bisect(d, e, 0, n - 1)
    assert np.max(np.abs(got - lam)) <= 1e-13 * norm


def _square_counts(m):
    h = 1.0 / (m + 1)
    s = np.sin(np.arange(1, m + 1) * np.pi * h / 2) ** 2
    lam = np.sort((4 / h ** 2) * (s[:, None] + s[None, :]).ravel())
    return lam, (lambda x: int(np.searchsorted(lam, x, side="left"))), 8 / h ** 2


def test_greedy_partition_balances_the_square_spectrum():
    lam, cnt, rho = _square_counts(48)
    n, P = lam.size, 16
    splits, loads, hist = O.greedy_partition(cnt, n, rho, P, n_a=7)
    assert splits.shape == (P - 1,) and np.all(np.diff(splits) > 0)
    assert 0 < splits[0] and splits[-1] < rho
    assert loads.sum() == n
    np.testing.assert_array_equal(loads, np.diff(np.concatenate([[0], [cnt(x) for x in splits], [n]])))
    # equal lengths are badly loaded (the density grows with lambda); the greedy
    # refinement gets close to even
    assert hist[0] > 1.8 * n / P
    assert loads.max() == min(hist) and loads.max() <= 1.2 * n / P
    # without refinement steps the answer is the equal-length split
    s0, l0, _ = O.greedy_partition(cnt, n, rho, P, n_a=0)
    np.testing.assert_allclose(s0, rho * np.arange(1, P) / P)
    assert l0.max() == hist[0]


def test_greedy_partition_with_inertia_counts_and_local_passes():
    """The counts come from the banded LDL^T of A - sigma I, as in the paper;
    the loads agree with the spectrum, and the local passes only ever even
    out neighbouring pairs."""
    p = I.ellipse_problem(24, seed=12)
    _, A = O.assemble(p.mask, p.h)
    lam, _ = O.eig_full(A.dense())
    # P = 5: no equal-length split falls on the diagonal value 4/h^2, where the
    # unpivoted banded LDL^T meets an exact zero pivot
    n, P, rho = A.n, 5, 8 / p.h ** 2
    splits, loads, hist = O.greedy_partition(lambda x: O.count_below(A, x), n, rho, P, n_a=4, n_b=2, n_c=12)
    np.testing.assert_array_equal(loads, np.diff(np.concatenate([[0], np.searchsorted(lam, splits), [n]])))
    assert loads.sum() == n and loads.max() <= 1.3 * n / P
    assert hist[-1] <= min(hist[:5])
