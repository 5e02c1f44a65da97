"""Host checks of the seeded input generators (no GPU): grid convention,
connectivity and tie-break of the kept component, hole and ellipse geometry,
dof ordering, the cubic forcings' degree, pair layout and determinism."""
import numpy as np
import pytest

from paper_1911_11906_gb300 import inputs as I

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def _components(mask, conn):
    lab, n = scipy_ndimage.label(mask, structure=scipy_ndimage.generate_binary_structure(mask.ndim, conn))
    return lab, n


def test_grid_convention():
    h, x = I.grid_coords(48, 2)
    assert h == 1 / 49 and np.allclose(x, (np.arange(48) + 1) / 49)
    s = I.square_problem(12, n_poly=0)
    assert s.n == 144 and s.ext == (12, 12, 1)


@pytest.mark.parametrize("m,seed", [(128, 1000), (48, 7), (20, 3000)])
def test_ellipse_mask_is_one_face_connected_component_inside_the_ellipses(m, seed):
    mask = I.ellipse_mask(m, 6, np.random.default_rng(seed))
    assert mask.dtype == np.uint8 and mask.any()
    assert _components(mask, 1)[1] == 1
    # inside the union of the six ellipses, drawn in the stated order
    rng = np.random.default_rng(seed)
    _, x = I.grid_coords(m, 2)
    X, Y = np.meshgrid(x, x, indexing="xy")
    union = np.zeros((m, m), bool)
    for _ in range(6):
        cx, cy = rng.uniform(0.2, 0.8, size=2)
        a, b = rng.uniform(0.1, 0.3, size=2)
        assert 0.2 <= cx <= 0.8 and 0.1 <= a <= 0.3
        union |= ((X - cx) / a) ** 2 + ((Y - cy) / b) ** 2 <= 1.0
    assert np.all(union[mask.astype(bool)])
    # and it is the largest face-connected component of that union
    lab, n = _components(union, 1)
    sizes = np.bincount(lab.ravel())[1:]
    assert mask.sum() == sizes.max()


def test_holed_cube_mask():
    m = 32
    mask = I.holed_cube_mask(m, 5, np.random.default_rng(2000))
    assert _components(mask, 1)[1] == 1
    rng = np.random.default_rng(2000)
    _, x = I.grid_coords(m, 3)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    for _ in range(5):
        cx, cy, cz = rng.uniform(0.2, 0.8, size=3)
        r = rng.uniform(0.05, 0.15)
        inside = (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2 <= r * r
        assert inside.any() and not np.any(mask[inside])
    assert int(mask.sum()) == 31996


def test_largest_component_ties_and_fallback(monkeypatch):
    # two components of 3 nodes each: the one holding the lowest row-major index wins
    keep = np.zeros((4, 6), bool)
    keep[0, 3:6] = True
    keep[2, 0:3] = True
    got = I._largest_component(keep)
    assert got[0, 3:6].all() and not got[2].any()
    # diagonal contact does not connect (4-connectivity)
    diag = np.zeros((3, 3), bool)
    diag[0, 0] = diag[1, 1] = diag[2, 2] = True
    assert I._largest_component(diag).sum() == 1
    # the plain flood fill gives scipy's answer
    rng = np.random.default_rng(5)
    cases = [rng.random((17, 23)) < 0.55 for _ in range(4)] + [rng.random((7, 8, 9)) < 0.6 for _ in range(3)]
    want = [I._largest_component(c) for c in cases]
    monkeypatch.setattr(I, "_ndimage", None)
    for c, w in zip(cases, want):
        assert np.array_equal(I._largest_component(c), w)
    assert I._largest_component(np.zeros((3, 3), bool)).sum() == 0


def test_dof_order_and_coordinates():
    mask = np.array([[1, 0, 1], [1, 1, 0]], np.uint8)  # [y, x]
    h = 0.25
    c = I.dof_coords(mask, h)
    # row-major over kept nodes, x fastest: (x, y) = (0,0), (2,0), (0,1), (1,1)
    assert np.allclose(c, np.array([[1, 1], [3, 1], [1, 2], [2, 2]]) * h)
    m3 = np.zeros((2, 2, 2), np.uint8)
    m3[1, 0, 1] = m3[0, 1, 0] = 1
    assert np.allclose(I.dof_coords(m3, 0.5), np.array([[1, 2, 1], [2, 1, 2]]) * 0.5)


@pytest.mark.parametrize("dim,terms", [(2, 10), (3, 20)])
def test_polynomial_forcings_are_full_cubics(dim, terms):
    rng = np.random.default_rng(11)
    coords = rng.random((200, dim))
    f = I.poly_forcing(coords, np.random.default_rng(3))

    def basis(maxdeg):
        cols = []
        for deg in range(maxdeg + 1):
            for e in np.ndindex(*(deg + 1,) * dim):
                if sum(e) == deg:
                    cols.append(np.prod(coords ** np.array(e), axis=1))
        return np.stack(cols, axis=1)

    B3, B2 = basis(3), basis(2)
    assert B3.shape[1] == terms
    res3 = np.linalg.lstsq(B3, f, rcond=None)[1]
    res2 = np.linalg.lstsq(B2, f, rcond=None)[1]
    assert res3.size and res3[0] <= 1e-20 * (f @ f)
    assert res2[0] > 1e-6 * (f @ f)


def test_sine_forcing_and_pairs():
    p = I.square_problem(8, n_poly=2, alphas=(0.5, 2.0))
    x, y = p.coords[:, 0], p.coords[:, 1]
    assert np.allclose(p.F[:, 0], np.sin(np.pi * x) * np.sin(np.pi * y))
    assert p.pair_f.tolist() == [0, 0, 1, 1, 2, 2]
    assert p.pair_alpha.tolist() == [0.5, 2.0] * 3
    assert p.F.flags.f_contiguous


def test_workload_pairs_and_determinism():
    e = I.ellipse_problem()
    assert sorted(set(e.pair_alpha.tolist())) == [i / 4 for i in range(1, 9)]
    c = I.holed_cube_problem(m=12, n_forcings=3)
    assert sorted(set(c.pair_alpha.tolist())) == [0.25, 0.75, 1.25, 1.75]
    a = I.apply_at_scale_problem(m=24, k=16)
    assert np.all((a.pair_alpha >= 0.1) & (a.pair_alpha <= 1.9)) and a.pair_f.tolist() == list(range(16))
    b1, b2 = I.batched_problems(5), I.batched_problems(5)
    for p, q in zip(b1, b2):
        assert np.array_equal(p.mask, q.mask) and np.array_equal(p.F, q.F)
        assert 20 <= p.mask.shape[0] <= 64
    assert len({p.mask.shape[0] for p in I.batched_problems(40)}) > 5
