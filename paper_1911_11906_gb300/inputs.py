"""Seeded synthetic inputs for the fractional Poisson workloads.

This module holds no arithmetic of the method itself: it draws domains
(masks), forcings and fractional orders, and nothing else.  The same arrays
feed both the CUDA path and the CPU oracle, so no cross-language random
number parity is needed.

Domain conventions (the discrete counterpart of the Dirichlet problem of
Sec. II, eq. (model_poisson)):

* A 2-D grid has ``m x m`` interior nodes at ``x_i = (i+1) h``, ``h = 1/(m+1)``;
  3-D grids likewise with ``m^3`` nodes.
* ``mask`` is ``uint8``, C-ordered ``[y, x]`` (2-D) or ``[z, y, x]`` (3-D), so
  ``x`` is the fastest index; 1 = the node is a degree of freedom.
* Degrees of freedom are numbered in row-major order over kept nodes.
* Irregular domains keep the largest 4-connected (2-D) or 6-connected (3-D)
  component, so the stencil matrix is irreducible; ties go to the component
  that contains the lowest row-major index.

Random draws use ``numpy.random.default_rng(seed)`` (PCG64); each workload
uses seed ``1000 * workload + item``.
"""
from __future__ import annotations

import dataclasses

import numpy as np

try:  # scipy is present on both machines; keep a plain fallback anyway
    from scipy import ndimage as _ndimage
except Exception:  # pragma: no cover
    _ndimage = None


@dataclasses.dataclass
class Problem:
    """One domain plus its forcings and (forcing, alpha) pairs."""

    name: str
    mask: np.ndarray          # uint8, [y, x] or [z, y, x]
    h: float                  # grid spacing
    F: np.ndarray             # (n, m) float64, column-major friendly (Fortran order)
    pair_f: np.ndarray        # (k,) int32, column of F used by pair j
    pair_alpha: np.ndarray    # (k,) float64, fractional order of pair j
    coords: np.ndarray        # (n, dim) float64, coordinates of the dofs

    @property
    def dim(self) -> int:
        return self.mask.ndim

    @property
    def ext(self) -> tuple:
        """Grid extents (nx, ny, nz) with nz = 1 in 2-D."""
        if self.mask.ndim == 2:
            return (self.mask.shape[1], self.mask.shape[0], 1)
        return (self.mask.shape[2], self.mask.shape[1], self.mask.shape[0])

    @property
    def n(self) -> int:
        return int(self.mask.sum())


def _largest_component(keep: np.ndarray) -> np.ndarray:
    """Largest face-connected component of a boolean grid (ties: lowest index)."""
    if not keep.any():
        return keep.astype(np.uint8)
    if _ndimage is not None:
        structure = _ndimage.generate_binary_structure(keep.ndim, 1)
        labels, nlab = _ndimage.label(keep, structure=structure)
    else:  # plain flood fill, raster order
        labels = np.zeros(keep.shape, np.int64)
        nlab = 0
        flat = keep.reshape(-1)
        lab = labels.reshape(-1)
        shape = keep.shape
        strides = [int(np.prod(shape[i + 1:])) for i in range(len(shape))]
        for start in range(flat.size):
            if not flat[start] or lab[start]:
                continue
            nlab += 1
            stack = [start]
            lab[start] = nlab
            while stack:
                p = stack.pop()
                coord = np.unravel_index(p, shape)
                for ax in range(len(shape)):
                    for dlt in (-1, 1):
                        c = coord[ax] + dlt
                        if 0 <= c < shape[ax]:
                            q = p + dlt * strides[ax]
                            if flat[q] and not lab[q]:
                                lab[q] = nlab
                                stack.append(q)
    sizes = np.bincount(labels.reshape(-1), minlength=nlab + 1)
    sizes[0] = 0
    best = int(np.argmax(sizes))  # labels are numbered in raster order: ties -> lowest index
    return (labels == best).astype(np.uint8)


def grid_coords(m: int, dim: int) -> tuple:
    h = 1.0 / (m + 1)
    x = (np.arange(m) + 1) * h
    return h, x


def square_mask(m: int, dim: int = 2) -> np.ndarray:
    return np.ones((m,) * dim, np.uint8)


def ellipse_mask(m: int, n_ellipses: int, rng: np.random.Generator) -> np.ndarray:
    """Union of axis-aligned ellipses (centres U(0.2,0.8), semi-axes U(0.1,0.3)),
    largest 4-connected component.  Draw order per ellipse: cx, cy, a, b."""
    _, x = grid_coords(m, 2)
    X, Y = np.meshgrid(x, x, indexing="xy")  # X[y, x] = x coordinate
    keep = np.zeros((m, m), bool)
    for _ in range(n_ellipses):
        cx, cy = rng.uniform(0.2, 0.8, size=2)
        a, b = rng.uniform(0.1, 0.3, size=2)
        keep |= ((X - cx) / a) ** 2 + ((Y - cy) / b) ** 2 <= 1.0
    return _largest_component(keep)


def holed_cube_mask(m: int, n_holes: int, rng: np.random.Generator) -> np.ndarray:
    """Cube minus spherical holes (centres U(0.2,0.8)^3, radius U(0.05,0.15)),
    largest 6-connected component.  Draw order per hole: cx, cy, cz, r."""
    _, x = grid_coords(m, 3)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    keep = np.ones((m, m, m), bool)
    for _ in range(n_holes):
        cx, cy, cz = rng.uniform(0.2, 0.8, size=3)
        r = rng.uniform(0.05, 0.15)
        keep &= (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2 > r * r
    return _largest_component(keep)


def dof_coords(mask: np.ndarray, h: float) -> np.ndarray:
    """Coordinates (x, y[, z]) of every dof, in dof order (row-major, x fastest)."""
    idx = np.nonzero(mask.reshape(-1))[0]
    unr = np.unravel_index(idx, mask.shape)        # (y, x) or (z, y, x)
    cols = [(np.asarray(u, np.float64) + 1.0) * h for u in reversed(unr)]
    return np.stack(cols, axis=1)


def poly_forcing(coords: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Cubic polynomial with N(0,1) coefficients in graded-lex monomial order
    (10 terms in 2-D, 20 in 3-D), evaluated at the dofs."""
    dim = coords.shape[1]
    exps = []
    for deg in range(4):
        if dim == 2:
            for a in range(deg, -1, -1):
                exps.append((a, deg - a))
        else:
            for a in range(deg, -1, -1):
                for b in range(deg - a, -1, -1):
                    exps.append((a, b, deg - a - b))
    c = rng.standard_normal(len(exps))
    f = np.zeros(coords.shape[0])
    for ck, e in zip(c, exps):
        term = np.full(coords.shape[0], ck)
        for d in range(dim):
            term = term * coords[:, d] ** e[d]
        f += term
    return f


def sine_forcing(coords: np.ndarray) -> np.ndarray:
    """f = prod_d sin(pi x_d): the lowest Dirichlet mode of the square/cube."""
    f = np.ones(coords.shape[0])
    for d in range(coords.shape[1]):
        f = f * np.sin(np.pi * coords[:, d])
    return f


def _pairs_all(m_f: int, alphas) -> tuple:
    pf = np.repeat(np.arange(m_f, dtype=np.int32), len(alphas))
    pa = np.tile(np.asarray(alphas, np.float64), m_f)
    return pf, pa


def square_problem(m: int = 48, n_poly: int = 4, alphas=(0.5, 1.0, 1.5, 2.0),
                   seed: int = 0) -> Problem:
    """Unit square, m x m interior grid: f0 = sin(pi x) sin(pi y) plus seeded
    cubic-polynomial forcings, all crossed with every alpha."""
    h, _ = grid_coords(m, 2)
    mask = square_mask(m)
    coords = dof_coords(mask, h)
    cols = [sine_forcing(coords)]
    for i in range(n_poly):
        cols.append(poly_forcing(coords, np.random.default_rng(seed + i)))
    F = np.asfortranarray(np.stack(cols, axis=1))
    pf, pa = _pairs_all(F.shape[1], alphas)
    return Problem(f"square{m}", mask, h, F, pf, pa, coords)


def ellipse_problem(m: int = 128, n_ellipses: int = 6, n_forcings: int = 16,
                    alphas=None, seed: int = 1000, name: str | None = None) -> Problem:
    """Masked 2-D grid (union of random ellipses), polynomial forcings."""
    if alphas is None:
        alphas = [i / 4.0 for i in range(1, 9)]     # 8 values evenly spaced in (0, 2]
    h, _ = grid_coords(m, 2)
    mask = ellipse_mask(m, n_ellipses, np.random.default_rng(seed))
    coords = dof_coords(mask, h)
    cols = [poly_forcing(coords, np.random.default_rng(seed + 1 + i)) for i in range(n_forcings)]
    F = np.asfortranarray(np.stack(cols, axis=1))
    pf, pa = _pairs_all(F.shape[1], alphas)
    return Problem(name or f"ellipse{m}", mask, h, F, pf, pa, coords)


def holed_cube_problem(m: int = 32, n_holes: int = 5, n_forcings: int = 64,
                       alphas=(0.25, 0.75, 1.25, 1.75), seed: int = 2000) -> Problem:
    h, _ = grid_coords(m, 3)
    mask = holed_cube_mask(m, n_holes, np.random.default_rng(seed))
    coords = dof_coords(mask, h)
    cols = [poly_forcing(coords, np.random.default_rng(seed + 1 + i)) for i in range(n_forcings)]
    F = np.asfortranarray(np.stack(cols, axis=1))
    pf, pa = _pairs_all(F.shape[1], alphas)
    return Problem(f"holedcube{m}", mask, h, F, pf, pa, coords)


def batched_problems(count: int = 256, n_forcings: int = 8,
                     alphas=(0.5, 1.0, 1.5, 2.0), seed: int = 3000) -> list:
    """Many masked 2-D grids, side U{20..64}, each with its own ellipse mask."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        side = int(rng.integers(20, 65))
        out.append(ellipse_problem(side, 6, n_forcings, alphas, seed=seed * 10 + 7 * i,
                                   name=f"batch{i}_side{side}"))
    return out


def apply_at_scale_problem(m: int = 192, k: int = 4096, seed: int = 4000) -> Problem:
    """Masked 2-D grid with k distinct forcings (half polynomial, half N(0,1)
    grid values) and one alpha ~ U(0.1, 1.9) per forcing."""
    h, _ = grid_coords(m, 2)
    mask = ellipse_mask(m, 6, np.random.default_rng(seed))
    coords = dof_coords(mask, h)
    n = coords.shape[0]
    rng = np.random.default_rng(seed + 1)
    F = np.empty((n, k), order="F")
    for j in range(k):
        if j % 2 == 0:
            F[:, j] = poly_forcing(coords, rng)
        else:
            F[:, j] = rng.standard_normal(n)
    pf = np.arange(k, dtype=np.int32)
    pa = rng.uniform(0.1, 1.9, size=k)
    return Problem(f"apply{m}", mask, h, F, pf, pa, coords)


def workload(i: int) -> Problem:
    """The five benchmark workloads (the batched one returns its first grid)."""
    if i == 0:
        return square_problem()
    if i == 1:
        return ellipse_problem()
    if i == 2:
        return holed_cube_problem()
    if i == 3:
        return batched_problems(1)[0]
    if i == 4:
        return apply_at_scale_problem()
    raise ValueError(i)
