"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

The arithmetic lives in ``fraclap_oracle.c``; this module compiles it with
the host C compiler on first use and marshals numpy arrays.  Matrices are
column-major (Fortran order) float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fraclap_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (IEEE double, no FMA
    contraction, OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    for extra in (["-fopenmp"], []):
        cmd = base + extra + ["-o", tmp, _SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _LIB_PATH)
            return _LIB_PATH
    raise RuntimeError("oracle build failed:\n" + r.stderr)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_number_dofs.restype = _i64
            lib.oracle_number_dofs.argtypes = [_p, _i64, _p]
            lib.oracle_assemble_csr.restype = _i64
            lib.oracle_assemble_csr.argtypes = [_p, ctypes.c_int, _p, _dbl, _p, _p, _p]
            lib.oracle_spmv.argtypes = [_i64, _p, _p, _p, _p, _p]
            lib.oracle_tridiagonalize.restype = ctypes.c_int
            lib.oracle_tridiagonalize.argtypes = [_i64, _p, _i64, _p, _p, _p, _i64]
            lib.oracle_tridiag_eig.restype = ctypes.c_int
            lib.oracle_tridiag_eig.argtypes = [_i64, _p, _p, _p, _i64, _i64, _i64]
            lib.oracle_eig_full.restype = ctypes.c_int
            lib.oracle_eig_full.argtypes = [_i64, _p, _i64, _p, _p, _i64]
            lib.oracle_eig_jacobi.restype = ctypes.c_int
            lib.oracle_eig_jacobi.argtypes = [_i64, _p, _i64, _p, _p, _i64, ctypes.c_int]
            lib.oracle_count_below.restype = _i64
            lib.oracle_count_below.argtypes = [_i64, _p, _p, _p, _dbl]
            lib.oracle_band_solve.restype = ctypes.c_int
            lib.oracle_band_solve.argtypes = [_i64, _p, _p, _p, _p, _p]
            lib.oracle_frac_apply.restype = ctypes.c_int
            lib.oracle_frac_apply.argtypes = [_i64, _p, _i64, _p, _p, _i64, _i64, _p, _p, _i64, _p, _i64]
            lib.oracle_frac_diffusion.restype = ctypes.c_int
            lib.oracle_frac_diffusion.argtypes = [_i64, _p, _i64, _p, _p, _i64, _i64, _p, _p, _p, _dbl,
                                                  _i64, _p, _i64]
            lib.oracle_assemble_fem.restype = _i64
            lib.oracle_assemble_fem.argtypes = [_p, ctypes.c_int, _p, _dbl, _p, _p, _p, _p]
            lib.oracle_eig_pencil.restype = ctypes.c_int
            lib.oracle_eig_pencil.argtypes = [_i64, _p, _i64, _p, _i64, _p, _p, _i64]
            lib.oracle_count_below_pencil.restype = _i64
            lib.oracle_count_below_pencil.argtypes = [_i64, _p, _p, _p, _p, _dbl]
            lib.oracle_frac_apply_mass.restype = ctypes.c_int
            lib.oracle_frac_apply_mass.argtypes = [_i64, _p, _i64, _p, _p, _p, _p, _p, _i64, _i64, _p, _p, _i64,
                                                   _p, _i64]
            lib.oracle_sturm_count.restype = _i64
            lib.oracle_sturm_count.argtypes = [_i64, _p, _p, _dbl]
            lib.oracle_bisect.restype = ctypes.c_int
            lib.oracle_bisect.argtypes = [_i64, _p, _p, _i64, _i64, _p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class CSR:
    """Compressed sparse rows of the assembled Laplacian (int64 rowptr, int32 col)."""

    def __init__(self, n, rowptr, col, val):
        self.n = int(n)
        self.rowptr = rowptr
        self.col = col
        self.val = val

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n), order="F")
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        A[rows, self.col] = self.val
        return A


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def assemble(mask: np.ndarray, h: float):
    """Returns (idx, CSR) of the 5-/7-point Dirichlet Laplacian on the mask
    (Sec. II eq. discrete_laplace with a nodal FD basis, M = I)."""
    lib = _load()
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    dim = mask.ndim
    ext = np.array(list(reversed(mask.shape)) + [1] * (3 - dim), dtype=np.int64)
    idx = np.empty(mask.size, np.int32)
    n = lib.oracle_number_dofs(_ptr(mask), mask.size, _ptr(idx))
    rowptr = np.empty(n + 1, np.int64)
    cap = max(1, (2 * dim + 1) * n)
    col = np.empty(cap, np.int32)
    val = np.empty(cap, np.float64)
    nnz = lib.oracle_assemble_csr(_ptr(idx), dim, _ptr(ext), float(h), _ptr(rowptr), _ptr(col), _ptr(val))
    return idx, CSR(n, rowptr, col[:nnz].copy(), val[:nnz].copy())


def spmv(A: CSR, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty(A.n)
    _load().oracle_spmv(A.n, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), _ptr(x), _ptr(y))
    return y


def tridiagonalize(A: np.ndarray, want_q: bool = True):
    """Householder reduction A = Q T Q^T; returns (d, e, Q or None)."""
    n = A.shape[0]
    W = np.array(A, dtype=np.float64, order="F", copy=True)
    d = np.empty(n)
    e = np.zeros(max(n - 1, 1))
    Q = np.empty((n, n), order="F") if want_q else None
    rc = _load().oracle_tridiagonalize(n, _ptr(W), n, _ptr(d), _ptr(e),
                                       _ptr(Q) if want_q else None, n)
    if rc != 0:
        raise RuntimeError(f"oracle_tridiagonalize failed ({rc})")
    return d, e[: max(n - 1, 0)], Q


def tridiag_eig(d: np.ndarray, e: np.ndarray, Z: np.ndarray | None = None,
                want_vectors: bool = True, max_steps: int | None = None):
    """Eigen-decomposition of the symmetric tridiagonal (d, e) by implicit QR
    steps.  If Z is given, its columns are rotated (Z <- Z * rotations), else
    Z starts as the identity.  Returns (lam ascending, Z or None)."""
    n = d.shape[0]
    dd = np.array(d, np.float64, copy=True)
    ee = np.zeros(max(n, 1))
    ee[: n - 1] = e[: n - 1]
    if want_vectors:
        ZZ = np.eye(n, order="F") if Z is None else np.array(Z, np.float64, order="F", copy=True)
        rows, ldz = ZZ.shape[0], ZZ.shape[0]
    else:
        ZZ, rows, ldz = None, 0, 1
    steps = 30 * n + 30 if max_steps is None else max_steps
    rc = _load().oracle_tridiag_eig(n, _ptr(dd), _ptr(ee), _ptr(ZZ) if want_vectors else None,
                                    ldz, rows, steps)
    if rc != 0:
        raise RuntimeError(f"oracle_tridiag_eig failed ({rc})")
    return dd, ZZ


def eig_full(A: np.ndarray):
    """Full FP64 eigendecomposition A = V diag(lam) V^T, lam ascending."""
    n = A.shape[0]
    A = np.asfortranarray(A, dtype=np.float64)
    lam = np.empty(n)
    V = np.empty((n, n), order="F")
    rc = _load().oracle_eig_full(n, _ptr(A), n, _ptr(lam), _ptr(V), n)
    if rc != 0:
        raise RuntimeError(f"oracle_eig_full failed ({rc})")
    return lam, V


def eig_jacobi(A: np.ndarray, max_sweeps: int = 100):
    n = A.shape[0]
    A = np.asfortranarray(A, dtype=np.float64)
    lam = np.empty(n)
    V = np.empty((n, n), order="F")
    rc = _load().oracle_eig_jacobi(n, _ptr(A), n, _ptr(lam), _ptr(V), n, max_sweeps)
    if rc != 0:
        raise RuntimeError(f"oracle_eig_jacobi failed ({rc})")
    return lam, V


def count_below(A: CSR, sigma: float) -> int:
    """#{lambda_i < sigma} from the inertia of A - sigma I (Sec. III-D-2)."""
    c = _load().oracle_count_below(A.n, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), float(sigma))
    if c < 0:
        raise RuntimeError(f"oracle_count_below failed ({c})")
    return int(c)


def band_solve(A: CSR, f: np.ndarray) -> np.ndarray:
    """Direct solve A u = f (the alpha = 2 case of the apply)."""
    f = np.ascontiguousarray(f, np.float64)
    u = np.empty(A.n)
    rc = _load().oracle_band_solve(A.n, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), _ptr(f), _ptr(u))
    if rc != 0:
        raise RuntimeError(f"oracle_band_solve failed ({rc})")
    return u


def frac_apply(V: np.ndarray, lam: np.ndarray, F: np.ndarray, pair_f, pair_alpha) -> np.ndarray:
    """u_j = V diag(lam^{-alpha_j/2}) V^T F[:, pair_f[j]] (Sec. II, eq. poisson_solution)."""
    V = np.asfortranarray(V, dtype=np.float64)
    n = V.shape[0]
    F = np.asfortranarray(F.reshape(n, -1), dtype=np.float64)
    m = F.shape[1]
    pf = np.ascontiguousarray(pair_f, np.int32)
    pa = np.ascontiguousarray(pair_alpha, np.float64)
    k = pf.shape[0]
    lam = np.ascontiguousarray(lam, np.float64)
    U = np.empty((n, k), order="F")
    rc = _load().oracle_frac_apply(n, _ptr(V), n, _ptr(lam), _ptr(F), n, m, _ptr(pf), _ptr(pa), k,
                                   _ptr(U), n)
    if rc != 0:
        raise RuntimeError(f"oracle_frac_apply failed ({rc})")
    return U


def frac_diffusion(V: np.ndarray, lam: np.ndarray, U0: np.ndarray, pair_f, pair_alpha, pair_t,
                   mu: float = 1.0) -> np.ndarray:
    """u_j = V diag(exp(-mu lam^{alpha_j/2} t_j)) V^T U0[:, pair_f[j]]: the
    fractional diffusion solution at time t_j (Sec. II, eq. diffusion_solution)."""
    V = np.asfortranarray(V, dtype=np.float64)
    n = V.shape[0]
    U0 = np.asfortranarray(U0.reshape(n, -1), dtype=np.float64)
    m = U0.shape[1]
    pf = np.ascontiguousarray(pair_f, np.int32)
    pa = np.ascontiguousarray(pair_alpha, np.float64)
    pt = np.ascontiguousarray(pair_t, np.float64)
    k = pf.shape[0]
    if pa.shape[0] != k or pt.shape[0] != k:
        raise ValueError("pair_f, pair_alpha and pair_t differ in length")
    lam = np.ascontiguousarray(lam, np.float64)
    U = np.empty((n, k), order="F")
    rc = _load().oracle_frac_diffusion(n, _ptr(V), n, _ptr(lam), _ptr(U0), n, m, _ptr(pf), _ptr(pa),
                                       _ptr(pt), float(mu), k, _ptr(U), n)
    if rc != 0:
        raise RuntimeError(f"oracle_frac_diffusion failed ({rc})")
    return U


def assemble_fem(mask: np.ndarray, h: float):
    """Returns (idx, K, M): the stiffness and mass matrices of bilinear (2-D) /
    trilinear (3-D) elements on the grid cells, Dirichlet zero outside the
    mask (Sec. II eq. discrete_laplace, K_ij = <grad e_i, grad e_j>,
    M_ij = <e_i, e_j>), as two CSR matrices with the same pattern."""
    lib = _load()
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    dim = mask.ndim
    ext = np.array(list(reversed(mask.shape)) + [1] * (3 - dim), dtype=np.int64)
    idx = np.empty(mask.size, np.int32)
    n = lib.oracle_number_dofs(_ptr(mask), mask.size, _ptr(idx))
    rowptr = np.empty(n + 1, np.int64)
    cap = max(1, 3 ** dim * n)
    col = np.empty(cap, np.int32)
    vk = np.empty(cap, np.float64)
    vm = np.empty(cap, np.float64)
    nnz = lib.oracle_assemble_fem(_ptr(idx), dim, _ptr(ext), float(h), _ptr(rowptr), _ptr(col), _ptr(vk), _ptr(vm))
    col = col[:nnz].copy()
    return idx, CSR(n, rowptr, col, vk[:nnz].copy()), CSR(n, rowptr.copy(), col.copy(), vm[:nnz].copy())


def eig_pencil(K: np.ndarray, M: np.ndarray):
    """K Phi = M Phi diag(theta), Phi^T M Phi = I, theta ascending (Cholesky
    reduction of the generalised problem of Sec. II eq. discrete_laplace)."""
    n = K.shape[0]
    K = np.asfortranarray(K, dtype=np.float64)
    M = np.asfortranarray(M, dtype=np.float64)
    theta = np.empty(n)
    Phi = np.empty((n, n), order="F")
    rc = _load().oracle_eig_pencil(n, _ptr(K), n, _ptr(M), n, _ptr(theta), _ptr(Phi), n)
    if rc != 0:
        raise RuntimeError(f"oracle_eig_pencil failed ({rc})")
    return theta, Phi


def count_below_pencil(K: CSR, M: CSR, sigma: float) -> int:
    """#{theta_i < sigma}: negative pivots of LDL^T(K - sigma M)."""
    if not (np.array_equal(K.rowptr, M.rowptr) and np.array_equal(K.col, M.col)):
        raise ValueError("K and M must share the CSR pattern")
    c = _load().oracle_count_below_pencil(K.n, _ptr(K.rowptr), _ptr(K.col), _ptr(K.val), _ptr(M.val),
                                          float(sigma))
    if c < 0:
        raise RuntimeError(f"oracle_count_below_pencil failed ({c})")
    return int(c)


def frac_apply_mass(Phi: np.ndarray, theta: np.ndarray, M: CSR, F: np.ndarray, pair_f, pair_alpha) -> np.ndarray:
    """u_j = Phi diag(theta^{-alpha_j/2}) Phi^T M F[:, pair_f[j]]: the apply
    of the generalised problem with the M-inner product."""
    Phi = np.asfortranarray(Phi, dtype=np.float64)
    n = Phi.shape[0]
    F = np.asfortranarray(F.reshape(n, -1), dtype=np.float64)
    m = F.shape[1]
    pf = np.ascontiguousarray(pair_f, np.int32)
    pa = np.ascontiguousarray(pair_alpha, np.float64)
    k = pf.shape[0]
    theta = np.ascontiguousarray(theta, np.float64)
    U = np.empty((n, k), order="F")
    rc = _load().oracle_frac_apply_mass(n, _ptr(Phi), n, _ptr(theta), _ptr(M.rowptr), _ptr(M.col), _ptr(M.val),
                                        _ptr(F), n, m, _ptr(pf), _ptr(pa), k, _ptr(U), n)
    if rc != 0:
        raise RuntimeError(f"oracle_frac_apply_mass failed ({rc})")
    return U


def sturm_count(d: np.ndarray, e: np.ndarray, sigma: float) -> int:
    """#{eigenvalues of the tridiagonal (d, e) below sigma}: negative pivots of
    LDL^T(T - sigma I) (Sylvester's law of inertia, Sec. III-D-2)."""
    d = np.ascontiguousarray(d, np.float64)
    ee = np.zeros(max(d.shape[0], 1))
    ee[: d.shape[0] - 1] = e[: d.shape[0] - 1]
    c = _load().oracle_sturm_count(d.shape[0], _ptr(d), _ptr(ee), float(sigma))
    if c < 0:
        raise RuntimeError(f"oracle_sturm_count failed ({c})")
    return int(c)


def bisect(d: np.ndarray, e: np.ndarray, k0: int, k1: int) -> np.ndarray:
    """Eigenvalues k0..k1 (0-based, ascending) of the tridiagonal (d, e) by
    bisection on the Sturm count."""
    d = np.ascontiguousarray(d, np.float64)
    n = d.shape[0]
    ee = np.zeros(max(n, 1))
    ee[: n - 1] = e[: n - 1]
    lam = np.empty(max(k1 - k0 + 1, 0))
    rc = _load().oracle_bisect(n, _ptr(d), _ptr(ee), int(k0), int(k1), _ptr(lam))
    if rc != 0:
        raise RuntimeError(f"oracle_bisect failed ({rc})")
    return lam


def _split_for_equal_loads(points, counts, n, P):
    """New split points for P equal loads under the piecewise-constant density
    that the counts at `points` describe: the cumulative count is linear
    between known points, and split j sits where it reaches j n / P."""
    out = []
    for j in range(1, P):
        target = j * n / P
        i = int(np.searchsorted(counts, target, side="left"))
        i = min(max(i, 1), len(points) - 1)
        c0, c1 = counts[i - 1], counts[i]
        x0, x1 = points[i - 1], points[i]
        out.append(x0 if c1 == c0 else x0 + (target - c0) / (c1 - c0) * (x1 - x0))
    return np.array(out)


def greedy_partition(count_below_fn, n: int, rho: float, P: int, n_a: int = 7, n_b: int = 0,
                     n_c: int = 10, imbalance: float = 0.25):
    """Spectrum slicing of Sec. III-D ("greedy partitioning"): split [0, rho]
    into P subintervals holding about n / P eigenvalues each.

    count_below_fn(sigma) is the exact count #{lambda < sigma} (one
    factorisation per call).  Start from P equally long subintervals; then
    n_a times: count at every split, read the counts as a piecewise-constant
    density of states, and move the splits to where that density gives equal
    loads; the best partition seen (smallest largest load) is kept.  Then up
    to n_b local passes: every pair of neighbouring subintervals whose loads
    differ by more than `imbalance` x n / P moves its shared split by a
    binary search of n_c counts towards an even pair (first the pairs
    starting at even positions, then the odd ones).
    Returns (splits, loads, history): splits has P - 1 increasing points,
    loads the P exact counts, history the largest load after each step."""
    ideal = n / P
    splits = rho * np.arange(1, P) / P

    def loads_of(s):
        c = np.array([count_below_fn(x) for x in s], dtype=np.int64)
        return c, np.diff(np.concatenate([[0], c, [n]]))

    counts, loads = loads_of(splits)
    best = (loads.max(), splits.copy(), loads.copy())
    history = [int(loads.max())]
    for _ in range(n_a):
        pts = np.concatenate([[0.0], splits, [rho]])
        cum = np.concatenate([[0], counts, [n]]).astype(np.float64)
        splits = _split_for_equal_loads(pts, cum, n, P)
        counts, loads = loads_of(splits)
        history.append(int(loads.max()))
        if loads.max() < best[0]:
            best = (loads.max(), splits.copy(), loads.copy())
    splits, loads = best[1].copy(), best[2].copy()
    for _ in range(n_b):
        changed = False
        for parity in (0, 1):
            for a in range(parity, P - 1, 2):
                if abs(int(loads[a]) - int(loads[a + 1])) <= imbalance * ideal:
                    continue
                lo = splits[a - 1] if a > 0 else 0.0
                hi = splits[a + 1] if a + 1 < P - 1 else rho
                left = 0 if a == 0 else count_below_fn(lo)
                want = left + (loads[a] + loads[a + 1]) / 2.0
                x0, x1 = lo, hi
                for _ in range(n_c):
                    mid = 0.5 * (x0 + x1)
                    if count_below_fn(mid) < want:
                        x0 = mid
                    else:
                        x1 = mid
                splits[a] = 0.5 * (x0 + x1)
                c = count_below_fn(splits[a])
                tot = loads[a] + loads[a + 1]
                loads[a], loads[a + 1] = c - left, tot - (c - left)
                changed = True
        history.append(int(loads.max()))
        if not changed:
            break
    return splits, loads, history


def solve(mask: np.ndarray, h: float, F: np.ndarray, pair_f, pair_alpha):
    """Whole path on the CPU: assemble, decompose, apply.  Returns (lam, V, U)."""
    _, A = assemble(mask, h)
    lam, V = eig_full(A.dense())
    U = frac_apply(V, lam, F, pair_f, pair_alpha)
    return lam, V, U


__all__ = ["build", "CSR", "num_threads", "assemble", "spmv", "tridiagonalize", "tridiag_eig",
           "eig_full", "eig_jacobi", "count_below", "band_solve", "frac_apply", "frac_diffusion", "assemble_fem",
           "eig_pencil", "count_below_pencil", "frac_apply_mass", "sturm_count", "bisect", "greedy_partition", "solve"]
