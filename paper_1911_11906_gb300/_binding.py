"""ctypes marshalling for libfraclap.so (see include/fraclap.h)."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libfraclap.so")
_lock = threading.Lock()
_lib = None

_i32, _i64, _dbl, _p, _sz = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t

# (name, restype, argtypes) of every exported entry point
SIGNATURES = {
    "fraclap_create": (_i32, [ctypes.POINTER(_p), _p]),
    "fraclap_destroy": (None, [_p]),
    "fraclap_strerror": (ctypes.c_char_p, [_i32]),
    "fraclap_last_error": (ctypes.c_char_p, [_p]),
    "fraclap_sync": (_i32, [_p, _p]),
    "fd_assemble": (_i32, [_p, _p, _i32, _p, _dbl, _p, _p, _p, _p, _p, _p, _p, _i64, _p]),
    "fraclap_eig_workspace_bytes": (_sz, [_p, _i64]),
    "eig_full": (_i32, [_p, _p, _i64, _i64, _p, _p, _i64, _p, _sz, _p, _p]),
    "fraclap_eig_mixed_workspace_bytes": (_sz, [_p, _i64]),
    "eig_full_mixed": (_i32, [_p, _p, _i64, _i64, _p, _p, _p, _i32, _p, _p, _i64, _p, _sz, _p, _p]),
    "fraclap_apply_workspace_bytes": (_sz, [_i64, _i64, _i64]),
    "frac_apply": (_i32, [_p, _p, _i64, _p, _i64, _p, _i64, _i64, _p, _p, _i64, _p, _i64, _p, _sz, _p]),
    "frac_diffusion": (_i32, [_p, _p, _i64, _p, _i64, _p, _i64, _i64, _p, _p, _p, _dbl, _i64, _p, _i64, _p, _sz,
                              _p]),
    "frac_apply_noalloc": (_i32, [_p, _i64, _p, _i64, _p, _i64, _i64, _p, _p, _i64, _p, _i64, _p, _p]),
    "fraclap_tridiagonalize": (_i32, [_p, _p, _i64, _i64, _p, _p, _p, _i64, _p, _sz, _p]),
    "fraclap_tridiag_workspace_bytes": (_sz, [_p, _i64]),
    "fraclap_tridiag_eig": (_i32, [_p, _p, _p, _i64, _p, _p, _i64, _p, _sz, _p]),
    "fraclap_set_profiling": (_i32, [_p, _i32]),
    "fraclap_stage_times": (_i32, [_p, _p, _p, _i32]),
    "fraclap_launch_count": (ctypes.c_longlong, [_p]),
    "fraclap_refine_stats": (_i32, [_p, _p, _i32]),
    "fraclap_set_tensor_route": (_i32, [_p, _i32]),
    "fraclap_set_refine_tau": (_i32, [_p, _dbl]),
    "fraclap_wait_selftest": (_i32, [_p, _i32, _p]),
    "fraclap_apply_graph_create": (_i32, [_p, _p, _i64, _p, _i64, _p, _i64, _i64, _p, _p, _p, _dbl, _i64, _p, _i64,
                                          _p, _sz, _p]),
    "fraclap_graph_launch": (_i32, [_p, _p]),
    "fraclap_graph_kernels": (ctypes.c_longlong, [_p]),
    "fraclap_graph_destroy": (None, [_p]),
    "fraclap_mask_hash": (ctypes.c_uint64, [_p, _i32, _p, _dbl]),
    "fraclap_save_decomposition": (_i32, [ctypes.c_char_p, _i64, _p, _p, _i64, _i32, _p, _dbl, ctypes.c_uint64]),
    "fraclap_load_decomposition": (_i32, [ctypes.c_char_p, _p, _p, _p, _p, _p, _p, _p, _i64, ctypes.c_uint64]),
    "fraclap_dgemm_ozaki_workspace_bytes": (_sz, [_i64, _i64, _i64, _i32]),
    "fraclap_dgemm_ozaki": (_i32, [_p, _i32, _i32, _i64, _i64, _i64, _dbl, _p, _i64, _p, _i64, _dbl, _p, _i64,
                                   _i32, _p, _sz, _p]),
    "fraclap_dgemm": (_i32, [_p, _i32, _i32, _i64, _i64, _i64, _dbl, _p, _i64, _p, _i64, _dbl, _p, _i64, _p]),
    "fraclap_sgemm_workspace_bytes": (ctypes.c_size_t, [_i64, _i64, _i64]),
    "fraclap_solve_batched": (_i32, [_p, _p, _i32, _i32, _p]),
    "fraclap_apply_workspace_bytes_ctx": (ctypes.c_size_t, [_p, _i64, _i64, _i64]),
    "fraclap_set_apply_slices": (_i32, [_p, _i32]),
    "fem_assemble": (_i32, [_p, _p, _i32, _p, _dbl, _p, _p, _p, _p, _p, _p, _p, _p, _p, _i64, _p]),
    "fraclap_eig_pencil_workspace_bytes": (_sz, [_p, _i64, _i64]),
    "eig_pencil": (_i32, [_p, _p, _i64, _i64, _p, _p, _p, _i64, _p, _p, _i64, _p, _sz, _p]),
    "fraclap_apply_mass_workspace_bytes": (_sz, [_p, _i64, _i64, _i64]),
    "frac_apply_mass": (_i32, [_p, _p, _i64, _p, _i64, _p, _p, _p, _p, _i64, _i64, _p, _p, _i64, _p, _i64, _p, _sz,
                               _p]),
    "fraclap_csr_half_bandwidth": (_i32, [_p, _i64, _p, _p, _p, _p]),
    "fraclap_inertia_workspace_bytes": (_sz, [_i64, _i64, _i64, _i32]),
    "fraclap_inertia_counts": (_i32, [_p, _i64, _p, _p, _p, _p, _i64, _p, _i64, _p, _p, _sz, _p]),
    "fraclap_sturm_counts": (_i32, [_p, _p, _p, _i64, _p, _i64, _p, _p]),
    "fraclap_bisect": (_i32, [_p, _p, _p, _i64, _i64, _i64, _p, _p]),
    "fraclap_partition_spectrum": (_i32, [_p, _i64, _p, _p, _p, _p, _i64, _dbl, _i32, _i32, _i32, _i32, _dbl, _p,
                                          _p, _p, _i32, _p, _sz, _p]),
    "fraclap_fma_throughput": (_i32, [_p, _i32, _i64, _p, _p]),
    "fraclap_set_schedule": (_i32, [_p, _i32, _i32]),
    "fraclap_get_schedule": (_i32, [_p, _i32]),
    "fraclap_sgemm": (_i32, [_p, _i32, _i32, _i32, _i64, _i64, _i64, ctypes.c_float, _p, _i64, _p, _i64,
                             ctypes.c_float, _p, _i64, _i32, _p, ctypes.c_size_t, _p]),
}


class FraclapError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fraclap error {code}: {msg}")
        self.code = code


class _Opts(ctypes.Structure):
    _fields_ = [("band_width", ctypes.c_int), ("leaf_size", ctypes.c_int), ("wait_timeout_s", ctypes.c_double)]


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Loads the in-tree CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(
                    f"CUDA library {_LIB_PATH} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
            lib = ctypes.CDLL(_LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Context:
    """A library context on the current CUDA device (owns a status word and
    an optional workspace)."""

    def __init__(self, band_width: int = 0, leaf_size: int = 0, wait_timeout_s: float = 0.0):
        self.lib = load_library()
        self.handle = ctypes.c_void_p()
        opts = _Opts(band_width, leaf_size, wait_timeout_s)
        rc = self.lib.fraclap_create(ctypes.byref(self.handle), ctypes.byref(opts))
        if rc != 0:
            raise FraclapError(rc, self.lib.fraclap_strerror(rc).decode())

    def close(self):
        if self.handle:
            self.lib.fraclap_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc: int):
        if rc != 0:
            msg = self.lib.fraclap_last_error(self.handle).decode()
            raise FraclapError(rc, msg)

    STAGES = ("assemble", "band_reduction", "bulge_chasing", "tridiag_dc", "back_q2", "back_q1", "apply",
              "refine", "residual_gemm", "refine_norms", "refine_update", "refine_sort", "refine_clusters",
              "refine_big_clusters", "slice_products")

    def set_profiling(self, enable: bool = True):
        self.check(self.lib.fraclap_set_profiling(self.handle, int(enable)))

    def stage_times(self) -> dict:
        """{stage: (milliseconds, records)} summed since the last call."""
        n = len(self.STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        self.check(self.lib.fraclap_stage_times(self.handle, ms, cnt, n))
        return {s: (ms[i], cnt[i]) for i, s in enumerate(self.STAGES)}

    REFINE_FIELDS = ("delta", "norm2_S_minus_D", "norm2_R", "fro_S_minus_D", "fro_R", "norm2_A_bound",
                     "clusters", "largest_cluster")

    def refine_stats(self) -> list:
        """Per iteration of the last mixed-precision refinement: dict of REFINE_FIELDS."""
        buf = (ctypes.c_double * 512)()
        nv = self.lib.fraclap_refine_stats(self.handle, buf, 512)
        f = self.REFINE_FIELDS
        return [dict(zip(f, buf[i:i + len(f)])) for i in range(0, min(nv, 512), len(f))]

    def set_refine_tau(self, tau: float):
        """Refinement safeguard: pairs with a first-order coefficient above tau are clustered."""
        self.check(self.lib.fraclap_set_refine_tau(self.handle, float(tau)))

    def set_apply_slices(self, slices: int):
        """frac_apply products: 0 = FP64 engine; s = 1..8 BF16 slices on the tensor cores."""
        self.check(self.lib.fraclap_set_apply_slices(self.handle, int(slices)))

    SCHEDULE_KNOBS = {"ozaki_group": 0, "ozaki_bits": 1, "fp32_stages_tc": 2, "ozaki_tile_n": 3, "q2_parts": 4,
                      "ozaki_cluster": 5}

    def set_schedule(self, knob: str, value: int):
        """Sets a schedule knob of the context (see SCHEDULE_KNOBS)."""
        self.check(self.lib.fraclap_set_schedule(self.handle, self.SCHEDULE_KNOBS[knob], int(value)))

    def get_schedule(self, knob: str) -> int:
        return int(self.lib.fraclap_get_schedule(self.handle, self.SCHEDULE_KNOBS[knob]))

    def set_tensor_route(self, route: int):
        """1: tcgen05 + TMA slice products (default); 0: mma.sync."""
        self.check(self.lib.fraclap_set_tensor_route(self.handle, int(route)))

    def wait_selftest(self, which: int, stream=None):
        """Drives one bounded device wait (0: grid barrier, 1: mbarrier) into
        its time limit; the next sync raises FraclapError(-4)."""
        self.check(self.lib.fraclap_wait_selftest(self.handle, int(which), ctypes.c_void_p(_stream(stream))))

    def fma_throughput(self, precision: int, iters: int | None = None, stream=None) -> float:
        """Measured FMA-pipe throughput in flop/s (precision 64 or 32)."""
        if iters is None:
            iters = (1 << 14) if precision == 64 else (1 << 18)
        out = ctypes.c_double(0.0)
        self.check(self.lib.fraclap_fma_throughput(self.handle, int(precision), int(iters), ctypes.byref(out),
                                                   ctypes.c_void_p(_stream(stream))))
        return float(out.value)

    def launch_count(self) -> int:
        return int(self.lib.fraclap_launch_count(self.handle))

    def sync(self, stream=None):
        """Waits for the stream and raises if a kernel recorded a failure."""
        self.check(self.lib.fraclap_sync(self.handle, ctypes.c_void_p(_stream(stream))))


_default = None


def default_context() -> Context:
    global _default
    if _default is None:
        _default = Context()
    return _default


def colmajor_layout_ok(shape, strides) -> bool:
    """True when a 2-D (rows, cols) layout can be handed to the library as a
    column-major matrix with leading dimension strides[1]: unit row stride
    and columns that do not overlap (strides[1] >= rows whenever there is
    more than one column).  An expanded or otherwise overlapping view fails:
    the library would read or write rows * cols elements through it."""
    rows, cols = shape
    if rows > 1 and cols > 0 and strides[0] != 1:
        return False
    if cols > 1 and strides[1] < max(rows, 1):
        return False
    return True


def _f64_colmajor(t: torch.Tensor, name: str, rows: int | None = None, cols: int | None = None,
                  device=None) -> torch.Tensor:
    """Returns a column-major (Fortran-order) float64 CUDA view: ld = t.stride(1).
    A view whose layout the library cannot walk (transposed, expanded) is
    copied into a column-major one; rows/cols, when given, must match, and
    device, when given, must be the tensor's device."""
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if device is not None and t.device != device:
        raise TypeError(f"{name} must be on {device}, not {t.device}")
    if t.dim() == 1:
        t = t.unsqueeze(1)
    if t.dim() != 2:
        raise ValueError(f"{name} must be a matrix")
    if (rows is not None and t.shape[0] != rows) or (cols is not None and t.shape[1] != cols):
        raise ValueError(f"{name} must have shape ({rows if rows is not None else '*'}, "
                         f"{cols if cols is not None else '*'}), not {tuple(t.shape)}")
    if not colmajor_layout_ok(tuple(t.shape), t.stride()):
        t = t.t().contiguous().t()
    return t


def _square(t: torch.Tensor, name: str) -> torch.Tensor:
    """A float64 CUDA matrix that must be square (n x n), column-major."""
    t = _f64_colmajor(t, name)
    if t.shape[0] != t.shape[1]:
        raise ValueError(f"{name} must be square, not {tuple(t.shape)}")
    return t


def _dev(t, dtype, name: str, device, numel: int | None = None) -> torch.Tensor:
    """A contiguous CUDA tensor of `dtype` on `device` (and `numel` long when
    given); anything else is refused, so that no host pointer and no short
    buffer ever reaches a kernel."""
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or t.device != device:
        raise TypeError(f"{name} must be a {dtype} CUDA tensor on {device}")
    t = t.contiguous()
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must hold {numel} elements, not {t.numel()}")
    return t


def _out(t: torch.Tensor, dtype, name: str, device, rows: int, cols: int) -> torch.Tensor:
    """A caller-provided output, written in place: column-major, `dtype`, on
    `device`, of shape (rows, cols)."""
    if (not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or t.device != device
            or tuple(t.shape) != (rows, cols) or not colmajor_layout_ok((rows, cols), t.stride())):
        raise TypeError(f"{name} must be a column-major {dtype} CUDA tensor of shape ({rows}, {cols}) on {device}"
                        " with non-overlapping columns")
    return t


def _ws(t: torch.Tensor, device) -> torch.Tensor:
    """A caller-provided device workspace (uint8, contiguous, on `device`)."""
    if not isinstance(t, torch.Tensor) or t.dtype != torch.uint8 or not t.is_cuda or t.device != device \
            or not t.is_contiguous():
        raise TypeError(f"workspace must be a contiguous uint8 CUDA tensor on {device}")
    return t


def _ld(t: torch.Tensor) -> int:
    return max(t.stride(1), t.shape[0], 1) if t.dim() == 2 else max(t.shape[0], 1)


def empty_colmajor(rows: int, cols: int, device=None) -> torch.Tensor:
    return torch.empty((cols, rows), dtype=torch.float64, device=device or "cuda").t()


def fd_assemble(mask: torch.Tensor, h: float, dense: bool = True, ctx: Context | None = None,
                stream=None):
    """Assembles the FD Laplacian of a uint8 mask ([y, x] or [z, y, x]) on the GPU.
    Returns dict(idx, n, rowptr, col, val, A (column-major dense or None))."""
    ctx = ctx or default_context()
    if mask.dtype != torch.uint8 or not mask.is_cuda:
        raise TypeError("mask must be a uint8 CUDA tensor")
    mask = mask.contiguous()
    dim = mask.dim()
    ext = (ctypes.c_int64 * 3)(*(list(reversed(mask.shape)) + [1] * (3 - dim)))
    idx = torch.empty(mask.shape, dtype=torch.int32, device=mask.device)
    n = ctypes.c_int64(-1)
    nnz = ctypes.c_int64(-1)
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.fd_assemble(ctx.handle, _ptr(mask), dim, ext, float(h), _ptr(idx), ctypes.byref(n),
                                  ctypes.byref(nnz), None, None, None, None, 0, st))
    N, NNZ = n.value, nnz.value
    rowptr = torch.empty(N + 1, dtype=torch.int64, device=mask.device)
    col = torch.empty(max(NNZ, 1), dtype=torch.int32, device=mask.device)
    val = torch.empty(max(NNZ, 1), dtype=torch.float64, device=mask.device)
    A = empty_colmajor(N, N, mask.device) if (dense and N > 0) else None
    ctx.check(ctx.lib.fd_assemble(ctx.handle, _ptr(mask), dim, ext, float(h), _ptr(idx), ctypes.byref(n),
                                  ctypes.byref(nnz), _ptr(rowptr), _ptr(col), _ptr(val), _ptr(A),
                                  max(N, 1), st))
    return {"idx": idx, "n": N, "rowptr": rowptr, "col": col[:NNZ], "val": val[:NNZ], "A": A}


def eig_full(A: torch.Tensor, ctx: Context | None = None, stream=None, workspace: torch.Tensor | None = None,
             sync: bool = True):
    """All eigenpairs of the symmetric matrix A (lower triangle read).
    Returns (lambda ascending, V column-major)."""
    ctx = ctx or default_context()
    A = _square(A, "A")
    n = A.shape[0]
    lam = torch.empty(n, dtype=torch.float64, device=A.device)
    V = empty_colmajor(n, n, A.device)
    if workspace is None:
        nbytes = ctx.lib.fraclap_eig_workspace_bytes(ctx.handle, n)
        workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=A.device)
    else:
        workspace = _ws(workspace, A.device)
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.eig_full(ctx.handle, _ptr(A), n, _ld(A), _ptr(lam), _ptr(V), max(n, 1),
                               _ptr(workspace), workspace.numel(), None, st))
    if sync:
        ctx.sync(stream)
    return lam, V


def eig_full_mixed(A: torch.Tensor, rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor,
                   refine_iters: int = 2, ctx: Context | None = None, stream=None,
                   workspace: torch.Tensor | None = None, sync: bool = True):
    """Mixed-precision decomposition (FP32 stages + Ogita-Aishima refinement).
    A: dense lower triangle; (rowptr, col, val): the same matrix in CSR."""
    ctx = ctx or default_context()
    A = _square(A, "A")
    n = A.shape[0]
    rowptr = _dev(rowptr, torch.int64, "rowptr", A.device, n + 1)
    col = _dev(col, torch.int32, "col", A.device)
    val = _dev(val, torch.float64, "val", A.device, col.numel())
    lam = torch.empty(n, dtype=torch.float64, device=A.device)
    V = empty_colmajor(n, n, A.device)
    if workspace is None:
        nbytes = ctx.lib.fraclap_eig_mixed_workspace_bytes(ctx.handle, n)
        workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=A.device)
    else:
        workspace = _ws(workspace, A.device)
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.eig_full_mixed(ctx.handle, _ptr(A), n, _ld(A), _ptr(rowptr), _ptr(col), _ptr(val),
                                     int(refine_iters), _ptr(lam), _ptr(V), max(n, 1), _ptr(workspace),
                                     workspace.numel(), None, st))
    if sync:
        ctx.sync(stream)
    return lam, V


def frac_apply(V: torch.Tensor, lam: torch.Tensor, F: torch.Tensor, pair_f, pair_alpha,
               ctx: Context | None = None, stream=None, out: torch.Tensor | None = None,
               workspace: torch.Tensor | None = None, sync: bool = True) -> torch.Tensor:
    """u_j = V diag(lam^{-alpha_j/2}) V^T F[:, pair_f[j]]; returns U (n x k, column-major)."""
    ctx = ctx or default_context()
    V = _square(V, "V")
    n = V.shape[0]
    dev = V.device
    F = _f64_colmajor(F, "F", rows=n, device=dev)
    pf = torch.as_tensor(pair_f, dtype=torch.int32).to(dev).contiguous()
    pa = torch.as_tensor(pair_alpha, dtype=torch.float64).to(dev).contiguous()
    k, m = pf.numel(), F.shape[1]
    if pa.numel() != k:
        raise ValueError("pair_f and pair_alpha differ in length")
    lam = _dev(lam, torch.float64, "lam", dev, n)
    U = _out(out, torch.float64, "out", dev, n, k) if out is not None else empty_colmajor(n, k, dev)
    if workspace is None:
        nbytes = ctx.lib.fraclap_apply_workspace_bytes_ctx(ctx.handle, n, m, k)
        workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    else:
        workspace = _ws(workspace, dev)
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.frac_apply(ctx.handle, _ptr(V), _ld(V), _ptr(lam.contiguous()), n, _ptr(F), _ld(F), m,
                                 _ptr(pf), _ptr(pa), k, _ptr(U), _ld(U), _ptr(workspace), workspace.numel(), st))
    if sync:
        ctx.sync(stream)
    return U


def frac_diffusion(V: torch.Tensor, lam: torch.Tensor, U0: torch.Tensor, pair_f, pair_alpha, pair_t,
                   mu: float = 1.0, ctx: Context | None = None, stream=None, out: torch.Tensor | None = None,
                   workspace: torch.Tensor | None = None, sync: bool = True) -> torch.Tensor:
    """u_j = V diag(exp(-mu lam^{alpha_j/2} t_j)) V^T U0[:, pair_f[j]]: the
    fractional diffusion solution at time t_j; returns U (n x k, column-major)."""
    ctx = ctx or default_context()
    V = _square(V, "V")
    n = V.shape[0]
    dev = V.device
    U0 = _f64_colmajor(U0, "U0", rows=n, device=dev)
    pf = torch.as_tensor(pair_f, dtype=torch.int32).to(dev).contiguous()
    pa = torch.as_tensor(pair_alpha, dtype=torch.float64).to(dev).contiguous()
    pt = torch.as_tensor(pair_t, dtype=torch.float64).to(dev).contiguous()
    k, m = pf.numel(), U0.shape[1]
    if pa.numel() != k or pt.numel() != k:
        raise ValueError("pair_f, pair_alpha and pair_t differ in length")
    lam = _dev(lam, torch.float64, "lam", dev, n)
    U = _out(out, torch.float64, "out", dev, n, k) if out is not None else empty_colmajor(n, k, dev)
    if workspace is None:
        nbytes = ctx.lib.fraclap_apply_workspace_bytes_ctx(ctx.handle, n, m, k)
        workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    else:
        workspace = _ws(workspace, dev)
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.frac_diffusion(ctx.handle, _ptr(V), _ld(V), _ptr(lam.contiguous()), n, _ptr(U0), _ld(U0), m,
                                     _ptr(pf), _ptr(pa), _ptr(pt), float(mu), k, _ptr(U), _ld(U),
                                     _ptr(workspace), workspace.numel(), st))
    if sync:
        ctx.sync(stream)
    return U


class ApplyGraph:
    """frac_apply (or frac_diffusion, when pair_t is given) captured once into
    a CUDA graph.  Later solves change the CONTENTS of the same buffers
    (self.F, self.pair_f, self.pair_alpha, self.pair_t, V, lam) and call
    launch(); the result is self.U.  Inputs must be CUDA tensors; pair
    arrays are copied to the device once, here."""

    def __init__(self, V: torch.Tensor, lam: torch.Tensor, F: torch.Tensor, pair_f, pair_alpha, pair_t=None,
                 mu: float = 1.0, ctx: Context | None = None, out: torch.Tensor | None = None):
        self.ctx = ctx or default_context()
        self.V = _square(V, "V")
        n, dev = self.V.shape[0], self.V.device
        self.F = _f64_colmajor(F, "F", rows=n, device=dev)
        self.lam = _dev(lam, torch.float64, "lam", dev, n)
        self.pair_f = torch.as_tensor(pair_f, dtype=torch.int32).to(dev).contiguous()
        self.pair_alpha = torch.as_tensor(pair_alpha, dtype=torch.float64).to(dev).contiguous()
        self.pair_t = None if pair_t is None else torch.as_tensor(pair_t, dtype=torch.float64).to(dev).contiguous()
        k, m = self.pair_f.numel(), self.F.shape[1]
        if self.pair_alpha.numel() != k or (self.pair_t is not None and self.pair_t.numel() != k):
            raise ValueError("pair arrays differ in length")
        self.U = _out(out, torch.float64, "out", dev, n, k) if out is not None else empty_colmajor(n, k, dev)
        nbytes = self.ctx.lib.fraclap_apply_workspace_bytes_ctx(self.ctx.handle, n, m, k)
        self.workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
        self.handle = ctypes.c_void_p()
        torch.cuda.synchronize(dev)  # the buffers above are ready before the capture reads their addresses
        self.ctx.check(self.ctx.lib.fraclap_apply_graph_create(
            self.ctx.handle, _ptr(self.V), _ld(self.V), _ptr(self.lam), n, _ptr(self.F), _ld(self.F), m,
            _ptr(self.pair_f), _ptr(self.pair_alpha), _ptr(self.pair_t), float(mu), k, _ptr(self.U), _ld(self.U),
            _ptr(self.workspace), self.workspace.numel(), ctypes.byref(self.handle)))

    @property
    def kernels(self) -> int:
        return int(self.ctx.lib.fraclap_graph_kernels(self.handle))

    def launch(self, stream=None, sync: bool = True) -> torch.Tensor:
        self.ctx.check(self.ctx.lib.fraclap_graph_launch(self.handle, ctypes.c_void_p(_stream(stream))))
        if sync:
            self.ctx.sync(stream)
        return self.U

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.ctx.lib.fraclap_graph_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tridiagonalize(A: torch.Tensor, want_q: bool = True, ctx: Context | None = None, stream=None):
    """A = Q T Q^T (two-stage reduction).  Returns (d, e, Q or None)."""
    ctx = ctx or default_context()
    A = _square(A, "A")
    n = A.shape[0]
    d = torch.empty(n, dtype=torch.float64, device=A.device)
    e = torch.empty(max(n - 1, 1), dtype=torch.float64, device=A.device)
    Q = empty_colmajor(n, n, A.device) if want_q else None
    nbytes = ctx.lib.fraclap_eig_workspace_bytes(ctx.handle, n)
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=A.device)
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.fraclap_tridiagonalize(ctx.handle, _ptr(A), n, _ld(A), _ptr(d), _ptr(e), _ptr(Q),
                                             max(n, 1), _ptr(ws), ws.numel(), st))
    ctx.sync(stream)
    return d, e[: max(n - 1, 0)], Q


def tridiag_eig(d: torch.Tensor, e: torch.Tensor, ctx: Context | None = None, stream=None):
    """Divide-and-conquer eigensolver of the symmetric tridiagonal (d, e)."""
    ctx = ctx or default_context()
    if not isinstance(d, torch.Tensor) or not d.is_cuda:
        raise TypeError("d must be a float64 CUDA tensor")
    d = _dev(d, torch.float64, "d", d.device)
    n = d.numel()
    e = _dev(e, torch.float64, "e", d.device, max(n - 1, 0))
    lam = torch.empty(n, dtype=torch.float64, device=d.device)
    Z = empty_colmajor(n, n, d.device)
    nbytes = ctx.lib.fraclap_tridiag_workspace_bytes(ctx.handle, n)
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=d.device)
    ee = e.contiguous() if e.numel() > 0 else torch.zeros(1, dtype=torch.float64, device=d.device)
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.fraclap_tridiag_eig(ctx.handle, _ptr(d.contiguous()), _ptr(ee), n, _ptr(lam), _ptr(Z),
                                          max(n, 1), _ptr(ws), ws.numel(), st))
    ctx.sync(stream)
    return lam, Z


def dgemm(A: torch.Tensor, B: torch.Tensor, trans_a=False, trans_b=False, alpha=1.0, beta=0.0,
          C: torch.Tensor | None = None, ctx: Context | None = None, stream=None) -> torch.Tensor:
    """C = alpha op(A) op(B) + beta C on the library's FP64 GEMM engine."""
    ctx = ctx or default_context()
    A = _f64_colmajor(A, "A")
    B = _f64_colmajor(B, "B", device=A.device)
    m = A.shape[1] if trans_a else A.shape[0]
    k = A.shape[0] if trans_a else A.shape[1]
    n = B.shape[0] if trans_b else B.shape[1]
    if (B.shape[1] if trans_b else B.shape[0]) != k:
        raise ValueError(f"inner dimensions differ: op(A) is {m} x {k}, op(B) has {B.shape[1] if trans_b else B.shape[0]} rows")
    if C is None:
        C = empty_colmajor(m, n, A.device)
        beta = 0.0
    else:
        C = _out(C, torch.float64, "C", A.device, m, n)
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.fraclap_dgemm(ctx.handle, int(trans_a), int(trans_b), m, n, k, float(alpha), _ptr(A),
                                    _ld(A), _ptr(B), _ld(B), float(beta), _ptr(C), _ld(C), st))
    ctx.sync(stream)
    return C


def sgemm(A: torch.Tensor, B: torch.Tensor, trans_a=False, trans_b=False, alpha=1.0, beta=0.0,
          C: torch.Tensor | None = None, form: int = 0, route: int = 1, ctx: Context | None = None,
          stream=None) -> torch.Tensor:
    """C = alpha op(A) op(B) + beta C in FP32: route 1 on the tensor cores (three TF32
    products), route 0 on the FP32 FMA kernel.  form 1: A symmetric (lower triangle read);
    form 2: only the lower triangle of C written."""
    ctx = ctx or default_context()
    for t, name in ((A, "A"), (B, "B")):
        if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 2 or t.device != A.device:
            raise TypeError(f"{name} must be a float32 CUDA matrix on A's device")
    A = A if colmajor_layout_ok(tuple(A.shape), A.stride()) else A.t().contiguous().t()
    B = B if colmajor_layout_ok(tuple(B.shape), B.stride()) else B.t().contiguous().t()
    m = A.shape[1] if trans_a else A.shape[0]
    k = A.shape[0] if trans_a else A.shape[1]
    n = B.shape[0] if trans_b else B.shape[1]
    if (B.shape[1] if trans_b else B.shape[0]) != k:
        raise ValueError("inner dimensions of op(A) and op(B) differ")
    if C is None:
        C = torch.zeros((n, m), dtype=torch.float32, device=A.device).t()
        beta = 0.0
    else:
        C = _out(C, torch.float32, "C", A.device, m, n)
    ws = ctx.lib.fraclap_sgemm_workspace_bytes(m, n, k)
    work = torch.empty(ws, dtype=torch.uint8, device=A.device)
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.fraclap_sgemm(ctx.handle, int(trans_a), int(trans_b), int(form), m, n, k, float(alpha),
                                    _ptr(A), _ld(A), _ptr(B), _ld(B), float(beta), _ptr(C), _ld(C), int(route),
                                    _ptr(work), ws, st))
    ctx.sync(stream)
    return C


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("A_dev", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("lambda_dev", ctypes.c_void_p), ("V_dev", ctypes.c_void_p), ("ldv", ctypes.c_int64),
                ("F_dev", ctypes.c_void_p), ("ldf", ctypes.c_int64), ("m", ctypes.c_int64),
                ("pair_f_dev", ctypes.c_void_p), ("pair_alpha_dev", ctypes.c_void_p), ("k", ctypes.c_int64),
                ("U_dev", ctypes.c_void_p), ("ldu", ctypes.c_int64),
                ("rowptr_dev", ctypes.c_void_p), ("col_dev", ctypes.c_void_p), ("val_dev", ctypes.c_void_p),
                ("refine_iters", ctypes.c_int)]


def solve_batched(problems, workers: int = 0, ctx: Context | None = None, stream=None) -> list:
    """Eigendecomposition (FP64 route) and spectral apply of many independent problems in
    one call.  problems: list of dicts with "A" (n x n float64 CUDA tensor) and optionally
    "F" (n x m), "pair_f", "pair_alpha" (k pairs), and "rowptr", "col", "val" (the CSR of A:
    the mixed route, with "refine_iters", default 6).  Returns per problem (lam, V, U or None)."""
    ctx = ctx or default_context()
    arr = (_Problem * max(len(problems), 1))()
    keep, out = [], []
    for i, pr in enumerate(problems):
        A = _square(pr["A"], f"problem {i}: A") if pr["A"].numel() else pr["A"]
        n = int(pr["A"].shape[0])
        dev = pr["A"].device
        lam = torch.empty(n, dtype=torch.float64, device=dev)
        V = empty_colmajor(n, n, dev)
        U = None
        k = 0
        if pr.get("pair_f") is not None and len(pr["pair_f"]) and n:
            Fm = _f64_colmajor(pr["F"], f"problem {i}: F", rows=n, device=dev)
            pf = torch.as_tensor(np.asarray(pr["pair_f"], dtype=np.int32)).to(dev)
            pa = torch.as_tensor(np.asarray(pr["pair_alpha"], dtype=np.float64)).to(dev)
            k = int(pf.numel())
            U = empty_colmajor(n, k, dev)
            keep += [Fm, pf, pa]
            arr[i].F_dev, arr[i].ldf, arr[i].m = Fm.data_ptr(), _ld(Fm), Fm.shape[1]
            arr[i].pair_f_dev, arr[i].pair_alpha_dev = pf.data_ptr(), pa.data_ptr()
            arr[i].U_dev, arr[i].ldu = U.data_ptr(), _ld(U)
        arr[i].n, arr[i].k = n, k
        if pr.get("rowptr") is not None and n:
            rp = _dev(pr["rowptr"], torch.int64, f"problem {i}: rowptr", dev, n + 1)
            cl = _dev(pr["col"], torch.int32, f"problem {i}: col", dev)
            vl = _dev(pr["val"], torch.float64, f"problem {i}: val", dev, cl.numel())
            keep += [rp, cl, vl]
            arr[i].rowptr_dev, arr[i].col_dev, arr[i].val_dev = rp.data_ptr(), cl.data_ptr(), vl.data_ptr()
            arr[i].refine_iters = int(pr.get("refine_iters", 6))
        if n:
            keep.append(A)
            arr[i].A_dev, arr[i].lda = A.data_ptr(), _ld(A)
            arr[i].lambda_dev, arr[i].V_dev, arr[i].ldv = lam.data_ptr(), V.data_ptr(), _ld(V)
        out.append((lam, V, U))
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.fraclap_solve_batched(ctx.handle, arr, len(problems), int(workers), st))
    ctx.sync(stream)
    return out


def dgemm_ozaki(A: torch.Tensor, B: torch.Tensor, trans_a=False, trans_b=False, alpha=1.0, beta=0.0,
                C: torch.Tensor | None = None, slices: int = 7, ctx: Context | None = None,
                stream=None) -> torch.Tensor:
    """C = alpha op(A) op(B) + beta C, FP64-accurate from BF16 tensor-core slices."""
    ctx = ctx or default_context()
    A = _f64_colmajor(A, "A")
    B = _f64_colmajor(B, "B", device=A.device)
    m = A.shape[1] if trans_a else A.shape[0]
    k = A.shape[0] if trans_a else A.shape[1]
    n = B.shape[0] if trans_b else B.shape[1]
    if (B.shape[1] if trans_b else B.shape[0]) != k:
        raise ValueError(f"inner dimensions differ: op(A) is {m} x {k}, op(B) has {B.shape[1] if trans_b else B.shape[0]} rows")
    if C is None:
        C = empty_colmajor(m, n, A.device)
        beta = 0.0
    else:
        C = _out(C, torch.float64, "C", A.device, m, n)
    nbytes = ctx.lib.fraclap_dgemm_ozaki_workspace_bytes(m, n, k, slices)
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=A.device)
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.fraclap_dgemm_ozaki(ctx.handle, int(trans_a), int(trans_b), m, n, k, float(alpha), _ptr(A),
                                          _ld(A), _ptr(B), _ld(B), float(beta), _ptr(C), _ld(C), int(slices),
                                          _ptr(ws), ws.numel(), st))
    ctx.sync(stream)
    return C


# ----------------------------------------------------------------------------
# the generalised problem K phi = theta M phi (finite elements)
# ----------------------------------------------------------------------------
def fem_assemble(mask: torch.Tensor, h: float, dense: bool = True, ctx: Context | None = None, stream=None):
    """Bilinear / trilinear finite-element stiffness K and mass M of a uint8
    mask ([y, x] or [z, y, x]) on the GPU.  Returns dict(idx, n, rowptr, col,
    valK, valM, K, M (column-major dense, or None))."""
    ctx = ctx or default_context()
    if mask.dtype != torch.uint8 or not mask.is_cuda:
        raise TypeError("mask must be a uint8 CUDA tensor")
    mask = mask.contiguous()
    dim = mask.dim()
    ext = (ctypes.c_int64 * 3)(*(list(reversed(mask.shape)) + [1] * (3 - dim)))
    idx = torch.empty(mask.shape, dtype=torch.int32, device=mask.device)
    n = ctypes.c_int64(-1)
    nnz = ctypes.c_int64(-1)
    st = ctypes.c_void_p(_stream(stream))
    ctx.check(ctx.lib.fem_assemble(ctx.handle, _ptr(mask), dim, ext, float(h), _ptr(idx), ctypes.byref(n),
                                   ctypes.byref(nnz), None, None, None, None, None, None, 0, st))
    N, NNZ = n.value, nnz.value
    rowptr = torch.empty(N + 1, dtype=torch.int64, device=mask.device)
    col = torch.empty(max(NNZ, 1), dtype=torch.int32, device=mask.device)
    vK = torch.empty(max(NNZ, 1), dtype=torch.float64, device=mask.device)
    vM = torch.empty(max(NNZ, 1), dtype=torch.float64, device=mask.device)
    K = empty_colmajor(N, N, mask.device) if (dense and N > 0) else None
    M = empty_colmajor(N, N, mask.device) if (dense and N > 0) else None
    ctx.check(ctx.lib.fem_assemble(ctx.handle, _ptr(mask), dim, ext, float(h), _ptr(idx), ctypes.byref(n),
                                   ctypes.byref(nnz), _ptr(rowptr), _ptr(col), _ptr(vK), _ptr(vM), _ptr(K), _ptr(M),
                                   max(N, 1), st))
    return {"idx": idx, "n": N, "rowptr": rowptr, "col": col[:NNZ], "valK": vK[:NNZ], "valM": vM[:NNZ], "K": K,
            "M": M}


def eig_pencil(K: torch.Tensor, rowptr, col, valM, half_bandwidth: int | None = None, ctx: Context | None = None,
               stream=None, sync: bool = True):
    """All eigenpairs of K phi = theta M phi (K dense, lower triangle read;
    M in CSR).  Returns (theta ascending, Phi column-major, Phi^T M Phi = I)."""
    ctx = ctx or default_context()
    K = _square(K, "K")
    n = K.shape[0]
    dev = K.device
    rowptr = _dev(rowptr, torch.int64, "rowptr", dev, n + 1)
    col = _dev(col, torch.int32, "col", dev)
    valM = _dev(valM, torch.float64, "valM", dev, col.numel())
    if half_bandwidth is None:
        half_bandwidth = csr_half_bandwidth(rowptr, col, ctx=ctx, stream=stream)
    theta = torch.empty(n, dtype=torch.float64, device=dev)
    Phi = empty_colmajor(n, n, dev)
    nbytes = ctx.lib.fraclap_eig_pencil_workspace_bytes(ctx.handle, n, int(half_bandwidth))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    ctx.check(ctx.lib.eig_pencil(ctx.handle, _ptr(K), _ld(K), n, _ptr(rowptr), _ptr(col), _ptr(valM),
                                 int(half_bandwidth), _ptr(theta), _ptr(Phi), max(n, 1), _ptr(ws), ws.numel(),
                                 ctypes.c_void_p(_stream(stream))))
    if sync:
        ctx.sync(stream)
    return theta, Phi


def frac_apply_mass(Phi: torch.Tensor, theta: torch.Tensor, rowptr, col, valM, F: torch.Tensor, pair_f, pair_alpha,
                    ctx: Context | None = None, stream=None, out: torch.Tensor | None = None,
                    sync: bool = True) -> torch.Tensor:
    """u_j = Phi diag(theta^{-alpha_j/2}) Phi^T M F[:, pair_f[j]] (the apply
    with the M-inner product); returns U (n x k, column-major)."""
    ctx = ctx or default_context()
    Phi = _square(Phi, "Phi")
    n = Phi.shape[0]
    dev = Phi.device
    F = _f64_colmajor(F, "F", rows=n, device=dev)
    rowptr = _dev(rowptr, torch.int64, "rowptr", dev, n + 1)
    col = _dev(col, torch.int32, "col", dev)
    valM = _dev(valM, torch.float64, "valM", dev, col.numel())
    theta = _dev(theta, torch.float64, "theta", dev, n)
    pf = torch.as_tensor(pair_f, dtype=torch.int32).to(dev).contiguous()
    pa = torch.as_tensor(pair_alpha, dtype=torch.float64).to(dev).contiguous()
    k, m = pf.numel(), F.shape[1]
    if pa.numel() != k:
        raise ValueError("pair_f and pair_alpha differ in length")
    U = _out(out, torch.float64, "out", dev, n, k) if out is not None else empty_colmajor(n, k, dev)
    nbytes = ctx.lib.fraclap_apply_mass_workspace_bytes(ctx.handle, n, m, k)
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    ctx.check(ctx.lib.frac_apply_mass(ctx.handle, _ptr(Phi), _ld(Phi), _ptr(theta), n, _ptr(rowptr), _ptr(col),
                                      _ptr(valM), _ptr(F), _ld(F), m, _ptr(pf), _ptr(pa), k, _ptr(U), _ld(U), _ptr(ws),
                                      ws.numel(), ctypes.c_void_p(_stream(stream))))
    if sync:
        ctx.sync(stream)
    return U


# ----------------------------------------------------------------------------
# exact eigenvalue counts and spectrum slicing (Sec. III-D)
# ----------------------------------------------------------------------------
def _csr_args(rowptr, col, valK, valM=None):
    if not isinstance(rowptr, torch.Tensor) or not rowptr.is_cuda:
        raise TypeError("rowptr must be an int64 CUDA tensor")
    dev = rowptr.device
    n = rowptr.numel() - 1
    if n < 1:
        raise ValueError("the matrix must have at least one row")
    rowptr = _dev(rowptr, torch.int64, "rowptr", dev)
    col = _dev(col, torch.int32, "col", dev)
    valK = _dev(valK, torch.float64, "valK", dev, col.numel())
    if valM is not None:
        valM = _dev(valM, torch.float64, "valM", dev, col.numel())
    return n, dev, rowptr, col, valK, valM


def csr_half_bandwidth(rowptr: torch.Tensor, col: torch.Tensor, ctx: Context | None = None, stream=None) -> int:
    """max(i - j) over the lower-triangle entries of a CSR matrix (synchronises)."""
    ctx = ctx or default_context()
    n = rowptr.numel() - 1
    bw = ctypes.c_int64(0)
    rp = _dev(rowptr, torch.int64, "rowptr", rowptr.device)
    cl = _dev(col, torch.int32, "col", rowptr.device)
    ctx.check(ctx.lib.fraclap_csr_half_bandwidth(ctx.handle, n, _ptr(rp), _ptr(cl), ctypes.byref(bw),
                                                 ctypes.c_void_p(_stream(stream))))
    return int(bw.value)


def inertia_counts(rowptr, col, valK, sigmas, valM=None, half_bandwidth: int | None = None,
                   ctx: Context | None = None, stream=None, sync: bool = True) -> torch.Tensor:
    """#{eigenvalues < sigma} of the CSR matrix K (or of the pencil (K, M))
    for every shift, from the inertia of the banded LDL^T (Sec. III-D-2);
    -1 where a pivot is exactly zero.  Returns an int64 CUDA tensor."""
    ctx = ctx or default_context()
    n, dev, rowptr, col, valK, valM = _csr_args(rowptr, col, valK, valM)
    sig = torch.as_tensor(sigmas, dtype=torch.float64).to(dev).contiguous().reshape(-1)
    if half_bandwidth is None:
        half_bandwidth = csr_half_bandwidth(rowptr, col, ctx=ctx, stream=stream)
    out = torch.empty(sig.numel(), dtype=torch.int64, device=dev)
    nbytes = ctx.lib.fraclap_inertia_workspace_bytes(n, int(half_bandwidth), sig.numel(), int(valM is not None))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    ctx.check(ctx.lib.fraclap_inertia_counts(ctx.handle, n, _ptr(rowptr), _ptr(col), _ptr(valK), _ptr(valM),
                                             int(half_bandwidth), _ptr(sig), sig.numel(), _ptr(out), _ptr(ws),
                                             ws.numel(), ctypes.c_void_p(_stream(stream))))
    if sync:
        ctx.sync(stream)
    return out


def _tridiag_args(d, e):
    if not isinstance(d, torch.Tensor) or not d.is_cuda:
        raise TypeError("d must be a float64 CUDA tensor")
    d = _dev(d, torch.float64, "d", d.device)
    n = d.numel()
    if n < 1:
        raise ValueError("T must have at least one row")
    e = _dev(e, torch.float64, "e", d.device, n - 1) if n > 1 else torch.zeros(1, dtype=torch.float64,
                                                                                device=d.device)
    return n, d, e


def sturm_counts(d, e, sigmas, ctx: Context | None = None, stream=None) -> torch.Tensor:
    """#{eigenvalues < sigma} of the tridiagonal (d, e) for every shift (Sturm recurrence)."""
    ctx = ctx or default_context()
    n, d, e = _tridiag_args(d, e)
    sig = torch.as_tensor(sigmas, dtype=torch.float64).to(d.device).contiguous().reshape(-1)
    out = torch.empty(sig.numel(), dtype=torch.int64, device=d.device)
    ctx.check(ctx.lib.fraclap_sturm_counts(ctx.handle, _ptr(d), _ptr(e), n, _ptr(sig), sig.numel(), _ptr(out),
                                           ctypes.c_void_p(_stream(stream))))
    ctx.sync(stream)
    return out


def bisect(d, e, k0: int, k1: int, ctx: Context | None = None, stream=None) -> torch.Tensor:
    """Eigenvalues k0..k1 (0-based, ascending) of the tridiagonal (d, e) by bisection."""
    ctx = ctx or default_context()
    n, d, e = _tridiag_args(d, e)
    lam = torch.empty(max(int(k1) - int(k0) + 1, 1), dtype=torch.float64, device=d.device)
    ctx.check(ctx.lib.fraclap_bisect(ctx.handle, _ptr(d), _ptr(e), n, int(k0), int(k1), _ptr(lam),
                                     ctypes.c_void_p(_stream(stream))))
    ctx.sync(stream)
    return lam


def partition_spectrum(rowptr, col, valK, rho: float, P: int, n_a: int = 7, n_b: int = 0, n_c: int = 10,
                       imbalance: float = 0.25, valM=None, half_bandwidth: int | None = None,
                       ctx: Context | None = None, stream=None):
    """Greedy spectrum slicing of Sec. III-D on GPU inertia counts: P
    subintervals of [0, rho] with about n / P eigenvalues each.  Returns
    (splits, loads, history) as numpy arrays (P - 1 split points, P exact
    loads, the largest load after each step)."""
    ctx = ctx or default_context()
    n, dev, rowptr, col, valK, valM = _csr_args(rowptr, col, valK, valM)
    if half_bandwidth is None:
        half_bandwidth = csr_half_bandwidth(rowptr, col, ctx=ctx, stream=stream)
    splits = np.zeros(max(P - 1, 1))
    loads = np.zeros(max(P, 1), dtype=np.int64)
    cap = 1 + n_a + n_b
    hist = np.zeros(cap, dtype=np.int64)
    nbytes = ctx.lib.fraclap_inertia_workspace_bytes(n, int(half_bandwidth), max(P - 1, 1), int(valM is not None))
    ws = torch.empty(nbytes + 512 + 16 * max(P - 1, 1), dtype=torch.uint8, device=dev)
    rc = ctx.lib.fraclap_partition_spectrum(ctx.handle, n, _ptr(rowptr), _ptr(col), _ptr(valK), _ptr(valM),
                                            int(half_bandwidth), float(rho), int(P), int(n_a), int(n_b), int(n_c),
                                            float(imbalance), splits.ctypes.data_as(ctypes.c_void_p),
                                            loads.ctypes.data_as(ctypes.c_void_p),
                                            hist.ctypes.data_as(ctypes.c_void_p), cap, _ptr(ws), ws.numel(),
                                            ctypes.c_void_p(_stream(stream)))
    if rc < 0:
        ctx.check(rc)
    return splits[: max(P - 1, 0)], loads[:P], hist[:rc]


def solve(mask: torch.Tensor, h: float, F: torch.Tensor, pair_f, pair_alpha, ctx: Context | None = None):
    """The whole path on the GPU: assemble, decompose, apply.  Returns (lam, V, U)."""
    asm = fd_assemble(mask, h, dense=True, ctx=ctx)
    lam, V = eig_full(asm["A"], ctx=ctx)
    U = frac_apply(V, lam, F, pair_f, pair_alpha, ctx=ctx)
    return lam, V, U


# ----------------------------------------------------------------------------
# checkpoint of a decomposition (host-side file I/O in the library)
# ----------------------------------------------------------------------------
def _host_mask(mask):
    m = mask.detach().cpu().numpy() if isinstance(mask, torch.Tensor) else np.asarray(mask)
    m = np.ascontiguousarray(m, dtype=np.uint8)
    if m.ndim not in (2, 3):
        raise ValueError("mask must be 2-D [y, x] or 3-D [z, y, x]")
    ext = np.array(list(reversed(m.shape)) + [1] * (3 - m.ndim), dtype=np.int64)
    return m, ext


def _check_io(lib, rc: int, what: str):
    if rc != 0:
        raise FraclapError(rc, f"{what}: {lib.fraclap_strerror(rc).decode()}")


def mask_hash(mask, h: float) -> int:
    """FNV-1a-64 of the grid (dimension, extents, h) and the mask, as stored
    in a checkpoint."""
    lib = load_library()
    m, ext = _host_mask(mask)
    return int(lib.fraclap_mask_hash(m.ctypes.data_as(ctypes.c_void_p), m.ndim,
                                     ext.ctypes.data_as(ctypes.c_void_p), float(h)))


def save_decomposition(path: str, lam, V, mask=None, h: float = 0.0) -> None:
    """Writes (n, lambda, V) to `path` (V is copied to the host), tagged with
    the grid of `mask` and h when given."""
    lib = load_library()
    lam_h = np.ascontiguousarray((lam.detach().cpu().numpy() if isinstance(lam, torch.Tensor) else lam), np.float64)
    V_h = np.asfortranarray((V.detach().cpu().numpy() if isinstance(V, torch.Tensor) else V), np.float64)
    n = lam_h.shape[0]
    if V_h.shape != (n, n):
        raise ValueError("V must be n x n")
    if mask is not None:
        m, ext = _host_mask(mask)
        dim, mh = m.ndim, mask_hash(m, h)
    else:
        ext, dim, mh = np.zeros(3, np.int64), 0, 0
    rc = lib.fraclap_save_decomposition(os.fsencode(path), n, lam_h.ctypes.data_as(ctypes.c_void_p),
                                        V_h.ctypes.data_as(ctypes.c_void_p), max(n, 1), dim,
                                        ext.ctypes.data_as(ctypes.c_void_p), float(h), mh)
    _check_io(lib, rc, f"save_decomposition({path})")


def load_decomposition(path: str, mask=None, h: float | None = None, device=None):
    """Reads (lambda, V) from `path` onto `device` (default: the current CUDA
    device if there is one, else the host); V is column-major.  With `mask`
    and h given, the file must belong to that grid."""
    lib = load_library()
    expect = mask_hash(mask, h) if mask is not None else 0
    n = ctypes.c_int64(0)
    rc = lib.fraclap_load_decomposition(os.fsencode(path), ctypes.byref(n), None, None, None, None, None, None, 0,
                                        expect)
    _check_io(lib, rc, f"load_decomposition({path})")
    nn = n.value
    lam_h = np.empty(max(nn, 1))
    V_h = np.empty((max(nn, 1), max(nn, 1)), order="F")
    rc = lib.fraclap_load_decomposition(os.fsencode(path), None, None, None, None, None,
                                        lam_h.ctypes.data_as(ctypes.c_void_p), V_h.ctypes.data_as(ctypes.c_void_p),
                                        max(nn, 1), expect)
    _check_io(lib, rc, f"load_decomposition({path})")
    if device is None:
        device = torch.device("cuda") if torch.cuda.is_available() else torch.device("cpu")
    lam = torch.from_numpy(lam_h[:nn].copy()).to(device)
    V = torch.from_numpy(np.ascontiguousarray(V_h[:nn, :nn].T)).to(device).t()
    return lam, V
