"""fraclap: fractional Poisson solves by eigenfunction expansion on GB300.

Thin Python binding of the C ABI in ``include/fraclap.h`` (argument
marshalling only; every step runs in the library's CUDA kernels).  PyTorch
supplies device memory and the current stream.  The library is built
in-tree by ``paper_1911_11906_gb300.build``; if it is missing, every call
raises instead of falling back to anything else.
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    FraclapError,
    Context,
    load_library,
    library_path,
    fd_assemble,
    eig_full,
    eig_full_mixed,
    frac_apply,
    frac_diffusion,
    ApplyGraph,
    tridiagonalize,
    tridiag_eig,
    dgemm,
    sgemm,
    dgemm_ozaki,
    solve,
    solve_batched,
    fem_assemble,
    eig_pencil,
    frac_apply_mass,
    csr_half_bandwidth,
    inertia_counts,
    sturm_counts,
    bisect,
    partition_spectrum,
    default_context,
    mask_hash,
    save_decomposition,
    load_decomposition,
)
from . import autotune  # noqa: E402,F401  (schedule autotuner with a persistent cache)
