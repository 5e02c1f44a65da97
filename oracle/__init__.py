"""FP64 CPU oracle (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is the plain, slow statement of
what the fractional Poisson path computes (arXiv:1911.11906, Sec. II and
Sec. III-D-2), written independently of the CUDA path: the two share no code.

Pinned functions (see ``tests/test_oracle_*.py``): assembly, Householder +
implicit-QR eigensolver, Jacobi, inertia counting, banded direct solve,
spectral apply, fractional diffusion, and the finite-element generalised
problem (assembly of K and M, Cholesky-reduced eigensolver, inertia of
K - sigma M, apply in the M-inner product), Sturm counts and bisection on
the tridiagonal form, and the greedy spectrum partitioner of Sec. III-D.  No function here is unpinned.
"""
from .oracle import *  # noqa: F401,F403
