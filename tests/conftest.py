import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: oracle runs of several seconds")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def square48():
    """The 48 x 48 unit-square workload and its oracle decomposition (computed once)."""
    import oracle as O
    from paper_1911_11906_gb300 import inputs as I
    p = I.square_problem(48)
    _, A = O.assemble(p.mask, p.h)
    lam, V = O.eig_full(A.dense())
    return p, A, lam, V


def square_closed_form(m: int, dim: int = 2) -> np.ndarray:
    """Eigenvalues (4/h^2) sum_d sin^2(j_d pi h / 2), j_d = 1..m, of the
    Dirichlet 5-/7-point Laplacian on the m^dim grid, ascending."""
    h = 1.0 / (m + 1)
    s = np.sin(np.arange(1, m + 1) * np.pi * h / 2.0) ** 2
    tot = np.zeros((m,) * dim)
    for d in range(dim):
        shape = [1] * dim
        shape[d] = m
        tot = tot + s.reshape(shape)
    return np.sort((4.0 / h ** 2) * tot.ravel())
