"""The CUDA-graph form of the apply: a replay gives what the direct call
gives, also after the inputs' contents change in place; diffusion and the
tensor-core route too; device errors still reach the context; the launch
count follows the replays."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _colmajor(a):
    a = np.asfortranarray(a, dtype=np.float64)
    return torch.from_numpy(a.T.copy()).cuda().t()


@pytest.fixture(scope="module")
def decomposition():
    p = I.square_problem(20)
    _, A = O.assemble(p.mask, p.h)
    lam, V = O.eig_full(A.dense())
    return p, _colmajor(V), torch.from_numpy(lam).cuda()


def _close(a, b, tol):
    return float((a - b).abs().max()) <= tol * float(b.abs().max())


@pytest.mark.parametrize("slices", [0, 6])
def test_graph_replays_the_apply(decomposition, slices):
    import paper_1911_11906_gb300 as F
    p, V, lam = decomposition
    ctx = F.Context()
    ctx.set_apply_slices(slices)
    Fd = _colmajor(p.F)
    g = F.ApplyGraph(V, lam, Fd, p.pair_f, p.pair_alpha, ctx=ctx)
    assert g.kernels > 0
    n0 = ctx.launch_count()
    U = g.launch().clone()
    assert ctx.launch_count() - n0 == g.kernels
    ref = F.frac_apply(V, lam, Fd, p.pair_f, p.pair_alpha, ctx=ctx)
    assert _close(U, ref, 0.0 if slices == 0 else 1e-14)
    # new forcings and orders in the same buffers, one more launch
    rng = np.random.default_rng(1)
    g.F.copy_(_colmajor(rng.standard_normal(p.F.shape)))
    g.pair_alpha.copy_(torch.from_numpy(rng.uniform(0.1, 1.9, p.pair_alpha.size)))
    U2 = g.launch()
    ref2 = F.frac_apply(V, lam, g.F, g.pair_f, g.pair_alpha, ctx=ctx)
    assert _close(U2, ref2, 0.0 if slices == 0 else 1e-14)
    g.close()


def test_graph_replays_the_diffusion_and_reports_errors(decomposition):
    import paper_1911_11906_gb300 as F
    p, V, lam = decomposition
    ctx = F.Context()
    Fd = _colmajor(p.F)
    k = p.pair_f.size
    t = np.linspace(0.0, 0.4, k)
    lam_buf = lam.clone()
    g = F.ApplyGraph(V, lam_buf, Fd, p.pair_f, p.pair_alpha, pair_t=t, mu=1.5, ctx=ctx)
    ref = F.frac_diffusion(V, lam, Fd, p.pair_f, p.pair_alpha, t, mu=1.5, ctx=ctx)
    assert torch.equal(g.launch(), ref)
    g.pair_t.mul_(0.5)
    ref = F.frac_diffusion(V, lam, Fd, p.pair_f, p.pair_alpha, t * 0.5, mu=1.5, ctx=ctx)
    assert torch.equal(g.launch(), ref)
    # an eigenvalue made zero in the graph's own buffer: the kernel's check reaches the context
    lam_buf[3] = 0.0
    with pytest.raises(F.FraclapError) as ei:
        g.launch()
    assert ei.value.code == -2
    ctx.sync()
    g.close()


def test_graph_needs_a_caller_workspace(decomposition):
    import paper_1911_11906_gb300 as F
    p, V, lam = decomposition
    ctx = F.Context()
    Fd = _colmajor(p.F)
    pf = torch.from_numpy(p.pair_f.astype(np.int32)).cuda()
    pa = torch.from_numpy(p.pair_alpha).cuda()
    U = F._binding.empty_colmajor(p.n, pf.numel(), V.device)
    h = ctypes.c_void_p()
    rc = ctx.lib.fraclap_apply_graph_create(ctx.handle, V.data_ptr(), p.n, lam.data_ptr(), p.n, Fd.data_ptr(),
                                            p.n, p.F.shape[1], pf.data_ptr(), pa.data_ptr(), None, 1.0,
                                            pf.numel(), U.data_ptr(), p.n, None, 0, ctypes.byref(h))
    assert rc == -1 and not h.value
    assert ctx.lib.fraclap_graph_launch(None, None) == -1
    assert ctx.lib.fraclap_graph_kernels(None) == -1
    ctx.lib.fraclap_graph_destroy(None)


def test_stage_times_stay_readable_after_a_capture_with_profiling(decomposition):
    """With profiling on, capturing the apply into a graph records no stage
    events inside the capture: stage_times() afterwards reads only the
    events of direct calls, and the graph's replays give the direct result."""
    import paper_1911_11906_gb300 as F
    p, V, lam = decomposition
    ctx = F.Context()
    ctx.set_profiling(True)
    Fd = _colmajor(p.F)
    direct = F.frac_apply(V, lam, Fd, p.pair_f, p.pair_alpha, ctx=ctx)
    g = F.ApplyGraph(V, lam, Fd, p.pair_f, p.pair_alpha, ctx=ctx)
    out = g.launch()
    times = ctx.stage_times()  # raised on captured events before
    assert times["apply"][1] == 1 and times["apply"][0] > 0.0
    assert _close(out, direct, 1e-15)
    F.frac_apply(V, lam, Fd, p.pair_f, p.pair_alpha, ctx=ctx)
    assert ctx.stage_times()["apply"][1] == 1
    g.close()
