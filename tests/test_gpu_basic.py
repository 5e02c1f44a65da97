"""GPU parity of the assembly kernel, the FP64 GEMM engine and the spectral
apply against the FP64 CPU oracle (all calls go through the C ABI)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _F():
    import paper_1911_11906_gb300 as F
    return F


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _colmajor(a):
    a = np.asfortranarray(a, dtype=np.float64)
    return torch.from_numpy(a.T.copy()).cuda().t()


@pytest.mark.parametrize("which", ["square48", "ellipse128", "holed_cube", "golden2d", "golden3d", "strip"])
def test_assembly_bitwise(which):
    F = _F()
    if which == "square48":
        p = I.square_problem(48); mask, h = p.mask, p.h
    elif which == "ellipse128":
        p = I.ellipse_problem(); mask, h = p.mask, p.h
    elif which == "holed_cube":
        p = I.holed_cube_problem(16, n_forcings=1); mask, h = p.mask, p.h
    elif which == "strip":
        mask, h = np.ones((1, 37), np.uint8), 1.0 / 38
    else:
        name = "assemble_2d_3x2.txt" if which == "golden2d" else "assemble_3d_2x2x2.txt"
        from test_oracle_pins import _read_golden
        mask, h, _ = _read_golden(name)
    idx_o, A_o = O.assemble(mask, h)
    out = F.fd_assemble(_cuda(mask), h, dense=A_o.n <= 12000)
    assert out["n"] == A_o.n
    np.testing.assert_array_equal(out["idx"].cpu().numpy().reshape(-1), idx_o)
    np.testing.assert_array_equal(out["rowptr"].cpu().numpy(), A_o.rowptr)
    np.testing.assert_array_equal(out["col"].cpu().numpy(), A_o.col)
    np.testing.assert_array_equal(out["val"].cpu().numpy(), A_o.val)  # bit-exact doubles
    if out["A"] is not None:
        np.testing.assert_array_equal(out["A"].cpu().numpy(), A_o.dense())


def test_assembly_empty_mask():
    F = _F()
    out = F.fd_assemble(_cuda(np.zeros((5, 7), np.uint8)), 0.1)
    assert out["n"] == 0 and out["rowptr"].cpu().numpy().tolist() == [0]
    assert np.all(out["idx"].cpu().numpy() == -1)


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (63, 65, 17), (130, 70, 200), (64, 64, 0), (257, 3, 1000)])
def test_dgemm_against_float64_reference(ta, tb, m, n, k):
    F = _F()
    rng = np.random.default_rng(m * 1000 + n * 10 + k)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C0 = rng.standard_normal((m, n))
    ref = 0.5 * (A.T if ta else A) @ (B.T if tb else B) - 2.0 * C0
    C = _colmajor(C0)
    F.dgemm(_colmajor(A), _colmajor(B), trans_a=ta, trans_b=tb, alpha=0.5, beta=-2.0, C=C)
    got = C.cpu().numpy()
    scale = np.abs(A).max(initial=1) * np.abs(B).max(initial=1) * max(k, 1)
    assert np.max(np.abs(got - ref)) <= 1e-14 * scale + 1e-13


@pytest.fixture(scope="module")
def square_small():
    p = I.square_problem(20)
    _, A = O.assemble(p.mask, p.h)
    lam, V = O.eig_full(A.dense())
    return p, A, lam, V


def test_frac_apply_matches_oracle(square_small):
    F = _F()
    p, A, lam, V = square_small
    U_o = O.frac_apply(V, lam, p.F, p.pair_f, p.pair_alpha)
    U = F.frac_apply(_colmajor(V), _cuda(lam), _colmajor(p.F), p.pair_f, p.pair_alpha).cpu().numpy()
    for j in range(U_o.shape[1]):
        assert np.linalg.norm(U[:, j] - U_o[:, j]) <= 1e-13 * np.linalg.norm(U_o[:, j])


def test_frac_apply_edge_cases(square_small):
    F = _F()
    p, A, lam, V = square_small
    Vd, ld = _colmajor(V), _cuda(lam)
    # alpha = 0 returns f; repeated forcings; negative orders
    U = F.frac_apply(Vd, ld, _colmajor(p.F), [0, 0, 1, 2], [0.0, -2.0, 0.0, 2.0]).cpu().numpy()
    assert np.linalg.norm(U[:, 0] - p.F[:, 0]) <= 1e-13 * np.linalg.norm(p.F[:, 0])
    Af = O.spmv(A, p.F[:, 0])
    assert np.linalg.norm(U[:, 1] - Af) <= 1e-12 * np.linalg.norm(Af)
    u2 = O.band_solve(A, p.F[:, 2])
    assert np.linalg.norm(U[:, 3] - u2) <= 1e-12 * np.linalg.norm(u2)
    # a non-positive eigenvalue with alpha != 0 is reported
    bad = lam.copy()
    bad[3] = 0.0
    with pytest.raises(F.FraclapError) as ei:
        F.frac_apply(Vd, _cuda(bad), _colmajor(p.F), [0], [1.0])
    assert ei.value.code == -2
    # ... but alpha = 0 never evaluates the power
    F.frac_apply(Vd, _cuda(bad), _colmajor(p.F), [0], [0.0])


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (63, 65, 17), (130, 70, 300), (257, 33, 1000)])
def test_dgemm_ozaki_is_fp64_accurate(ta, tb, m, n, k):
    """BF16-slice products reach FP64 accuracy (7 slices) against an exact
    reference computed with error-free accumulation (math.fsum)."""
    import math
    F = _F()
    rng = np.random.default_rng(m + 7 * n + 13 * k)
    A = rng.standard_normal((k, m) if ta else (m, k)) * np.exp(rng.uniform(-8, 8, size=(k, m) if ta else (m, k)))
    B = rng.standard_normal((n, k) if tb else (k, n))
    opA, opB = (A.T if ta else A), (B.T if tb else B)
    C0 = rng.standard_normal((m, n))
    C = _colmajor(C0)
    F.dgemm_ozaki(_colmajor(A), _colmajor(B), trans_a=ta, trans_b=tb, alpha=0.5, beta=-2.0, C=C)
    got = C.cpu().numpy()
    for (i, j) in [(0, 0), (m - 1, n - 1), (m // 2, n // 3)]:
        exact = 0.5 * math.fsum(opA[i, :] * opB[:, j]) - 2.0 * C0[i, j]
        scale = 0.5 * np.abs(opA[i, :]).max() * np.abs(opB[:, j]).max() * k + 2 * abs(C0[i, j])
        assert abs(got[i, j] - exact) <= 4e-16 * scale
    ref = 0.5 * opA @ opB - 2.0 * C0
    rowmax = np.abs(opA).max(axis=1)[:, None] * np.abs(opB).max(axis=0)[None, :] * k
    assert np.max(np.abs(got - ref) / (rowmax + 1e-300)) <= 1e-15


@pytest.mark.parametrize("group,bits,tile_n,cluster", [
    (0, 7, 128, 1), (1, 7, 128, 1), (3, 8, 128, 1), (8, 8, 128, 1), (8, 7, 128, 1), (0, 7, 256, 1), (4, 7, 256, 1),
    (2, 8, 256, 1), (0, 7, 128, 2), (0, 7, 256, 2), (3, 8, 256, 2), (4, 7, 256, 2), (1, 8, 128, 2),
    (0, 7, 192, 1), (3, 8, 192, 1), (0, 7, 192, 2), (2, 7, 192, 2)])
@pytest.mark.parametrize("ta,m,n,k", [(True, 300, 260, 1000), (False, 520, 130, 2000), (True, 129, 385, 257),
                                      (True, 640, 600, 300)])
def test_dgemm_ozaki_schedules_agree(group, bits, tile_n, cluster, ta, m, n, k):
    """Every tile order (raster group), tile width, cluster size (B tile
    shared by TMA multicast; clusters that run past the last tile row) and
    digit width gives an FP64-accurate product (against math.fsum at sampled
    entries and the FP64 product everywhere), and schedules with the same
    digit width give the same bits: only the tiling and the order of the
    tiles over the CTAs differ, not the sums of any output element."""
    import math
    F = _F()
    rng = np.random.default_rng(m + 3 * n + k + group)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((k, n))
    opA = A.T if ta else A
    ctx = F.Context(wait_timeout_s=2.0)
    ctx.set_schedule("ozaki_group", group)
    ctx.set_schedule("ozaki_bits", bits)
    ctx.set_schedule("ozaki_tile_n", tile_n)
    ctx.set_schedule("ozaki_cluster", cluster)
    assert ctx.get_schedule("ozaki_group") == group and ctx.get_schedule("ozaki_bits") == bits
    assert ctx.get_schedule("ozaki_tile_n") == tile_n and ctx.get_schedule("ozaki_cluster") == cluster
    got = F.dgemm_ozaki(_colmajor(A), _colmajor(B), trans_a=ta, ctx=ctx).cpu().numpy()
    scale = np.abs(opA).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :] * k
    assert np.max(np.abs(got - opA @ B) / scale) <= 1e-15
    for (i, j) in [(0, 0), (m - 1, n - 1), (m // 2, n // 3), (m - 1, 0)]:
        assert abs(got[i, j] - math.fsum(opA[i, :] * B[:, j])) <= 4e-16 * scale[i, j]
    ref_ctx = F.Context(wait_timeout_s=2.0)
    ref_ctx.set_schedule("ozaki_group", 0)
    ref_ctx.set_schedule("ozaki_bits", bits)
    same = F.dgemm_ozaki(_colmajor(A), _colmajor(B), trans_a=ta, ctx=ref_ctx).cpu().numpy()
    assert np.array_equal(got, same)


def test_schedule_knobs_reject_bad_values():
    F = _F()
    ctx = F.Context()
    for knob, bad in (("ozaki_group", -1), ("ozaki_bits", 6), ("ozaki_bits", 9), ("ozaki_tile_n", 160),
                      ("fp32_stages_tc", 2), ("q2_parts", 5), ("ozaki_cluster", 3), ("ozaki_cluster", 4)):
        with pytest.raises(F.FraclapError):
            ctx.set_schedule(knob, bad)
    assert ctx.lib.fraclap_set_schedule(ctx.handle, 99, 1) == -1


def test_dgemm_ozaki_fewer_slices_bound():
    F = _F()
    rng = np.random.default_rng(5)
    A = rng.standard_normal((200, 300))
    B = rng.standard_normal((300, 150))
    ref = A @ B
    for s in (3, 5):
        got = F.dgemm_ozaki(_colmajor(A), _colmajor(B), slices=s).cpu().numpy()
        scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :] * 300
        assert np.max(np.abs(got - ref) / scale) <= 2.0 ** (-8 * s + 4)


@pytest.mark.parametrize("m,n,k", [(128, 64, 64), (130, 70, 300), (257, 200, 1000), (64, 300, 64)])
def test_tcgen05_slice_products_match_mma_sync_route(m, n, k):
    """The tcgen05/TMA route and the mma.sync route compute the same exact
    slice products: results agree to the last bits, and both match FP64."""
    F = _F()
    rng = np.random.default_rng(m * 3 + n * 5 + k)
    A = rng.standard_normal((k, m))
    B = rng.standard_normal((k, n))
    ctx_tc = F.Context(wait_timeout_s=2.0)
    ctx_ms = F.Context(wait_timeout_s=2.0)
    ctx_ms.set_tensor_route(0)
    out = [F.dgemm_ozaki(_colmajor(A), _colmajor(B), trans_a=True, ctx=ctx).cpu().numpy()
           for ctx in (ctx_tc, ctx_ms)]
    ref = A.T @ B
    scale = np.abs(A).max(axis=0)[:, None] * np.abs(B).max(axis=0)[None, :] * k
    assert np.max(np.abs(out[0] - out[1]) / scale) <= 1e-16
    assert np.max(np.abs(out[0] - ref) / scale) <= 1e-15


def _f32_colmajor(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32).T)).cuda().t()


def _sgemm_case(route, form, ta, tb, m, n, k):
    """FP32 GEMM (tensor-core route: three TF32 products; FMA route) against an
    FP64 product of the same FP32 inputs, relative to sum_k |a_ik| |b_kj|."""
    F = _F()
    rng = np.random.default_rng(m * 7 + n * 3 + k + form)
    A = rng.standard_normal((k, m) if ta else (m, k)).astype(np.float32)
    if form == 1:
        A = np.tril(A) + np.tril(A, -1).T  # only the lower triangle is read
        A_stored = np.tril(A) + 1e3 * np.triu(np.ones_like(A), 1)  # garbage above
    else:
        A_stored = A
    B = rng.standard_normal((n, k) if tb else (k, n)).astype(np.float32)
    C0 = rng.standard_normal((m, n)).astype(np.float32)
    opA = (A.T if ta else A).astype(np.float64)
    opB = (B.T if tb else B).astype(np.float64)
    ref = 0.5 * opA @ opB - 2.0 * C0.astype(np.float64)
    scale = 0.5 * np.abs(opA) @ np.abs(opB) + 2.0 * np.abs(C0.astype(np.float64))
    C = _f32_colmajor(C0)
    F.sgemm(_f32_colmajor(A_stored), _f32_colmajor(B), trans_a=ta, trans_b=tb, alpha=0.5, beta=-2.0, C=C,
            form=form, route=route)
    got = C.cpu().numpy().astype(np.float64)
    if form == 2:
        low = np.tril(np.ones((m, n), bool))
        assert np.array_equal(got[~low], C0.astype(np.float64)[~low])  # untouched above the diagonal
        got, ref, scale = got[low], ref[low], scale[low]
    assert np.max(np.abs(got - ref) / scale) <= 4e-6


@pytest.mark.parametrize("route", [1, 0])
@pytest.mark.parametrize("form", [0, 2])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("m,n,k", [(128, 64, 64), (130, 70, 300), (300, 257, 1000), (1000, 129, 64), (64, 40, 30)])
def test_sgemm_fp32_accurate(route, form, ta, tb, m, n, k):
    """Plain (form 0) and lower-triangular-C (form 2) FP32 products."""
    _sgemm_case(route, form, ta, tb, m, n, k)


@pytest.mark.parametrize("route", [1, 0])
@pytest.mark.parametrize("tb", [False, True])
@pytest.mark.parametrize("m,n", [(128, 64), (256, 96), (520, 130), (1000, 257), (64, 40)])
def test_sgemm_fp32_symmetric_a(route, tb, m, n):
    """Symmetric A read from its lower triangle (form 1, the SYMM of the band
    reduction): square and untransposed by definition, garbage above the
    diagonal that must not be read."""
    _sgemm_case(route, 1, False, tb, m, n, m)


@pytest.mark.parametrize("slices,tol", [(7, 1e-13), (5, 1e-10), (3, 1e-5)])
def test_frac_apply_tensor_slices(square_small, slices, tol):
    """frac_apply with its products as BF16 slices on the tensor cores,
    against the oracle's FP64 apply: 7 slices reach FP64 level, fewer slices
    lose about 8 bits each."""
    F = _F()
    p, A, lam, V = square_small
    U_o = O.frac_apply(V, lam, p.F, p.pair_f, p.pair_alpha)
    ctx = F.Context()
    ctx.set_apply_slices(slices)
    U = F.frac_apply(_colmajor(V), _cuda(lam), _colmajor(p.F), p.pair_f, p.pair_alpha, ctx=ctx).cpu().numpy()
    for j in range(U_o.shape[1]):
        assert np.linalg.norm(U[:, j] - U_o[:, j]) <= tol * np.linalg.norm(U_o[:, j])


def test_binding_refuses_bad_shapes_and_devices():
    """Shapes and devices the library cannot take are refused before any
    call: a non-square V or A, forcings with the wrong row count or on the
    host, an expanded (overlapping) output; a transposed or expanded input is
    copied into a column-major one instead."""
    import paper_1911_11906_gb300 as F
    n = 6
    V = torch.eye(n, dtype=torch.float64, device="cuda")
    lam = torch.ones(n, dtype=torch.float64, device="cuda")
    Fd = torch.ones(n, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        F.frac_apply(V[:, :4], lam, Fd, [0], [1.0])
    with pytest.raises(ValueError):
        F.frac_apply(V, lam, Fd[:4], [0], [1.0])
    with pytest.raises(TypeError):
        F.frac_apply(V, lam, Fd.cpu(), [0], [1.0])
    with pytest.raises(ValueError):
        F.eig_full(torch.ones(n, n - 1, dtype=torch.float64, device="cuda"))
    out = torch.empty(n, 1, dtype=torch.float64, device="cuda").expand(n, 2)
    with pytest.raises(TypeError):
        F.frac_apply(V, lam, Fd, [0, 1], [1.0, 1.0], out=out)
    # an expanded input is read through a column-major copy: alpha = 0 returns it
    col = torch.arange(n, dtype=torch.float64, device="cuda").unsqueeze(1).expand(n, 2)
    U = F.frac_apply(V, lam, col, [0, 1], [0.0, 0.0])
    assert torch.equal(U, col)
