"""Host-side checks that need no GPU: the C-ABI library loads and exports
every entry point that include/fraclap.h declares, the binding's table
matches the header, host-only entry points (error strings, workspace sizes,
argument checks that return before any CUDA call) behave as documented, the
binding refuses to run without the CUDA library, the seeded workloads have
their stated sizes, and the benchmark's multi-rank reduction works over two
gloo ranks."""
import ctypes
import os
import re
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fraclap.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return re.findall(r"^[ \t]*(?:const[ \t]+)?[A-Za-z_]\w*(?:[ \t]+[A-Za-z_]\w*)*[ \t*]+\**([A-Za-z_]\w*)\s*\(",
                      src, flags=re.M)


@pytest.fixture(scope="module")
def lib():
    from paper_1911_11906_gb300 import build
    path = build.build()  # incremental: a no-op when the library is current
    L = ctypes.CDLL(path)
    return L


def test_header_declares_the_boundary():
    names = _declared()
    assert len(names) == len(set(names))
    for core in ("fraclap_create", "fd_assemble", "eig_full", "eig_full_mixed", "frac_apply",
                 "frac_diffusion", "frac_apply_noalloc", "fraclap_solve_batched"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_table_matches_header():
    from paper_1911_11906_gb300 import _binding
    declared = set(_declared())
    assert set(_binding.SIGNATURES) == declared


def test_error_strings(lib):
    lib.fraclap_strerror.restype = ctypes.c_char_p
    seen = set()
    for code in range(0, -9, -1):
        s = lib.fraclap_strerror(code)
        assert s and s not in seen
        seen.add(s)
    assert lib.fraclap_strerror(-1000)  # unknown codes still get a string


def test_workspace_sizes_are_host_arithmetic(lib):
    f = lib.fraclap_apply_workspace_bytes
    f.restype, f.argtypes = ctypes.c_size_t, [ctypes.c_int64] * 3
    # V^T F (n x m) and the coefficients (n x k), each rounded up to 256 bytes, plus slack
    for n, m, k in [(1, 1, 1), (100, 3, 7), (8810, 16, 128)]:
        want = -(-8 * n * m // 256) * 256 + -(-8 * n * k // 256) * 256 + 512
        assert f(n, m, k) == want
    assert f(-1, 1, 1) == 0
    g = lib.fraclap_apply_workspace_bytes_ctx
    g.restype, g.argtypes = ctypes.c_size_t, [ctypes.c_void_p] + [ctypes.c_int64] * 3
    assert g(None, 100, 3, 7) == f(100, 3, 7)


def test_noalloc_argument_checks_return_before_any_launch(lib):
    """frac_apply_noalloc validates sizes, pointers and the scratch bound on
    the host; none of these calls touches a device."""
    fn = lib.frac_apply_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                   ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    fake = ctypes.c_void_p(4096)  # never dereferenced: every call below returns first
    assert fn(fake, 10, fake, -1, fake, 10, 1, fake, fake, 1, fake, 10, None, None) == -1
    assert fn(fake, 10, fake, 0, fake, 10, 1, fake, fake, 1, fake, 10, None, None) == 0
    assert fn(fake, 10, fake, 10, fake, 10, 1, fake, fake, 0, fake, 10, None, None) == 0
    assert fn(None, 10, fake, 10, fake, 10, 1, fake, fake, 1, fake, 10, None, None) == -1
    assert fn(fake, 9, fake, 10, fake, 10, 1, fake, fake, 1, fake, 10, None, None) == -1
    big = 1 << 20
    assert fn(fake, big, fake, big, fake, big, 1, fake, fake, 4, fake, big, None, None) == -7


def test_context_calls_reject_null_context(lib):
    for name, args in [("fraclap_set_apply_slices", (None, 3)), ("fraclap_set_profiling", (None, 1))]:
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        assert fn(*args) != 0


def test_create_without_a_device_fails_cleanly():
    """Without a GPU, fraclap_create returns FRACLAP_ERR_CUDA (in a child
    process, so a driver-less import cannot disturb this one)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    code = ("import ctypes; from paper_1911_11906_gb300 import build; L = ctypes.CDLL(build.LIB); "
            "p = ctypes.c_void_p(); print(L.fraclap_create(ctypes.byref(p), None))")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "-6"


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    pytest.importorskip("torch")
    from paper_1911_11906_gb300 import _binding
    monkeypatch.setattr(_binding, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_binding, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _binding.load_library()


def test_workload_sizes():
    from paper_1911_11906_gb300 import inputs as I
    p = I.ellipse_problem()
    assert (p.n, p.F.shape[1], len(p.pair_f)) == (8810, 16, 128)
    q = I.ellipse_problem()
    assert np.array_equal(p.mask, q.mask) and np.array_equal(p.F, q.F)  # seeded
    s = I.square_problem(48)
    assert s.n == 2304 and abs(s.h - 1 / 49) < 1e-15
    b = I.batched_problems(256)
    assert len(b) == 256 and min(x.n for x in b) >= 1 and max(x.n for x in b) <= 64 * 64
    assert all(len(x.pair_f) == 32 for x in b)


def test_bench_work_counts():
    sys.path.insert(0, ROOT)
    import bench
    # 7-bit slices: 40, 48, 56 bits -> 6, 7, 8 slices; the last allowed iteration is full
    assert bench.refine_slice_counts(3, 6) == [6, 7, 8]
    assert bench.refine_slice_counts(1, 1) == [8]
    assert bench.ozaki_bf16_flops(4, 2) == 2.0 * 3 * 4 * 10
    # q2: reflectors of length min(b, n - r0) at r0 = s + 1, s + 1 + b, ...; brute force for a tiny case
    n, b = 7, 3
    tot = sum(min(b, n - r0) for s in range(n - 1) for r0 in range(s + 1, n, b) if min(b, n - r0) > 1)
    assert bench.q2_flops(n, b) == 4.0 * tot * n
    assert bench.whole_job_rate(128, 4, 500.0) == 1024.0
    # the apply's two sliced products V^T F (n x m) and V C (n x k), inner dimension n:
    # 2 flops per digit pair p + q < d per output element per k; d = ceil(8 s / 7) 7-bit digits
    n, m, k, s = 5, 3, 4, 6
    d = -(-8 * s // 7)
    pairs = sum(1 for p in range(d) for q in range(d) if p + q < d)
    assert bench.apply_slice_flops(n, m, k, s) == 2.0 * pairs * n * n * (m + k)
    assert bench.apply_slice_flops(n, m, k, s, digit_bits=8) == 2.0 * (s * (s + 1) // 2) * n * n * (m + k)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks([10.0 + rank, 5.0 - rank], world)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(" ".join(str(v) for v in got))
    finally:
        dist.destroy_process_group()


def test_bench_max_over_two_gloo_ranks(tmp_path):
    """The multi-rank timing reduction of the benchmark (slowest rank wins)
    over two gloo ranks on the host."""
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        vals = [float(v) for v in open(tmp_path / f"r{r}.txt").read().split()]
        assert vals == [11.0, 5.0]
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]


def test_reference_arm_other_ranks_do_nothing(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 1
    bench.run_reference(A(), rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_bench_jsonl_records():
    sys.path.insert(0, ROOT)
    import bench
    line = {"steps": 3, "config": {"workload": "w", "n": 10, "path": "mixed"},
            "roofline": {"frac": 0.4},
            "paths": {"fp64": {"ms_per_step": 2000.0, "solves_per_s": 64.0, "eig_s": 1.9,
                               "eig_tflops_credited_fp64": 0.5, "eig_frac_of_fp64_peak": 0.4,
                               "accuracy": {"orth_sampled_max": 1e-15}, "stage_ms": {"apply": 1.0}},
                      "mixed": {"ms_per_step": 500.0, "solves_per_s": 256.0, "eig_s": 0.45,
                                "accuracy": {"u_rel_l2_alpha2_vs_cg_max": 1e-14}}}}
    recs = bench.jsonl_records(line)
    assert [r["precision"] for r in recs] == ["fp64", "mixed"]
    assert recs[0]["seconds"] == 2.0 and recs[0]["err_orth"] == 1e-15 and "roofline" not in recs[0]
    assert recs[1]["roofline"] == {"frac": 0.4} and recs[1]["err_u_alpha2"] == 1e-14
    assert bench.jsonl_records({}) == []


def test_public_calls_refuse_host_tensors():
    """No CPU fallback: the compute entry points raise on host tensors (or,
    without a GPU, when the context cannot be created) instead of computing
    anything on the CPU."""
    torch = pytest.importorskip("torch")
    import paper_1911_11906_gb300 as F
    A = torch.eye(4, dtype=torch.float64)
    lam = torch.ones(4, dtype=torch.float64)
    Fm = torch.ones(4, 1, dtype=torch.float64)
    calls = [lambda: F.eig_full(A), lambda: F.frac_apply(A, lam, Fm, [0], [1.0]),
             lambda: F.frac_diffusion(A, lam, Fm, [0], [1.0], [0.1]), lambda: F.dgemm(A, A),
             lambda: F.fd_assemble(torch.ones(3, 3, dtype=torch.uint8), 0.25)]
    for call in calls:
        with pytest.raises((TypeError, F.FraclapError, RuntimeError)):
            call()


def test_binding_input_guards():
    """The binding's guards refuse host tensors, wrong dtypes, short buffers
    and row-major outputs before any pointer reaches the library."""
    torch = pytest.importorskip("torch")
    from paper_1911_11906_gb300 import _binding as B
    dev = torch.device("cuda", 0)
    for call in (lambda: B._dev(torch.ones(3), torch.float32, "x", dev),
                 lambda: B._dev(torch.ones(3, dtype=torch.int32), torch.float32, "x", dev),
                 lambda: B._out(torch.ones(3, 2, dtype=torch.float64), torch.float64, "out", dev, 3, 2),
                 lambda: B._ws(torch.empty(8, dtype=torch.uint8), dev)):
        with pytest.raises(TypeError):
            call()


def test_binding_layout_guard_refuses_overlapping_columns():
    """The layout the binding hands to the library must be column-major with
    non-overlapping columns: an expanded output (stride 0 along the columns)
    or a column stride below the row count would make the library write or
    read rows x cols elements through too little storage."""
    torch = pytest.importorskip("torch")
    from paper_1911_11906_gb300._binding import colmajor_layout_ok as ok
    n, k = 5, 3
    base = torch.empty(k, n, dtype=torch.float64).t()          # column-major n x k
    assert ok(tuple(base.shape), base.stride())
    expanded = torch.empty(n, 1, dtype=torch.float64).expand(n, k)
    assert expanded.stride() == (1, 0) and not ok(tuple(expanded.shape), expanded.stride())
    rowmajor = torch.empty(n, k, dtype=torch.float64)
    assert not ok(tuple(rowmajor.shape), rowmajor.stride())
    short = torch.empty(20, dtype=torch.float64).as_strided((n, k), (1, 2))  # columns overlap
    assert not ok(tuple(short.shape), short.stride())
    padded = torch.empty(k, n + 3, dtype=torch.float64).t()[:n]  # ld = n + 3 >= n
    assert ok(tuple(padded.shape), padded.stride())
    one_col = torch.empty(n, 1, dtype=torch.float64)           # a single column: any column stride
    assert ok(tuple(one_col.shape), one_col.stride())
    assert ok((1, k), (k, 1)) and ok((1, k), (1, 1))           # one row: columns one element apart
    assert not ok((1, k), (1, 0))                               # ... but not all the same element
