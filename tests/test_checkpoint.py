"""Checkpoint of a decomposition (host-side file I/O of the library; no
GPU): bit-exact round trips, the documented little-endian layout, the grid
hash, and every failure a damaged or foreign file must report."""
import ctypes
import os
import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1911_11906_gb300 as F  # noqa: E402
from paper_1911_11906_gb300 import _binding as B  # noqa: E402


def _fnv1a64(data: bytes) -> int:
    h = 14695981039346656037
    for b in data:
        h = ((h ^ b) * 1099511628211) % (1 << 64)
    return h


def _problem(n=29, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n), np.asfortranarray(rng.standard_normal((n, n)))


def test_round_trip_is_bit_exact(tmp_path):
    lam, V = _problem()
    mask = (np.random.default_rng(1).random((5, 8)) < 0.8).astype(np.uint8)
    path = str(tmp_path / "a.fraclap")
    F.save_decomposition(path, lam, V, mask=mask, h=0.125)
    l2, V2 = F.load_decomposition(path, mask=mask, h=0.125, device="cpu")
    assert np.array_equal(l2.numpy(), lam) and np.array_equal(V2.numpy(), V)
    assert V2.stride() == (1, lam.size)  # column-major
    # no leftover temporary file
    assert sorted(os.listdir(tmp_path)) == ["a.fraclap"]


def test_file_layout(tmp_path):
    lam, V = _problem(n=5)
    mask = np.ones((2, 3, 4), np.uint8)
    path = str(tmp_path / "b.fraclap")
    F.save_decomposition(path, lam, V, mask=mask, h=0.2)
    raw = open(path, "rb").read()
    n = 5
    assert len(raw) == 68 + 8 * n + 8 * n * n + 8
    magic, ver, dim, nn, e0, e1, e2, h, mh, res = struct.unpack("<8sIiqqqqdQI", raw[:68])
    assert (magic, ver, dim, nn, (e0, e1, e2), h, res) == (b"FRACLAPD", 1, 3, 5, (4, 3, 2), 0.2, 0)
    assert mh == F.mask_hash(mask, 0.2)
    assert struct.unpack("<5d", raw[68:108]) == tuple(lam)
    assert np.array_equal(np.frombuffer(raw[108:108 + 8 * n * n], "<f8").reshape(n, n, order="F"), V)
    assert struct.unpack("<Q", raw[-8:])[0] == _fnv1a64(raw[:-8])


def test_mask_hash_definition_and_sensitivity():
    mask = (np.random.default_rng(3).random((7, 6)) < 0.5).astype(np.uint8)
    h = 1.0 / 9.0
    data = struct.pack("<Iqqqd", 2, 6, 7, 1, h) + bytes(mask.reshape(-1))
    assert F.mask_hash(mask, h) == _fnv1a64(data)
    assert F.mask_hash(mask * 3, h) == F.mask_hash(mask, h)  # nonzero reads as 1
    flipped = mask.copy()
    flipped[2, 4] ^= 1
    assert F.mask_hash(flipped, h) != F.mask_hash(mask, h)
    assert F.mask_hash(mask, np.nextafter(h, 1.0)) != F.mask_hash(mask, h)  # one ulp of h
    assert F.mask_hash(mask.reshape(1, 7, 6), h) != F.mask_hash(mask, h)
    assert F.mask_hash(torch.from_numpy(mask), h) == F.mask_hash(mask, h)


def test_strided_buffers_and_header_query(tmp_path):
    lib = B.load_library()
    n = 11
    lam, V = _problem(n, seed=5)
    big = np.zeros((n + 4, n), order="F")
    big[:n] = V
    ext = np.array([3, 4, 1], np.int64)
    path = str(tmp_path / "c.fraclap").encode()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    assert lib.fraclap_save_decomposition(path, n, p(lam), p(big), n + 4, 2, p(ext), 0.25, 77) == 0
    nn, dim, h, mh = ctypes.c_int64(0), ctypes.c_int(0), ctypes.c_double(0), ctypes.c_uint64(0)
    eo = np.zeros(3, np.int64)
    rc = lib.fraclap_load_decomposition(path, ctypes.byref(nn), ctypes.byref(dim), p(eo), ctypes.byref(h),
                                        ctypes.byref(mh), None, None, 0, 0)
    assert rc == 0 and (nn.value, dim.value, h.value, mh.value) == (n, 2, 0.25, 77)
    assert eo.tolist() == [3, 4, 1]
    l2 = np.empty(n)
    V2 = np.full((n + 2, n), 7.0, order="F")
    assert lib.fraclap_load_decomposition(path, None, None, None, None, None, p(l2), p(V2), n + 2, 77) == 0
    assert np.array_equal(l2, lam) and np.array_equal(V2[:n], V) and np.all(V2[n:] == 7.0)
    assert lib.fraclap_load_decomposition(path, None, None, None, None, None, p(l2), p(V2), n - 1, 0) == -1
    assert lib.fraclap_load_decomposition(path, None, None, None, None, None, None, None, 0, 78) == -1


def test_damaged_and_foreign_files(tmp_path):
    lam, V = _problem()
    path = str(tmp_path / "d.fraclap")
    F.save_decomposition(path, lam, V)
    raw = bytearray(open(path, "rb").read())

    def load_bytes(data, name):
        q = str(tmp_path / name)
        open(q, "wb").write(bytes(data))
        with pytest.raises(F.FraclapError) as ei:
            F.load_decomposition(q, device="cpu")
        return ei.value.code

    flipped = bytearray(raw)
    flipped[200] ^= 0x10
    assert load_bytes(flipped, "flip") == -8          # checksum
    assert load_bytes(raw[:-9], "short") == -8        # truncated
    assert load_bytes(raw + b"x", "long") == -8       # trailing bytes
    bad = bytearray(raw)
    bad[0:8] = b"NOTMAGIC"
    assert load_bytes(bad, "magic") == -8
    ver = bytearray(raw)
    ver[8] = 2
    assert load_bytes(ver, "version") == -8
    with pytest.raises(F.FraclapError) as ei:
        F.load_decomposition(str(tmp_path / "missing"), device="cpu")
    assert ei.value.code == -8
    # a file of another grid
    mask = np.ones((3, 3), np.uint8)
    F.save_decomposition(path, lam, V, mask=mask, h=0.25)
    other = mask.copy()
    other[1, 1] = 0
    with pytest.raises(F.FraclapError) as ei:
        F.load_decomposition(path, mask=other, h=0.25, device="cpu")
    assert ei.value.code == -1
    # a save that cannot be written leaves nothing behind
    with pytest.raises(F.FraclapError) as ei:
        F.save_decomposition(str(tmp_path / "no_dir" / "x"), lam, V)
    assert ei.value.code == -8 and not (tmp_path / "no_dir").exists()


def test_empty_decomposition(tmp_path):
    path = str(tmp_path / "e.fraclap")
    F.save_decomposition(path, np.zeros(0), np.zeros((0, 0)))
    lam, V = F.load_decomposition(path, device="cpu")
    assert lam.shape == (0,) and V.shape == (0, 0)
    assert os.path.getsize(path) == 68 + 8
