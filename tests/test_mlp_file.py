"""Network parameter files through the C ABI with host buffers (no GPU).

The layout is the one include/bamg.h documents: "BAMGMLP1", the entry count
and the 32-bit FNV-1a hash of the entry bytes as little-endian uint32, then
the entries as little-endian binary32.  The tests write and parse that layout
in Python on their own, so the library is checked against the documented
format and not only against itself."""
import ctypes
import struct

import numpy as np
import pytest

NP = 9360


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    from paper_1402_4005_gb300 import _lib
    lib = _lib.lib()
    assert lib.bamg_mlp_num_params() == NP
    return lib


def fnv1a32(data: bytes) -> int:
    h = 2166136261
    for b in data:
        h = ((h ^ b) * 16777619) & 0xFFFFFFFF
    return h


def encode(w: np.ndarray, count=None, tag=b"BAMGMLP1", hash_fix=0) -> bytes:
    body = np.asarray(w, dtype="<f4").tobytes()
    n = len(w) if count is None else count
    return tag + struct.pack("<II", n, (fnv1a32(body) + hash_fix) & 0xFFFFFFFF) + body


def params(seed=3):
    return np.random.default_rng(seed).standard_normal(NP).astype(np.float32)


def _buf(w):
    return w.ctypes.data_as(ctypes.c_void_p)


def test_save_writes_the_documented_layout(L, tmp_path):
    w = params()
    path = tmp_path / "net.bin"
    assert L.bamg_mlp_save(str(path).encode(), _buf(w), 0, None) == 0
    raw = path.read_bytes()
    assert raw == encode(w)
    assert len(raw) == 16 + 4 * NP


def test_load_reads_a_file_written_from_the_layout(L, tmp_path):
    w = params(4)
    w[:4] = [0.0, -0.0, 1e-45, -3.4e38]         # signed zero, a subnormal, a large value: bits kept
    path = tmp_path / "net.bin"
    path.write_bytes(encode(w))
    out = np.full(NP, 7.0, np.float32)
    assert L.bamg_mlp_load(str(path).encode(), _buf(out), 0, None) == 0
    assert out.tobytes() == w.tobytes()


def test_round_trip_through_the_library(L, tmp_path):
    w = params(5)
    path = tmp_path / "rt.bin"
    assert L.bamg_mlp_save(str(path).encode(), _buf(w), 0, None) == 0
    out = np.zeros(NP, np.float32)
    assert L.bamg_mlp_load(str(path).encode(), _buf(out), 0, None) == 0
    assert np.array_equal(out.view(np.uint32), w.view(np.uint32))


@pytest.mark.parametrize("case", ["tag", "count", "truncated", "trailing", "hash", "flipped", "empty"])
def test_malformed_files_are_io_errors_and_leave_the_output(L, tmp_path, case):
    w = params(6)
    good = encode(w)
    bad = {
        "tag": encode(w, tag=b"BAMGMLP2"),
        "count": encode(w, count=NP - 1),
        "truncated": good[:-4],
        "trailing": good + b"\0",
        "hash": encode(w, hash_fix=1),
        "flipped": good[:100] + bytes([good[100] ^ 0x10]) + good[101:],
        "empty": b"",
    }[case]
    path = tmp_path / f"{case}.bin"
    path.write_bytes(bad)
    out = np.full(NP, 7.0, np.float32)
    assert L.bamg_mlp_load(str(path).encode(), _buf(out), 0, None) == 10      # BAMG_ERR_IO
    assert np.all(out == 7.0)
    assert L.bamg_last_error()


def test_missing_file_null_arguments_and_non_finite_entries(L, tmp_path):
    out = np.full(NP, 7.0, np.float32)
    assert L.bamg_mlp_load(str(tmp_path / "none.bin").encode(), _buf(out), 0, None) == 10
    assert L.bamg_mlp_load(None, _buf(out), 0, None) == 1
    assert L.bamg_mlp_load(b"x", None, 0, None) == 1
    assert L.bamg_mlp_save(None, _buf(out), 0, None) == 1
    # an unwritable path (a directory) is an IO error
    assert L.bamg_mlp_save(str(tmp_path).encode(), _buf(out), 0, None) == 10
    w = params(7)
    w[123] = np.nan
    assert L.bamg_mlp_save(str(tmp_path / "nan.bin").encode(), _buf(w), 0, None) == 7     # BAMG_ERR_NUMERIC
    assert not (tmp_path / "nan.bin").exists()
    w[123] = np.inf
    (tmp_path / "inf.bin").write_bytes(encode(w))
    assert L.bamg_mlp_load(str(tmp_path / "inf.bin").encode(), _buf(out), 0, None) == 7
    assert np.all(out == 7.0)


def test_python_binding_on_cpu_tensors(L, tmp_path):
    import torch
    from paper_1402_4005_gb300 import bamg_mlp_load, bamg_mlp_save
    from paper_1402_4005_gb300._lib import BamgError
    t = torch.from_numpy(params(8))
    path = tmp_path / "py.bin"
    bamg_mlp_save(t, path)
    back = bamg_mlp_load(path, device="cpu")
    assert torch.equal(back, t)
    with pytest.raises(ValueError):
        bamg_mlp_save(t[:-1], path)
    with pytest.raises(BamgError):
        bamg_mlp_load(tmp_path / "missing.bin", device="cpu")
