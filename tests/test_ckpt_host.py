"""Checkpoint files on the host (no GPU): dcd_load and dcd_mlp_load reject a
file that is missing, foreign or damaged before they create anything on the
device.  Each file here is written from the layout that include/dcd.h states:
a 256-byte header, 8-byte-padded sections, a 64-bit FNV-1a checksum over the
8-byte little-endian words before it."""
import ctypes
import struct

import numpy as np
import pytest


@pytest.fixture(scope="module")
def libdcd():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1904_08553_gb300 import dcd

    return dcd


def fnv_words(data: bytes) -> int:
    assert len(data) % 8 == 0
    h = 1469598103934665603
    for (x,) in struct.iter_unpack("<Q", data):
        h = ((h ^ x) * 1099511628211) & ((1 << 64) - 1)
    return h


def header(n=4, nnz=2, t=1, mode=2, nb=1, version=1, flags=0, magic=b"DCDCKPT1"):
    cfg = struct.pack("<4i12i", mode, 500, 64, 1_000_000, *([0] * 12))
    var = struct.pack("<12i", 8, *([0] * 11))
    hi = struct.pack("<12q", -1, *([0] * 11))
    h = magic + struct.pack("<IIqqqii", version, flags, n, nnz, t, mode, nb) + cfg + var + hi
    assert len(h) == 256
    return h


def load_rc(libdcd, path):
    h = ctypes.c_void_p()
    return libdcd.lib().dcd_load(str(path).encode(), None, ctypes.byref(h))


def test_fnv_reference_value():
    # FNV-1a 64 of one zero word is a single multiply of the offset basis
    assert fnv_words(bytes(8)) == (1469598103934665603 * 1099511628211) % (1 << 64)


def test_missing_file_is_an_io_error(libdcd, tmp_path):
    assert load_rc(libdcd, tmp_path / "absent.ckpt") == libdcd.DCD_EIO
    h = ctypes.c_void_p()
    assert libdcd.lib().dcd_mlp_load(str(tmp_path / "absent.mlp").encode(), None,
                                     ctypes.byref(h)) == libdcd.DCD_EIO


def test_null_arguments(libdcd):
    L = libdcd.lib()
    h = ctypes.c_void_p()
    assert L.dcd_save(None, b"x") == libdcd.DCD_EINVAL
    assert L.dcd_load(None, None, ctypes.byref(h)) == libdcd.DCD_EINVAL
    assert L.dcd_load(b"x", None, None) == libdcd.DCD_EINVAL
    assert L.dcd_mlp_save(None, b"x") == libdcd.DCD_EINVAL
    assert L.dcd_get_state(None, None, None, None) == libdcd.DCD_EINVAL
    assert libdcd.DCD_EIO == -7 and b"file" in L.dcd_strerror(libdcd.DCD_EIO)


@pytest.mark.parametrize("kw", [
    dict(magic=b"DCDCKPT2"),       # another format
    dict(version=2),               # another version
    dict(flags=2),                 # unknown flag
    dict(n=0),                     # no vertices
    dict(n=1 << 31),               # above the id range
    dict(nnz=-2),
    dict(nnz=3),                   # odd: an edge stored in one row only
    dict(n=4, nnz=14),             # more entries than n (n - 1)
    dict(t=-1),
    dict(mode=5),                  # unknown mode
    dict(nb=0), dict(nb=13),       # plan size outside 1..12
])
def test_bad_header_is_rejected_on_the_host(libdcd, tmp_path, kw):
    p = tmp_path / "bad.ckpt"
    p.write_bytes(header(**kw) + bytes(64))
    assert load_rc(libdcd, p) == libdcd.DCD_EINVAL


def test_truncated_header_is_rejected(libdcd, tmp_path):
    p = tmp_path / "short.ckpt"
    p.write_bytes(header()[:200])
    assert load_rc(libdcd, p) == libdcd.DCD_EINVAL
    p.write_bytes(b"")
    assert load_rc(libdcd, p) == libdcd.DCD_EINVAL


def mlp_file(params: np.ndarray, checksum=None) -> bytes:
    body = b"DCDMLP01" + struct.pack("<II", 1, 5057) + np.append(params, np.float32(0)).astype("<f4").tobytes()
    return body + struct.pack("<Q", fnv_words(body) if checksum is None else checksum)


@pytest.mark.parametrize("case", ["magic", "checksum", "nan", "inf", "size", "trailing"])
def test_bad_network_file_is_rejected_on_the_host(libdcd, tmp_path, case):
    params = np.linspace(-1, 1, 5057).astype(np.float32)
    if case == "nan":
        params[100] = np.nan
    if case == "inf":
        params[7] = np.inf
    data = mlp_file(params)
    if case == "magic":
        data = b"DCDMLP02" + data[8:]
    if case == "checksum":
        data = data[:-8] + struct.pack("<Q", fnv_words(data[:-8]) ^ 1)
    if case == "size":
        data = data[:-12] + data[-8:]
    if case == "trailing":
        data = data + b"\0"
    p = tmp_path / "bad.mlp"
    p.write_bytes(data)
    h = ctypes.c_void_p()
    assert libdcd.lib().dcd_mlp_load(str(p).encode(), None, ctypes.byref(h)) == libdcd.DCD_EINVAL
