"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/soar.h declares; host-side argument checks reject bad input
before any device work (no compute calls here)."""
import ctypes as ct
import struct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def _declared():
    names = []
    for h in HEADERS:
        src = open(h).read()
        names += re.findall(r"^SOAR_API\s+[\w\s\*]+?\b(soar_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_00774_gb300 import build
    path = build.build()
    return ct.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("soar_train_centroids", "soar_assign", "soar_index_build", "soar_search",
                     "soar_index_free", "soar_last_error", "soar_exact_mips", "soar_select_partitions"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_names_match_the_abi():
    from paper_2404_00774_gb300 import binding
    for name in binding._SIGS:
        assert name in _declared()
    for name in _declared():
        if name in ("soar_last_error", "soar_version", "soar_index_get_info", "soar_index_free"):
            continue                      # used inside the binding's helpers and Index class
        if name.startswith("soar_server_"):
            assert hasattr(binding, "Server")  # the serving loop is wrapped by binding.Server
            continue
        assert hasattr(binding, name), f"binding lacks {name}"


def test_version_and_error_string_without_gpu(lib):
    lib.soar_version.restype = ct.c_char_p
    assert b"sm_103a" in lib.soar_version()
    lib.soar_last_error.restype = ct.c_char_p
    assert lib.soar_last_error() == b""


def test_invalid_arguments_rejected_on_host(lib):
    # null pointers and bad sizes fail with SOAR_EINVAL before touching a device
    lib.soar_last_error.restype = ct.c_char_p
    f = lib.soar_assign
    f.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_int32, ct.c_void_p, ct.c_int32, ct.c_float,
                  ct.c_int32, ct.c_void_p, ct.c_void_p]
    f.restype = ct.c_int32
    assert f(None, 0, 10, 4, None, 4, 1.0, 1, None, None) == 1
    assert b"null pointer" in lib.soar_last_error()
    dummy = ct.c_void_p(16)
    assert f(dummy, 0, 10, 4, dummy, 4, float("nan"), 1, dummy, None) == 1
    assert b"lambda" in lib.soar_last_error()
    assert f(dummy, 0, 10, 4, dummy, 1, 1.0, 1, dummy, None) == 1        # c < 1 + spills
    assert f(dummy, 0, 10, 4, dummy, 8, 1.0, 5, dummy, None) == 1        # spills > 4
    assert f(dummy, 7, 10, 4, dummy, 8, 1.0, 1, dummy, None) == 1        # unknown dtype
    s = lib.soar_search
    s.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_int32, ct.c_int32, ct.c_void_p,
                  ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_void_p]
    s.restype = ct.c_int32
    assert s(None, dummy, 0, 1, 10, 4, None, 0, dummy, dummy, None) == 1


def test_index_load_rejects_a_foreign_file_before_any_device_work(lib, tmp_path):
    # the header is checked on the host: no GPU is needed to reject the file
    bad = tmp_path / "not_an_index.bin"
    bad.write_bytes(b"definitely not a SOAR index file" * 4)
    lib.soar_index_load.argtypes = [ct.c_char_p, ct.POINTER(ct.c_void_p), ct.c_void_p]
    lib.soar_index_load.restype = ct.c_int
    lib.soar_last_error.restype = ct.c_char_p
    out = ct.c_void_p()
    assert lib.soar_index_load(str(bad).encode(), ct.byref(out), None) == 1      # SOAR_EINVAL
    assert b"not a SOAR index" in lib.soar_last_error()
    assert lib.soar_index_load(str(tmp_path / "missing.bin").encode(), ct.byref(out), None) == 1
    assert out.value is None


# ---------------------------------------------- index files checked on the host

_HDR = struct.Struct("<8sII5q12i17Q")      # magic, version, header bytes, 5 int64, 12 int32, 17 section sizes


def _index_file(path, *, version=2, rows=None, sections=None, extra=b"", cut=0):
    """A file shaped like a saved fp32 index of n = 10 points (d = 4, c = 2,
    one spill) holding only the required sections: offsets, ids, vectors,
    centroids, sized as the format defines them."""
    n, d, c, spills = 10, 4, 2, 1
    rows = n * (1 + spills) if rows is None else rows
    sizes = [0] * 17
    sizes[0] = 8 * (c + 1)            # offsets int64 [c + 1]
    sizes[1] = 4 * rows               # ids int32 [rows]
    sizes[2] = 4 * rows * d           # vectors fp32 [rows][row_stride = d]
    sizes[5] = 4 * c * d              # centroids fp32 [c][d]
    for i, b in (sections or {}).items():
        sizes[i] = b
    hdr = _HDR.pack(b"SOARIDX1", version, _HDR.size, n, rows, 12, 0, 0,
                    d, c, spills, 0, 0, d, 0, 8, 8, 1, 0, 0, *sizes)
    body = bytes(sum(sizes))
    data = hdr + body + extra
    path.write_bytes(data[:len(data) - cut])
    return path


def _load(lib, path):
    lib.soar_index_load.argtypes = [ct.c_char_p, ct.POINTER(ct.c_void_p), ct.c_void_p]
    lib.soar_index_load.restype = ct.c_int
    lib.soar_last_error.restype = ct.c_char_p
    lib.soar_index_free.argtypes = [ct.c_void_p]
    out = ct.c_void_p()
    st = lib.soar_index_load(str(path).encode(), ct.byref(out), None)
    if st == 0:                       # only where a GPU took the arrays
        lib.soar_index_free(out)
    else:
        assert out.value is None
    return st, lib.soar_last_error()


def test_index_file_checks_run_on_the_host(lib, tmp_path):
    assert _HDR.size == 240
    # an exact file passes every host check: with no GPU the first device
    # allocation is what fails
    st, msg = _load(lib, _index_file(tmp_path / "ok.bin"))
    assert st != 1, msg
    for kwargs, code, text in [
        (dict(cut=1), 1, b"truncated"),
        (dict(cut=200), 1, b"truncated"),
        (dict(extra=b"\0"), 1, b"trailing bytes"),
        (dict(sections={1: 76}), 1, b"section 1 has the wrong size"),
        (dict(sections={5: 0}), 1, b"required section is missing"),
        (dict(sections={2: 0}), 1, b"required section is missing"),
        (dict(rows=21), 1, b"out of range"),
        (dict(version=3), 5, b"unsupported format version"),
    ]:
        st, msg = _load(lib, _index_file(tmp_path / "bad.bin", **kwargs))
        assert st == code and text in msg, (kwargs, st, msg)
