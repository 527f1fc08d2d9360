"""The C ABI library builds for sm_103a, loads, and exports every declared entry
point; the Python binding carries the same names; the product never touches
the oracle (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "benelux.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"\b(bnx_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_01099_gb300 import benelux as B

    return B.lib()


def test_header_declares_the_boundary_calls():
    names = declared()
    for n in ("bnx_create", "bnx_destroy", "bnx_search", "bnx_rad_segment", "bnx_search_hash", "bnx_batch",
              "bnx_server_submit", "bnx_server_poll", "bnx_strerror", "bnx_autotune"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_has_same_names():
    from paper_2506_01099_gb300 import benelux as B

    for name in declared():
        assert callable(getattr(B, name)), name


def test_strerror(lib):
    from paper_2506_01099_gb300 import benelux as B

    assert B.bnx_strerror(0) == "ok"
    assert B.bnx_strerror(B.BNX_E_TRUNCATED) == "output truncated"
    assert B.bnx_strerror(999) == "unknown error"


def test_create_rejects_bad_arguments(lib):
    from paper_2506_01099_gb300 import benelux as B

    h = ctypes.c_void_p()
    assert lib.bnx_create(None, 0, 1 << 20, None, None) == B.BNX_E_ARG
    assert lib.bnx_create(ctypes.byref(h), 0, (1 << 42) + 1, None, None) == B.BNX_E_ARG
    assert lib.bnx_create(ctypes.byref(h), -1, 1 << 20, None, None) == B.BNX_E_ARG
    assert not h.value


def test_null_context_is_an_argument_error(lib):
    from paper_2506_01099_gb300 import benelux as B

    n = ctypes.c_size_t()
    assert lib.bnx_search(None, 1, 10, 3, None, 0, ctypes.byref(n)) == B.BNX_E_ARG
    assert lib.bnx_server_stop(None) == B.BNX_E_ARG
    lib.bnx_destroy(None)  # accepted


def test_no_gpu_means_loud_failure(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2506_01099_gb300 import benelux as B

    with pytest.raises(B.BnxError):
        B.bnx_create(0, 1 << 20)


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2506_01099_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "benelux_oracle" not in text and "liboracle" not in text, f


def test_ncu_record_follows_the_code_not_the_comments(tmp_path):
    """The benchmark keys its committed ncu record (traffic, instructions per integer) by a
    hash of the sieve's code: comments and blank lines do not change it, code does."""
    import sys

    sys.path.insert(0, ROOT)
    import bench

    src = tmp_path / "k.cu"
    src.write_text("int f(int x) {\n    return x + 1;  // one more\n}\n")
    h = bench.code_sha256(str(src))
    src.write_text("// a kernel\nint f(int x) {\n\n    return x + 1;  // the successor\n}\n")
    assert bench.code_sha256(str(src)) == h
    src.write_text("int f(int x) {\n    return x + 2;\n}\n")
    assert bench.code_sha256(str(src)) != h
    assert bench.sieve_record(3) is not None  # the committed capture matches the current kernel


def test_same_rad_rejects_bad_arguments_before_the_device(lib):
    """bnx_same_rad checks its arguments on the host first (no device is touched)."""
    from paper_2506_01099_gb300 import benelux as B

    P = ctypes.POINTER(ctypes.c_uint64)
    x = (ctypes.c_uint64 * 2)(6, 0)
    y = (ctypes.c_uint64 * 2)(12, 5)
    out = (ctypes.c_uint8 * 2)()
    assert lib.bnx_same_rad(x, y, 0, out) == B.BNX_OK  # nothing to do
    assert lib.bnx_same_rad(x, y, 2, out) == B.BNX_E_ARG  # a zero value
    assert lib.bnx_same_rad(None, y, 1, out) == B.BNX_E_ARG
    assert lib.bnx_same_rad(x, y, 1, None) == B.BNX_E_ARG
    assert lib.bnx_same_rad(ctypes.cast(x, P), ctypes.cast(y, P), (1 << 24) + 1, out) == B.BNX_E_ARG
