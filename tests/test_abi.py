"""CPU-side checks of the C ABI library (no kernel is launched here).

libhs.so must build for sm_103a, load, and export every function that
include/hs.h declares; the size queries must agree with the oracle's
parameter derivation; and the product package must not reach the oracle.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_23969_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"hs_keygen", "hs_sign_batch", "hs_verify_batch"} <= set(names)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_size_queries_match_oracle(lib, O):
    names = ("128f", "192f", "256f", "toy", "128s", "192s", "256s",
             "shake-128f", "shake-192f", "shake-256f", "shake-128s", "shake-192s", "shake-256s",
             "robust-128f", "robust-192f", "robust-256f")
    for pid, ps in enumerate(names):
        P = O.params(ps)
        for fn, want in (("hs_sig_bytes", P.sig_bytes), ("hs_pk_bytes", 2 * P.n),
                         ("hs_sk_bytes", 4 * P.n), ("hs_seed_bytes", 3 * P.n)):
            f = getattr(lib, fn)
            f.argtypes = [C.c_int]
            f.restype = C.c_size_t
            assert f(pid) == want, (fn, ps)
    lib.hs_sig_bytes.argtypes = [C.c_int]
    lib.hs_sig_bytes.restype = C.c_size_t
    assert lib.hs_sig_bytes(len(names)) == 0 and lib.hs_sig_bytes(-1) == 0
    lib.hs_sign_kernel_count.restype = C.c_int
    assert lib.hs_sign_kernel_count() == 7


def test_count_zero_and_bad_enum_need_no_gpu(lib):
    lib.hs_sign_batch.restype = C.c_int
    lib.hs_sign_batch.argtypes = [C.c_int, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_uint32, C.c_void_p, C.c_void_p]
    assert lib.hs_sign_batch(16, None, 1, None, None, None, 1, None, None) == 1     # HS_EINVAL
    assert lib.hs_sign_batch(0, None, 1, None, None, None, 0, None, None) == 0      # count 0: no-op
    lib.hs_last_error.restype = C.c_char_p
    assert b"parameter set" in lib.hs_last_error()


def test_product_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2512_23969_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), f
                assert "spx_oracle" not in text, f


def test_last_error_copy_fills_caller_buffer(lib):
    """hs_last_error_copy: the thread's last error text into the caller's
    buffer, truncated and NUL-terminated; NULL or empty buffers are refused."""
    lib.hs_set_chain_checkpoint.argtypes = [C.c_uint32]
    lib.hs_set_chain_checkpoint.restype = C.c_int
    lib.hs_last_error.restype = C.c_char_p
    lib.hs_last_error_copy.argtypes = [C.c_char_p, C.c_size_t]
    lib.hs_last_error_copy.restype = C.c_int
    assert lib.hs_set_chain_checkpoint(3) == 1                  # HS_EINVAL, sets the text
    full = lib.hs_last_error()
    assert b"stride" in full
    buf = C.create_string_buffer(b"\xff" * 256, 256)
    assert lib.hs_last_error_copy(buf, 256) == 0
    assert buf.value == full
    small = C.create_string_buffer(b"\xff" * 8, 8)
    assert lib.hs_last_error_copy(small, 8) == 0
    assert small.raw == full[:7] + b"\0"                        # 7 bytes and the terminator
    assert lib.hs_last_error_copy(None, 16) == 1
    assert lib.hs_last_error_copy(small, 0) == 1
    assert lib.hs_last_error() == full                          # a refused copy keeps the text
    assert lib.hs_set_chain_checkpoint(2) == 0                  # the default again
