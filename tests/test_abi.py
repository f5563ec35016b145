"""The C ABI library builds, loads and exports every function include/ck.h
declares; argument checks that need no GPU answer as documented."""
import ctypes
import os
import re

from paper_1605_05236_gb300 import build as ckbuild
from paper_1605_05236_gb300 import ck

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ck.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+(ck_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    path = ckbuild.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    names = declared_functions()
    assert "ck_insert_batch" in names and "ck_lookup_batch" in names and "ck_delete_batch" in names
    for n in names:
        assert hasattr(L, n), "libck.so does not export " + n


def test_required_bytes_shapes():
    assert ck.required_bytes(1 << 14, 4, 2, ck.RANDOM) >= (1 << 14) * 4 * 8 + (1 << 14) * 4
    assert ck.required_bytes(1 << 14, 8, 2, ck.QUEUE | ck.GHOST) > 0
    assert ck.required_bytes(1 << 14, 1, 3, ck.RATTLE) > 0
    assert ck.required_bytes(1 << 14, 1, 4, ck.RANDOM) > 0
    # search policies provision per-searcher scratch
    assert ck.required_bytes(1 << 14, 4, 2, ck.SORTED) > ck.required_bytes(1 << 14, 4, 2, ck.RANDOM)
    # invalid shapes and mixes
    for args in ((1 << 14, 2, 2, ck.RANDOM), (1 << 14, 4, 3, ck.RANDOM), (1 << 14, 1, 4, ck.QUEUE),
                 (1 << 14, 1, 3, ck.RANDOM | ck.GHOST), (1 << 14, 4, 2, ck.RATTLE), (1, 4, 2, ck.RANDOM),
                 (1 << 32, 4, 2, ck.RANDOM), (1 << 14, 4, 2, 7), (2, 1, 3, ck.RATTLE)):
        assert ck.required_bytes(*args) == 0, args


def test_invalid_arguments_need_no_gpu():
    L = ck.load()
    h = ctypes.c_void_p()
    assert L.ck_create(ctypes.byref(h), 1 << 10, 5, 2, 0, 0) == ck.EINVAL
    assert L.ck_create(None, 1 << 10, 4, 2, 0, 0) == ck.EINVAL
    assert L.ck_create_on(ctypes.byref(h), None, 0, 1 << 10, 4, 2, 0, 0, None) == ck.EINVAL
    # misaligned caller buffer
    assert L.ck_create_on(ctypes.byref(h), ctypes.c_void_p(0x1001), 1 << 20, 1 << 10, 4, 2, 0, 0, None) == ck.EINVAL
    assert L.ck_set_param(None, ck.PARAM_CHAIN_CAP, 10) == ck.EINVAL
    assert L.ck_insert_batch(None, None, None, 0, None, None) == ck.EINVAL
    assert L.ck_lookup_batch(None, None, 1, None, None, None) == ck.EINVAL
    assert L.ck_delete_batch(None, None, 1, None, None) == ck.EINVAL
    assert L.ck_stats(None, None) == ck.EINVAL
    assert ck.strerror(ck.EINVAL) == "invalid argument"
    assert ck.strerror(12345) == "unknown error"


def test_txn_invalid_arguments_need_no_gpu():
    from paper_1605_05236_gb300 import txn
    L = txn._lib()
    h = ctypes.c_void_p()
    assert L.ck_txn_create(None, 1 << 10, 8, 1, 0) == ck.EINVAL
    assert L.ck_txn_create(ctypes.byref(h), 1 << 10, 5, 1, 0) == ck.EINVAL   # B must be 4 or 8
    assert L.ck_txn_create(ctypes.byref(h), 1 << 10, 8, 0, 0) == ck.EINVAL   # no trials
    assert L.ck_txn_create(ctypes.byref(h), 1 << 28, 8, 1, 0) == ck.EINVAL   # slot indices overflow
    assert L.ck_txn_run(None, 0, None, None, None, 1, 1, 1, None, None, None, None, None, None) == ck.EINVAL
    assert L.ck_txn_reset(None) == ck.EINVAL
    assert L.ck_txn_stats(None, None, 1) == ck.EINVAL
    assert L.ck_txn_export(None, 0, None) == ck.EINVAL
    L.ck_txn_destroy(None)


def test_import_invalid_arguments_need_no_gpu():
    L = ck.load()
    assert L.ck_import(None, None, None) == ck.EINVAL


def test_debug_claims_invalid_arguments_need_no_gpu():
    L = ck.load()
    assert L.ck_debug_claims(None, 0, 1, 0) == ck.EINVAL
