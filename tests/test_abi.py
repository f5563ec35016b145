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


def test_binding_constants_match_the_header():
    """Every CK_* constant the Python bindings name (policy codes, statuses,
    error codes, parameter keys, flags, operation kinds) has the header's
    value.  Binding name -> header name, per module."""
    from paper_1605_05236_gb300 import multi, serve, txn
    src = open(os.path.join(ROOT, "include", "ck.h")).read()
    header = {}
    for name, val in re.findall(r"^#define CK_([A-Z0-9_]+)\s+\(?(-?(?:0x[0-9A-Fa-f]+|[0-9]+))u?\)?", src, flags=re.M):
        header[name] = int(val, 0)
    pairs = [(ck, n, n) for n in ("OK", "EINVAL", "ENOMEM", "ECUDA", "EBUSY", "ENOTSUP", "ST_OK", "ST_FAILED",
                                  "ST_ABORTED", "ST_INVALID", "ST_UPDATED", "CHAIN_BUCKETS", "RANDOM", "BFS",
                                  "SORTED", "QUEUE", "RATTLE", "HYBRID", "GHOST", "INS_SERIAL", "INS_UPSERT")]
    pairs += [(ck, n, n) for n in header if n.startswith("PARAM_")]
    pairs += [(multi, n, n) for n in ("MULTI_TILE", "MULTI_BLOCK", "MULTI_BLOCKS_PER_SM", "MULTI_CHAIN_CAP")]
    pairs += [(multi, "CAPTURE_CLEAR", "MULTI_CAPTURE_CLEAR"), (multi, "CAPTURE_PER_TABLE", "MULTI_CAPTURE_PER_TABLE")]
    pairs += [(serve, n, n) for n in ("OP_LOOKUP", "OP_INSERT", "OP_DELETE", "ST_BUSY")]
    pairs += [(txn, n, n) for n in ("TX_INSERT", "TX_READ", "TX_OVERWRITE", "TX_DELETE")]
    pairs += [(txn, n, "TXF_" + n) for n in ("LOCAL_RETRY", "QUEUE", "SYSTEM", "CLAIM")]
    pairs += [(txn, "MAX_OPS", "TXN_MAX_OPS"), (txn, "N_COUNTERS", "TXN_COUNTERS")]
    for mod, py, h in pairs:
        assert getattr(mod, py) == header[h], (mod.__name__, py, h)
    assert len(pairs) >= 45
