"""Thin Python binding of libck.so (C ABI in include/ck.h).

Argument marshalling only: every operation runs in the library's CUDA
kernels.  Device memory comes from torch tensors, streams from torch's
current stream.  There is no CPU fallback: if libck.so cannot be loaded the
binding raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

# return codes
OK, EINVAL, ENOMEM, ECUDA, EBUSY, ENOTSUP = 0, -1, -2, -3, -4, -5
# per-key insert status
ST_OK, ST_FAILED, ST_ABORTED, ST_INVALID, ST_UPDATED = 0, 1, 2, 3, 5
CHAIN_BUCKETS = 40  # CK_CHAIN_BUCKETS
# policies (Sec. 3-7) and the ghost flag (Sec. 4)
RANDOM, BFS, SORTED, QUEUE, RATTLE, HYBRID = 0, 1, 2, 3, 4, 5
GHOST = 0x100
# parameters
PARAM_CHAIN_CAP, PARAM_MAX_RETRIES, PARAM_RNG_SEED = 1, 2, 3
PARAM_HASH_SEED0, PARAM_BLOCK = 10, 20
PARAM_RATTLE_TIE_RESIDENT, PARAM_ORDERED_WRITES, PARAM_OVERLAP, PARAM_HASH_FAMILY = 30, 31, 32, 33
PARAM_SPAWN_K, PARAM_MAX_INFLIGHT, PARAM_SEARCH_WARP, PARAM_SEARCH_WARP_LOAD = 34, 35, 36, 37
INS_SERIAL, INS_UPSERT = 1, 2
HIST_BUCKETS = 200

POLICY_NAMES = {"random": RANDOM, "bfs": BFS, "sorted": SORTED, "queue": QUEUE, "rattle": RATTLE,
                "hybrid": HYBRID}


class CkStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "inserts_ok", "inserts_failed", "inserts_aborted", "bins_viewed", "kicks", "chain_max",
        "aborts", "ghost_pairs_made", "dup_evictions", "size", "live_ghosts", "lookups",
        "lookup_hits", "deletes", "delete_hits", "delete_aborts", "conflict_views", "bins_viewed_all",
        "total_slots")] + [
        ("load", ctypes.c_double), ("bins_viewed_per_insert", ctypes.c_double),
        ("aborts_per_insert", ctypes.c_double), ("updates", ctypes.c_uint64)]


_lib = None
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libck.so (building it in-tree first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libck.so is not built (run __graft_entry__.build())")
        path = _build.build()
    L = ctypes.CDLL(path)
    L.ck_required_bytes.restype = ctypes.c_size_t
    L.ck_required_bytes.argtypes = [_u64, _u32, _u32, _u32]
    L.ck_create.argtypes = [ctypes.POINTER(_vp), _u64, _u32, _u32, _u32, _u64]
    L.ck_create_on.argtypes = [ctypes.POINTER(_vp), _vp, ctypes.c_size_t, _u64, _u32, _u32, _u32, _u64, _vp]
    L.ck_set_param.argtypes = [_vp, ctypes.c_int, ctypes.c_int64]
    L.ck_insert_batch.argtypes = [_vp, _vp, _vp, _u64, _vp, _vp]
    L.ck_insert_batch_ex.argtypes = [_vp, _vp, _vp, _u64, _vp, _vp, _u32, _vp]
    L.ck_lookup_batch.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp]
    L.ck_delete_batch.argtypes = [_vp, _vp, _u64, _vp, _vp]
    L.ck_stats.argtypes = [_vp, ctypes.POINTER(CkStats)]
    L.ck_load_histogram.argtypes = [_vp, _vp, _vp]
    L.ck_reset_stats.argtypes = [_vp]
    L.ck_chain_histogram.argtypes = [_vp, _vp]
    L.ck_clear.argtypes = [_vp, _vp]
    L.ck_export.argtypes = [_vp, _vp, _vp]
    L.ck_destroy.argtypes = [_vp]
    L.ck_destroy.restype = None
    L.ck_shape.argtypes = [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                           ctypes.POINTER(_u32)]
    L.ck_gather_probe.argtypes = [_vp, ctypes.c_size_t, _u32, _u64, _u64, _vp, _vp]
    L.ck_gather_probe_ex.argtypes = [_vp, ctypes.c_size_t, _u32, _u64, _u64, _u32, _u32, _u32, _vp, _vp]
    L.ck_atomic_probe.argtypes = [_vp, ctypes.c_size_t, _u32, _u64, _u64, _vp, _vp]
    L.ck_import.argtypes = [_vp, _vp, _vp]
    L.ck_debug_claims.argtypes = [_vp, _u64, _u32, _u32]
    L.ck_strerror.restype = ctypes.c_char_p
    L.ck_strerror.argtypes = [ctypes.c_int]
    _lib = L
    return L


def strerror(rc: int) -> str:
    return load().ck_strerror(rc).decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise RuntimeError("%s: %s (%d)" % (what, strerror(rc), rc))


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _u32_view(t):
    """uint32 data as torch stores it (int32 bit pattern or uint32)."""
    if t.dtype in (torch.int32, torch.uint32):
        return t
    raise ValueError("keys/values must be int32 or uint32 tensors (bit patterns)")


def required_bytes(bins, slots_per_bin, d=2, policy=RANDOM) -> int:
    return int(load().ck_required_bytes(bins, slots_per_bin, d, policy))


class CuckooTable:
    """A cuckoo table in device memory owned by a torch tensor.

    bins, slots_per_bin (4 or 8 with d=2; 1 with d=3/4), d, policy
    (RANDOM/BFS/SORTED/QUEUE/HYBRID, optionally | GHOST; RATTLE/RANDOM for d-ary),
    seed: the kick-out draw seed.
    """

    def __init__(self, bins, slots_per_bin, d=2, policy=RANDOM, seed=0, device=None, stream=None):
        L = load()
        self.bins, self.B, self.d, self.policy = int(bins), int(slots_per_bin), int(d), int(policy)
        nbytes = int(L.ck_required_bytes(self.bins, self.B, self.d, self.policy))
        if nbytes == 0:
            raise ValueError("invalid table shape (bins=%d, B=%d, d=%d, policy=%#x)"
                             % (self.bins, self.B, self.d, self.policy))
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self._buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self._buf.data_ptr()
        self._off = (-base) % 256
        self.nbytes = nbytes
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            rc = L.ck_create_on(ctypes.byref(h), ctypes.c_void_p(base + self._off), nbytes, self.bins,
                                self.B, self.d, self.policy, seed, _stream(stream))
        _check(rc, "ck_create_on")
        self._h = h

    # ---- lifetime ----
    def close(self):
        if getattr(self, "_h", None):
            load().ck_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def total_slots(self) -> int:
        return self.bins * self.B

    def set_param(self, key: int, value: int):
        _check(load().ck_set_param(self._h, key, int(value)), "ck_set_param")

    # ---- batch operations ----
    def insert(self, keys, vals, status=None, viewed=None, serial=False, stream=None, upsert=False):
        keys, vals = _u32_view(keys), _u32_view(vals)
        n = keys.numel()
        if vals.numel() != n:
            raise ValueError("keys and values differ in length")
        if status is None:
            status = torch.empty(n, dtype=torch.uint8, device=keys.device)
        flags = (INS_SERIAL if serial else 0) | (INS_UPSERT if upsert else 0)
        rc = load().ck_insert_batch_ex(self._h, _ptr(keys), _ptr(vals), n, _ptr(status), _ptr(viewed),
                                       flags, _stream(stream))
        _check(rc, "ck_insert_batch")
        return status

    def insert_batch(self, keys, vals, status=None, stream=None):
        """ck_insert_batch exactly (no per-key trace)."""
        keys, vals = _u32_view(keys), _u32_view(vals)
        rc = load().ck_insert_batch(self._h, _ptr(keys), _ptr(vals), keys.numel(), _ptr(status),
                                    _stream(stream))
        _check(rc, "ck_insert_batch")
        return status

    def lookup(self, keys, vals=None, found=None, stream=None):
        keys = _u32_view(keys)
        n = keys.numel()
        if vals is None:
            vals = torch.empty(n, dtype=torch.int32, device=keys.device)
        if found is None:
            found = torch.empty(n, dtype=torch.uint8, device=keys.device)
        rc = load().ck_lookup_batch(self._h, _ptr(keys), n, _ptr(vals), _ptr(found), _stream(stream))
        _check(rc, "ck_lookup_batch")
        return vals, found

    def delete(self, keys, found=None, stream=None):
        keys = _u32_view(keys)
        n = keys.numel()
        if found is None:
            found = torch.empty(n, dtype=torch.uint8, device=keys.device)
        rc = load().ck_delete_batch(self._h, _ptr(keys), n, _ptr(found), _stream(stream))
        _check(rc, "ck_delete_batch")
        return found

    def clear(self, stream=None):
        _check(load().ck_clear(self._h, _stream(stream)), "ck_clear")

    # ---- state ----
    def stats(self) -> dict:
        s = CkStats()
        _check(load().ck_stats(self._h, ctypes.byref(s)), "ck_stats")
        return {name: getattr(s, name) for name, _ in CkStats._fields_}

    def chain_histogram(self) -> np.ndarray:
        """Successful insertions by chain length (CHAIN_BUCKETS buckets, see
        ck_chain_histogram)."""
        out = np.zeros(CHAIN_BUCKETS, dtype=np.uint64)
        _check(load().ck_chain_histogram(self._h, out.ctypes.data_as(_vp)), "ck_chain_histogram")
        return out

    def reset_stats(self):
        _check(load().ck_reset_stats(self._h), "ck_reset_stats")

    def load_histogram(self):
        v = np.zeros(HIST_BUCKETS, dtype=np.uint64)
        c = np.zeros(HIST_BUCKETS, dtype=np.uint64)
        _check(load().ck_load_histogram(self._h, v.ctypes.data_as(ctypes.c_void_p),
                                        c.ctypes.data_as(ctypes.c_void_p)), "ck_load_histogram")
        return v, c

    def export(self):
        slots = np.zeros(self.bins * self.B, dtype=np.uint64)
        meta = np.zeros(self.bins, dtype=np.uint32)
        _check(load().ck_export(self._h, slots.ctypes.data_as(ctypes.c_void_p),
                                meta.ctypes.data_as(ctypes.c_void_p)), "ck_export")
        return slots, meta

    def import_snapshot(self, slots: np.ndarray, meta: np.ndarray):
        """ck_import: restore the slots and meta an export() of a table of
        the same shape returned."""
        slots = np.ascontiguousarray(slots, dtype=np.uint64)
        meta = np.ascontiguousarray(meta, dtype=np.uint32)
        if slots.size != self.bins * self.B or meta.size != self.bins:
            raise ValueError("snapshot shape differs from the table's")
        _check(load().ck_import(self._h, slots.ctypes.data_as(ctypes.c_void_p),
                                meta.ctypes.data_as(ctypes.c_void_p)), "ck_import")

    def debug_claims(self, bin: int, set_mask: int = 0, clear_mask: int = 0):
        """ck_debug_claims: set / clear claim flags of one bin (testing aid)."""
        _check(load().ck_debug_claims(self._h, bin, set_mask, clear_mask), "ck_debug_claims")

    def contents(self) -> dict:
        slots, _ = self.export()
        live = slots[slots != np.uint64(0xFFFFFFFFFFFFFFFF)]
        return {int(r >> np.uint64(32)): int(r & np.uint64(0xFFFFFFFF)) for r in live}


def as_u32_tensor(a: np.ndarray, device="cuda") -> torch.Tensor:
    """uint32 numpy array -> int32 CUDA tensor with the same bit pattern."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).to(device)


def u32_numpy(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def gather_probe(buf: torch.Tensor, width: int, n_reads: int, seed: int, sink: torch.Tensor, stream=None):
    """Random reads of `width` bytes from `buf` (see ck_gather_probe)."""
    rc = load().ck_gather_probe(_ptr(buf), buf.numel() * buf.element_size(), width, n_reads, seed,
                                _ptr(sink), _stream(stream))
    _check(rc, "ck_gather_probe")


def gather_probe_ex(buf: torch.Tensor, width: int, n_reads: int, seed: int, per_thread: int, block: int,
                    max_blocks: int, sink: torch.Tensor, stream=None):
    """Random reads with a given launch shape (see ck_gather_probe_ex)."""
    rc = load().ck_gather_probe_ex(_ptr(buf), buf.numel() * buf.element_size(), width, n_reads, seed, per_thread,
                                   block, max_blocks, _ptr(sink), _stream(stream))
    _check(rc, "ck_gather_probe_ex")


def atomic_probe(buf: torch.Tensor, kind: int, n_ops: int, seed: int, sink: torch.Tensor, stream=None):
    """Random atomics on `buf` (see ck_atomic_probe; kind 0: red.add.u32,
    1: atom.add.u32, 2: atom.cas.b64)."""
    rc = load().ck_atomic_probe(_ptr(buf), buf.numel() * buf.element_size(), kind, n_ops, seed,
                                _ptr(sink), _stream(stream))
    _check(rc, "ck_atomic_probe")
