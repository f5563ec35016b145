"""Binding of the batched form (ck_multi_* in include/ck.h): many independent
two-choice tables in one device buffer, filled by one persistent launch."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import ck

MULTI_TILE, MULTI_BLOCK, MULTI_BLOCKS_PER_SM, MULTI_CHAIN_CAP = 1, 2, 3, 4
CAPTURE_CLEAR, CAPTURE_PER_TABLE = 1, 2


class MultiDesc(ctypes.Structure):
    _fields_ = [("bins", ctypes.c_uint64), ("slots_per_bin", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("key_offset", ctypes.c_uint64), ("n_keys", ctypes.c_uint64)]


_bound = False


def _lib():
    global _bound
    L = ck.load()
    if not _bound:
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        L.ck_multi_required_bytes.restype = ctypes.c_size_t
        L.ck_multi_required_bytes.argtypes = [vp, u32]
        L.ck_multi_create_on.argtypes = [ctypes.POINTER(vp), vp, ctypes.c_size_t, vp, u32, u32, u64, vp]
        L.ck_multi_set_param.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
        L.ck_multi_insert.argtypes = [vp, vp, vp, vp, vp]
        L.ck_multi_insert_per_table.argtypes = [vp, vp, vp, vp, vp]
        L.ck_multi_lookup.argtypes = [vp, vp, vp, u64, vp, vp, vp]
        L.ck_multi_table_stats.argtypes = [vp, u32, ctypes.POINTER(ck.CkStats)]
        L.ck_multi_stats.argtypes = [vp, ctypes.POINTER(ck.CkStats)]
        L.ck_multi_export.argtypes = [vp, u32, vp, vp]
        L.ck_multi_clear.argtypes = [vp, vp]
        L.ck_multi_destroy.argtypes = [vp]
        L.ck_multi_destroy.restype = None
        L.ck_multi_capture.argtypes = [vp, vp, vp, vp, u32, vp, ctypes.POINTER(vp)]
        L.ck_graph_launch.argtypes = [vp, vp]
        L.ck_graph_destroy.argtypes = [vp]
        L.ck_graph_destroy.restype = None
        _bound = True
    return L


def _descs(bins, slots, n_keys):
    n = len(bins)
    arr = (MultiDesc * n)()
    off = 0
    for i in range(n):
        arr[i].bins = int(bins[i])
        arr[i].slots_per_bin = int(slots[i])
        arr[i].key_offset = off
        arr[i].n_keys = int(n_keys[i])
        off += int(n_keys[i])
    return arr


class Graph:
    """A captured batched fill (ck_multi_capture): launch() replays it."""

    def __init__(self, handle, table):
        self._h = handle
        self._table = table  # keeps the tables (and their buffer) alive

    def launch(self, stream=None):
        ck._check(_lib().ck_graph_launch(self._h, ck._stream(stream)), "ck_graph_launch")

    def close(self):
        if getattr(self, "_h", None):
            _lib().ck_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiTable:
    """n independent tables: bins[i] x slots[i], n_keys[i] keys each (keys of
    table i are the i-th contiguous segment of the shared arrays)."""

    def __init__(self, bins, slots, n_keys, policy=ck.QUEUE, seed=0, stream=None):
        L = _lib()
        self.n_tables = len(bins)
        self.bins = np.asarray(bins, dtype=np.uint64)
        self.slots = np.asarray(slots, dtype=np.uint32)
        self.n_keys = np.asarray(n_keys, dtype=np.uint64)
        self.offsets = np.concatenate([[0], np.cumsum(self.n_keys)[:-1]]).astype(np.uint64)
        self._desc = _descs(self.bins, self.slots, self.n_keys)
        nbytes = int(L.ck_multi_required_bytes(ctypes.byref(self._desc), self.n_tables))
        if nbytes == 0:
            raise ValueError("invalid multi-table shapes")
        self._buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self._buf.data_ptr()
        off = (-base) % 256
        h = ctypes.c_void_p()
        rc = L.ck_multi_create_on(ctypes.byref(h), ctypes.c_void_p(base + off), nbytes, ctypes.byref(self._desc),
                                  self.n_tables, policy, seed, ck._stream(stream))
        ck._check(rc, "ck_multi_create_on")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib().ck_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_param(self, key, value):
        ck._check(_lib().ck_multi_set_param(self._h, key, int(value)), "ck_multi_set_param")

    def insert(self, keys, vals, status=None, per_table=False, stream=None):
        f = _lib().ck_multi_insert_per_table if per_table else _lib().ck_multi_insert
        ck._check(f(self._h, ck._ptr(keys), ck._ptr(vals), ck._ptr(status), ck._stream(stream)), "ck_multi_insert")
        return status

    def capture(self, keys, vals, status=None, per_table=False, clear=True, stream=None) -> "Graph":
        """Capture a fill (optionally after clearing every table) as a CUDA
        graph; Graph.launch() runs it.  The arrays must outlive the graph."""
        flags = (CAPTURE_CLEAR if clear else 0) | (CAPTURE_PER_TABLE if per_table else 0)
        h = ctypes.c_void_p()
        ck._check(_lib().ck_multi_capture(self._h, ck._ptr(keys), ck._ptr(vals), ck._ptr(status), flags,
                                          ck._stream(stream), ctypes.byref(h)), "ck_multi_capture")
        return Graph(h, self)

    def lookup(self, tab, keys, vals=None, found=None, stream=None):
        n = keys.numel()
        if vals is None:
            vals = torch.empty(n, dtype=torch.int32, device=keys.device)
        if found is None:
            found = torch.empty(n, dtype=torch.uint8, device=keys.device)
        ck._check(_lib().ck_multi_lookup(self._h, ck._ptr(tab), ck._ptr(keys), n, ck._ptr(vals), ck._ptr(found),
                                         ck._stream(stream)), "ck_multi_lookup")
        return vals, found

    def clear(self, stream=None):
        ck._check(_lib().ck_multi_clear(self._h, ck._stream(stream)), "ck_multi_clear")

    def stats(self, table=None) -> dict:
        s = ck.CkStats()
        if table is None:
            ck._check(_lib().ck_multi_stats(self._h, ctypes.byref(s)), "ck_multi_stats")
        else:
            ck._check(_lib().ck_multi_table_stats(self._h, table, ctypes.byref(s)), "ck_multi_table_stats")
        return {name: getattr(s, name) for name, _ in ck.CkStats._fields_}

    def contents(self, table) -> dict:
        ns = int(self.bins[table]) * int(self.slots[table])
        sl = np.zeros(ns, dtype=np.uint64)
        ck._check(_lib().ck_multi_export(self._h, table, sl.ctypes.data_as(ctypes.c_void_p), None), "ck_multi_export")
        live = sl[sl != np.uint64(0xFFFFFFFFFFFFFFFF)]
        return {int(r >> np.uint64(32)): int(r & np.uint64(0xFFFFFFFF)) for r in live}
