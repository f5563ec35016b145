"""Binding of the serving form (ck_server_* in include/ck.h): a
continuous-batching request loop over one resident table, with native
open-loop replay of a trace and the sequential bulk-call reference."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import ck

OP_LOOKUP, OP_INSERT, OP_DELETE = 0, 1, 2
ST_BUSY = 4


class ServerConfig(ctypes.Structure):
    _fields_ = [("wave_keys", ctypes.c_uint64), ("wave_slots", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("load_hi", ctypes.c_double), ("max_defer_us", ctypes.c_uint64), ("hbm_fraction", ctypes.c_double)]


_bound = False


def _lib():
    global _bound
    L = ck.load()
    if not _bound:
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        L.ck_server_create.argtypes = [ctypes.POINTER(vp), vp, ctypes.POINTER(ServerConfig)]
        L.ck_server_replay.argtypes = [vp, u64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.ck_replay_sequential.argtypes = [vp, u64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.ck_server_info.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(u32)]
        L.ck_server_destroy.argtypes = [vp]
        L.ck_server_destroy.restype = None
        L.ck_now_ns.restype = ctypes.c_int64
        _bound = True
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _results(trace):
    n = len(trace["keys"])
    return np.zeros(n, dtype=np.uint32), np.zeros(n, dtype=np.uint8), np.zeros(len(trace["op"]), dtype=np.int64)


class Server:
    """Owns a CuckooTable (it must not be used otherwise while the server runs)."""

    def __init__(self, table: ck.CuckooTable, wave_keys=1 << 20, wave_slots=4, load_hi=0.97,
                 max_defer_us=20000, hbm_fraction=0.25):
        L = _lib()
        torch.cuda.synchronize()
        cfg = ServerConfig(wave_keys, wave_slots, 0, load_hi, max_defer_us, hbm_fraction)
        h = ctypes.c_void_p()
        ck._check(L.ck_server_create(ctypes.byref(h), table._h, ctypes.byref(cfg)), "ck_server_create")
        self._h = h
        self.table = table

    def close(self):
        if getattr(self, "_h", None):
            _lib().ck_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        w, b, ld, sl = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double(), ctypes.c_uint32()
        ck._check(_lib().ck_server_info(self._h, ctypes.byref(w), ctypes.byref(b), ctypes.byref(ld), ctypes.byref(sl)),
                  "ck_server_info")
        return {"waves": w.value, "busy_rejects": b.value, "load": ld.value, "wave_slots": sl.value}

    def replay(self, trace, time_scale=1.0):
        """Submit request i at arrive_ns[i] * time_scale after the start;
        returns (vals_out, status_out, latency_ns)."""
        vals, st, lat = _results(trace)
        arrive = (trace["arrive_ns"].astype(np.float64) * time_scale).astype(np.int64)
        rc = _lib().ck_server_replay(self._h, len(trace["op"]), _p(trace["op"]), _p(trace["key_off"]),
                                     _p(trace["n_keys"]), _p(arrive), _p(trace["keys"]), _p(trace["vals"]),
                                     _p(vals), _p(st), _p(lat))
        ck._check(rc, "ck_server_replay")
        return vals, st, lat


def replay_sequential(table: ck.CuckooTable, trace, time_scale=1.0, stream=None):
    """The trace as plain sequential bulk calls (the reference)."""
    vals, st, lat = _results(trace)
    arrive = (trace["arrive_ns"].astype(np.float64) * time_scale).astype(np.int64)
    rc = _lib().ck_replay_sequential(table._h, len(trace["op"]), _p(trace["op"]), _p(trace["key_off"]),
                                     _p(trace["n_keys"]), _p(arrive), _p(trace["keys"]), _p(trace["vals"]),
                                     _p(vals), _p(st), _p(lat), ck._stream(stream))
    ck._check(rc, "ck_replay_sequential")
    return vals, st, lat
