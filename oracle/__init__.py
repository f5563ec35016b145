"""Serial CPU oracle for the cuckoo-table hot path (arXiv:1605.05236).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library in ``paper_1605_05236_gb300``; the two meet only
in the seeded input generator ``paper_1605_05236_gb300.inputs``, which holds
none of the method's arithmetic.

The arithmetic lives in ``ck_oracle.c`` (plain C, one insertion at a time,
each policy written in the order the paper describes it).  This module
compiles it with gcc and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ck_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libck_oracle.so")

RANDOM, BFS, SORTED, QUEUE, RATTLE, HYBRID = 0, 1, 2, 3, 4, 5
GHOST = 0x100
ST_OK, ST_FAILED, ST_INVALID, ST_UPDATED = 0, 1, 3, 5

# order of the counters returned by stats()
STAT_NAMES = (
    "inserts_ok", "inserts_failed", "bins_viewed", "kicks", "chain_max",
    "ghost_pairs_made", "dup_evictions", "size", "live_ghosts", "lookups",
    "lookup_hits", "deletes", "delete_hits", "prop41_violations",
    "prop41_checks", "updates",
)

DEFAULT_SEEDS = (0x9E3779B9, 0x85EBCA6B, 0xC2B2AE35, 0x27D4EB2F)


def build(force: bool = False) -> str:
    """Compile ck_oracle.c into oracle/_build/libck_oracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-pthread",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, u32p]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_insert_batch.argtypes = [ctypes.c_void_p, u32p, u32p, ctypes.c_uint64, u8p, u32p, u32p]
        L.orc_lookup_batch.argtypes = [ctypes.c_void_p, u32p, ctypes.c_uint64, u32p, u8p]
        L.orc_delete_batch.argtypes = [ctypes.c_void_p, u32p, ctypes.c_uint64, u8p]
        L.orc_lookup_batch_threads.argtypes = [ctypes.c_void_p, u32p, ctypes.c_uint64, u32p, u8p, ctypes.c_uint32]
        L.orc_lookup_batch_threads.restype = ctypes.c_int
        L.orc_delete_batch_threads.argtypes = [ctypes.c_void_p, u32p, ctypes.c_uint64, u8p, ctypes.c_uint32]
        L.orc_delete_batch_threads.restype = ctypes.c_int
        L.orc_upsert_batch.argtypes = [ctypes.c_void_p, u32p, u32p, ctypes.c_uint64, u8p]
        L.orc_stats.argtypes = [ctypes.c_void_p, u64p]
        L.orc_n_stats.restype = ctypes.c_uint32
        L.orc_export.argtypes = [ctypes.c_void_p, u64p, u8p, u8p, u8p, u8p]
        L.orc_check_invariants.restype = ctypes.c_int
        L.orc_check_invariants.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_uint64]
        L.orc_set_spawn_k.restype = ctypes.c_int
        L.orc_set_spawn_k.argtypes = [ctypes.c_void_p, ctypes.c_uint32]
        L.orc_set_spawn.restype = ctypes.c_int
        L.orc_set_spawn.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32]
        L.orc_set_bins_override.restype = ctypes.c_int
        L.orc_set_bins_override.argtypes = [ctypes.c_void_p, u32p, u64p, ctypes.c_uint64]
        L.orc_set_rattle_tie_resident.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_hash_family.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_bins.argtypes = [ctypes.c_void_p, ctypes.c_uint32, u64p]
        L.orc_fmix32.restype = ctypes.c_uint32
        L.orc_fmix32.argtypes = [ctypes.c_uint32]
        L.orc_splitmix64_at.restype = ctypes.c_uint64
        L.orc_splitmix64_at.argtypes = [ctypes.c_uint64]
        assert L.orc_n_stats() == len(STAT_NAMES)
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def fmix32(x: int) -> int:
    return int(lib().orc_fmix32(x & 0xFFFFFFFF))


def splitmix64_at(x: int) -> int:
    return int(lib().orc_splitmix64_at(x & 0xFFFFFFFFFFFFFFFF))


class OracleTable:
    """One serial cuckoo table.

    bins, slots_per_bin (B), d, policy (RANDOM/BFS/SORTED/QUEUE/RATTLE/HYBRID,
    OR GHOST), rng_seed (the kick-out draws), cap (kick-out cap for walks,
    try cap for rattle, bin budget for searches), seeds (hash seeds).
    """

    def __init__(self, bins, slots_per_bin, d=2, policy=RANDOM, rng_seed=0, cap=500,
                 seeds=DEFAULT_SEEDS):
        L = lib()
        self.bins, self.B, self.d, self.policy = int(bins), int(slots_per_bin), int(d), int(policy)
        s = np.array(list(seeds)[:4] + [0] * (4 - len(seeds)), dtype=np.uint32)
        self._h = L.orc_create(self.bins, self.B, self.d, self.policy, rng_seed, cap,
                               _ptr(s, ctypes.c_uint32))
        if not self._h:
            raise ValueError("orc_create rejected the parameters")

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_spawn_k(self, k):
        """Searches: spawns per round, their bins viewed together (1..8; 1 = plain)."""
        if lib().orc_set_spawn_k(self._h, int(k)) != 0:
            raise ValueError("spawn_k must be 1..8")

    def set_spawn(self, bin, count):
        """Fixtures: start `bin` with spawn count `count` (0..15)."""
        if lib().orc_set_spawn(self._h, int(bin), int(count)) != 0:
            raise ValueError("spawn count out of range")

    def set_bins(self, keys, bins):
        keys = np.ascontiguousarray(keys, dtype=np.uint32)
        bins = np.ascontiguousarray(bins, dtype=np.uint64).reshape(-1)
        rc = lib().orc_set_bins_override(self._h, _ptr(keys, ctypes.c_uint32),
                                         _ptr(bins, ctypes.c_uint64), len(keys))
        if rc != 0:
            raise ValueError("bad bin override")

    def set_hash_family(self, family: int):
        lib().orc_set_hash_family(self._h, int(family))

    def set_rattle_tie_resident(self, on: bool):
        lib().orc_set_rattle_tie_resident(self._h, 1 if on else 0)

    def bins_of(self, key):
        out = np.zeros(4, dtype=np.uint64)
        lib().orc_bins(self._h, key, _ptr(out, ctypes.c_uint64))
        return [int(x) for x in out[: self.d]]

    def insert(self, keys, vals, trace=False):
        keys = np.ascontiguousarray(keys, dtype=np.uint32)
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        n = len(keys)
        st = np.zeros(n, dtype=np.uint8)
        viewed = np.zeros(n, dtype=np.uint32) if trace else None
        kicks = np.zeros(n, dtype=np.uint32) if trace else None
        lib().orc_insert_batch(self._h, _ptr(keys, ctypes.c_uint32), _ptr(vals, ctypes.c_uint32), n,
                               _ptr(st, ctypes.c_uint8), _ptr(viewed, ctypes.c_uint32),
                               _ptr(kicks, ctypes.c_uint32))
        if trace:
            return st, viewed, kicks
        return st

    def lookup(self, keys):
        keys = np.ascontiguousarray(keys, dtype=np.uint32)
        vals = np.zeros(len(keys), dtype=np.uint32)
        found = np.zeros(len(keys), dtype=np.uint8)
        lib().orc_lookup_batch(self._h, _ptr(keys, ctypes.c_uint32), len(keys),
                               _ptr(vals, ctypes.c_uint32), _ptr(found, ctypes.c_uint8))
        return vals, found

    def delete(self, keys):
        keys = np.ascontiguousarray(keys, dtype=np.uint32)
        found = np.zeros(len(keys), dtype=np.uint8)
        lib().orc_delete_batch(self._h, _ptr(keys, ctypes.c_uint32), len(keys),
                               _ptr(found, ctypes.c_uint8))
        return found

    def lookup_threads(self, keys, threads):
        """lookup() split over `threads` host threads; returns (vals, found,
        threads actually used)."""
        keys = np.ascontiguousarray(keys, dtype=np.uint32)
        vals = np.zeros(len(keys), dtype=np.uint32)
        found = np.zeros(len(keys), dtype=np.uint8)
        used = lib().orc_lookup_batch_threads(self._h, _ptr(keys, ctypes.c_uint32), len(keys),
                                              _ptr(vals, ctypes.c_uint32), _ptr(found, ctypes.c_uint8), threads)
        return vals, found, used

    def delete_threads(self, keys, threads):
        """delete() of distinct keys split over `threads` host threads;
        returns (found, threads actually used)."""
        keys = np.ascontiguousarray(keys, dtype=np.uint32)
        found = np.zeros(len(keys), dtype=np.uint8)
        used = lib().orc_delete_batch_threads(self._h, _ptr(keys, ctypes.c_uint32), len(keys),
                                              _ptr(found, ctypes.c_uint8), threads)
        return found, used

    def upsert(self, keys, vals):
        """Insert, or overwrite the value of a present key (status 5)."""
        keys = np.ascontiguousarray(keys, dtype=np.uint32)
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        st = np.zeros(len(keys), dtype=np.uint8)
        lib().orc_upsert_batch(self._h, _ptr(keys, ctypes.c_uint32), _ptr(vals, ctypes.c_uint32), len(keys),
                               _ptr(st, ctypes.c_uint8))
        return st

    def stats(self) -> dict:
        out = np.zeros(len(STAT_NAMES), dtype=np.uint64)
        lib().orc_stats(self._h, _ptr(out, ctypes.c_uint64))
        return {k: int(v) for k, v in zip(STAT_NAMES, out)}

    def export(self) -> dict:
        ns = self.bins * self.B
        rec = np.zeros(ns, dtype=np.uint64)
        dup = np.zeros(ns, dtype=np.uint8)
        rat = np.zeros(ns, dtype=np.uint8)
        hit = np.zeros(self.bins, dtype=np.uint8)
        spawn = np.zeros(self.bins, dtype=np.uint8)
        lib().orc_export(self._h, _ptr(rec, ctypes.c_uint64), _ptr(dup, ctypes.c_uint8),
                         _ptr(rat, ctypes.c_uint8), _ptr(hit, ctypes.c_uint8),
                         _ptr(spawn, ctypes.c_uint8))
        return {"rec": rec, "dup": dup, "rattle": rat, "hit": hit, "spawn": spawn}

    def check_invariants(self):
        buf = ctypes.create_string_buffer(256)
        bad = lib().orc_check_invariants(self._h, buf, 256)
        return bad, buf.value.decode()

    def contents(self) -> dict:
        """key -> value over the live keys (each ghost pair once)."""
        rec = self.export()["rec"]
        live = rec[rec != np.uint64(0xFFFFFFFFFFFFFFFF)]
        return {int(r >> np.uint64(32)): int(r & np.uint64(0xFFFFFFFF)) for r in live}
