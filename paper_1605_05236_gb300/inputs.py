"""Seeded synthetic inputs shared by the library's tests, benchmark and oracle.

This module only generates keys, values and key orders.  It holds none of
the cuckoo method's arithmetic (no hashing into bins, no policy), so the
CUDA path and the CPU oracle can both consume its output without sharing
any of the computation under test.

Recipe (the paper uses "uniformly randomly generated hashes" and keys that
are absent when inserted, Sec. 3):
  * key stream of seed s: SplitMix64 seeded with s, high 32 bits of each
    output; 0xFFFFFFFF (the empty-slot marker), repeats and excluded keys
    are skipped, so the first n survivors are n distinct uniform uint32 keys;
  * value of key k: k * 2654435761 mod 2^32;
  * absent keys for lookups continue the same stream after the inserted
    keys, skipping every inserted key;
  * orders: forward Fisher-Yates shuffles driven by the stream of another
    seed (position i swaps with i + out_i mod (n - i)).

The work is done by inputs_gen.c (compiled with gcc on first use); the
``ref_*`` functions restate it in numpy/Python for tests on small sizes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

RESERVED_KEY = 0xFFFFFFFF
GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "inputs_gen.c")
_LIB = os.path.join(_HERE, "_build", "libckgen.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _gen():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.gen_distinct_keys.restype = ctypes.c_int64
        L.gen_distinct_keys.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                        ctypes.c_uint64, ctypes.c_void_p]
        L.gen_permutation.restype = ctypes.c_int
        L.gen_permutation.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
        L.gen_gather_u32.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and len(a) else None


def splitmix64_stream(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of SplitMix64 seeded with `seed`
    (Steele, Lea and Flood 2014): state_i = seed + (i+1)*gamma, then mixed."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def distinct_keys(n: int, seed: int, exclude: np.ndarray | None = None,
                  start: int = 0) -> tuple[np.ndarray, int]:
    """n distinct uint32 keys from the stream of `seed` beginning at output
    `start`, skipping `exclude`; returns (keys, stream index after the last key)."""
    out = np.empty(n, dtype=np.uint32)
    ex = None if exclude is None else np.ascontiguousarray(exclude, dtype=np.uint32)
    nxt = _gen().gen_distinct_keys(seed & 0xFFFFFFFFFFFFFFFF, start, n, _p(ex), 0 if ex is None else len(ex),
                                   _p(out))
    if nxt < 0:
        raise MemoryError("key generator: out of memory")
    return out, int(nxt)


def permutation(n: int, seed: int, k: int | None = None) -> np.ndarray:
    """The first k (default n) entries of a forward Fisher-Yates shuffle of range(n)."""
    k = n if k is None else min(k, n)
    out = np.empty(k, dtype=np.uint64)
    if _gen().gen_permutation(seed & 0xFFFFFFFFFFFFFFFF, n, k, _p(out)) != 0:
        raise MemoryError("permutation: out of memory")
    return out.astype(np.int64)


def values_for(keys: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        return (keys.astype(np.uint64) * np.uint64(2654435761) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def lookup_keys(inserted: np.ndarray, n: int, seed: int, hit_fraction: float = 0.5,
                next_start: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """n lookup keys: round(n*hit_fraction) distinct present keys drawn from
    `inserted` and the rest absent keys continuing the key stream of `seed`
    at `next_start`; shuffled together.  Returns (keys, expected_present)."""
    n_hit = min(int(round(n * hit_fraction)), len(inserted))
    present = inserted[permutation(len(inserted), seed + 1000, n_hit)]
    absent, _ = distinct_keys(n - n_hit, seed, exclude=inserted, start=next_start)
    keys = np.concatenate([present, absent])
    flag = np.concatenate([np.ones(n_hit, np.uint8), np.zeros(n - n_hit, np.uint8)])
    order = permutation(n, seed + 2000)
    return keys[order], flag[order]


def delete_keys(inserted: np.ndarray, n: int, seed: int) -> np.ndarray:
    """The first n keys of a random permutation of the inserted set."""
    return inserted[permutation(len(inserted), seed + 3000, n)]


def load_target(slots: int, load: float) -> int:
    """Number of keys that fills `slots` slots to `load` (rounded down)."""
    return int(np.floor(slots * load + 1e-9))


# ---- plain restatements for tests (small sizes) ----

def ref_distinct_keys(n, seed, exclude=(), start=0):
    seen = set(int(x) for x in exclude)
    out, i = [], start
    while len(out) < n:
        k = int(splitmix64_stream(seed, i, 1)[0]) >> 32
        i += 1
        if k == RESERVED_KEY or k in seen:
            continue
        seen.add(k)
        out.append(k)
    return np.array(out, dtype=np.uint32), i


def ref_permutation(n, seed, k=None):
    k = n if k is None else min(k, n)
    a = list(range(n))
    outs = splitmix64_stream(seed, 0, max(n, 1))
    for i in range(min(k, n - 1) if n else 0):
        j = i + int(outs[i]) % (n - i)
        a[i], a[j] = a[j], a[i]
    return np.array(a[:k], dtype=np.int64)


def multi_shapes(n_tables: int, seed: int = 7, lo_log2: int = 10, hi_log2: int = 18):
    """Shapes of the batched workload: table i has floor(2^(lo + (hi-lo)*u))
    bins, u uniform in [0,1) from output 2i of the stream of `seed` (top 53
    bits), and 4 or 8 slots per bin from the top bit of output 2i+1."""
    out = splitmix64_stream(seed, 0, 2 * n_tables)
    u = (out[0::2] >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    bins = np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.uint64)
    slots = np.where((out[1::2] >> np.uint64(63)) == 0, 4, 8).astype(np.uint32)
    return bins, slots


def multi_keys(bins, slots, load: float, seed0: int = 8):
    """Per table i: floor(load * slots) distinct keys from the stream of seed
    seed0 + i, concatenated; returns (keys, values, n_keys)."""
    n_keys = np.array([load_target(int(b) * int(s), load) for b, s in zip(bins, slots)], dtype=np.uint64)
    keys = np.empty(int(n_keys.sum()), dtype=np.uint32)
    off = 0
    for i, n in enumerate(n_keys):
        k, _ = distinct_keys(int(n), seed0 + i)
        keys[off:off + int(n)] = k
        off += int(n)
    return keys, values_for(keys), n_keys


def serving_trace(prefill_keys: np.ndarray, n_req: int, mix: tuple, seed: int = 11,
                  rate_per_ms: float = 20000.0, max_log2: int = 16, hit_fraction: float = 0.5):
    """A request trace for the serving loop.

    Arrivals: a Poisson process of `rate_per_ms` requests per millisecond
    (exponential gaps from the stream of seed+1).  Sizes: floor(2^(max_log2*u))
    keys, u uniform (log-uniform 1 .. 2^max_log2; stream seed+2).  Kinds:
    lookup / insert / delete with probabilities `mix` (stream seed+3).
    Keys are drawn so every result is fixed by the trace alone, whatever
    runs concurrently: lookups take present keys from the first half of the
    prefilled set (never deleted) and absent keys never inserted; inserts
    take fresh keys; deletes take keys of the second half of the prefilled
    set, each once.

    Returns dict(op, n_keys, key_off, arrive_ns, keys, vals, expect) with
    expect = the per-key result (lookups: 1 present / 0 absent; inserts and
    deletes: 1)."""
    out = splitmix64_stream(seed + 1, 0, n_req)
    u = (out >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    gaps = -np.log1p(-u) / rate_per_ms * 1e6
    arrive = np.cumsum(gaps).astype(np.int64)
    arrive -= arrive[0]
    u2 = (splitmix64_stream(seed + 2, 0, n_req) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    n_keys = np.maximum(1, np.floor(2.0 ** (max_log2 * u2))).astype(np.uint64)
    u3 = (splitmix64_stream(seed + 3, 0, n_req) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    cum = np.cumsum(mix) / np.sum(mix)
    op = np.searchsorted(cum, u3, side="right").astype(np.uint32)
    op = np.minimum(op, 2)
    half = len(prefill_keys) // 2
    stable, deletable = prefill_keys[:half], prefill_keys[half:]
    n_look = int(n_keys[op == 0].sum())
    n_ins = int(n_keys[op == 1].sum())
    n_del = int(n_keys[op == 2].sum())
    if n_del > len(deletable):
        raise ValueError("trace deletes more keys than the prefilled set can give")
    n_hit = int(round(n_look * hit_fraction))
    fresh, _ = distinct_keys(n_ins + (n_look - n_hit), seed + 4, exclude=prefill_keys)
    ins_keys, absent = fresh[:n_ins], fresh[n_ins:]
    present = stable[permutation(len(stable), seed + 5, n_hit)]
    look = np.concatenate([present, absent])
    look_exp = np.concatenate([np.ones(n_hit, np.uint8), np.zeros(n_look - n_hit, np.uint8)])
    order = permutation(n_look, seed + 6)
    look, look_exp = look[order], look_exp[order]
    dele = deletable[permutation(len(deletable), seed + 7, n_del)]
    keys = np.empty(int(n_keys.sum()), dtype=np.uint32)
    expect = np.ones(len(keys), dtype=np.uint8)
    key_off = np.concatenate([[0], np.cumsum(n_keys)[:-1]]).astype(np.uint64)
    pos = [0, 0, 0]
    for i in range(n_req):
        o, n, off = int(op[i]), int(n_keys[i]), int(key_off[i])
        src = (look, ins_keys, dele)[o]
        keys[off:off + n] = src[pos[o]:pos[o] + n]
        if o == 0:
            expect[off:off + n] = look_exp[pos[o]:pos[o] + n]
        pos[o] += n
    return {"op": op, "n_keys": n_keys, "key_off": key_off, "arrive_ns": arrive, "keys": keys,
            "vals": values_for(keys), "expect": expect}


TX_INSERT, TX_READ, TX_OVERWRITE, TX_DELETE = 0, 1, 2, 3


def txn_workload(n_workers: int, txns_per_worker: int, ops_per_txn: int, mix: tuple, seed: int = 13,
                 fill_to: int | None = None):
    """Transactions for the transactional layer (Sec. 8 experiments).

    Worker w runs transactions w*T .. w*T + T - 1 in order, each of
    `ops_per_txn` operations: insert / delete / overwrite / read with
    weights `mix` (the paper's delete-light 1:0:1:1 and delete-heavy
    2:1:2:2).  Inserts take fresh distinct keys (stream of `seed`) and
    random values.  A read, overwrite or delete targets a uniformly drawn
    key among all the keys the same worker inserted in its earlier
    transactions, deleted ones included (Sec. 8 draws from every record the
    thread ever inserted), at most once per transaction; with none
    available the operation becomes an insert.  Choices come from SplitMix64
    streams of seed+1 (kinds), seed+2 (targets) and seed+3 (values).

    `delta` is each transaction's net change of the table's size (inserts
    less deletes of keys still present), from the generator's own record of
    each worker's live keys.  With `fill_to`, every worker keeps only its
    first t transactions, t the least for which the workers' total net
    inserts reach `fill_to` (txns_per_worker is then an upper bound).
    Returns dict(op, key, val, delta, workers, txns_per_worker,
    ops_per_txn); operations transaction-major."""
    T, L = txns_per_worker, ops_per_txn
    n = n_workers * T * L
    fresh, _ = distinct_keys(n, seed)
    kind_u = (splitmix64_stream(seed + 1, 0, n) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    pick = splitmix64_stream(seed + 2, 0, n)
    vals = (splitmix64_stream(seed + 3, 0, n) >> np.uint64(32)).astype(np.uint32)
    cum = np.cumsum(mix) / float(np.sum(mix))
    kinds = np.minimum(np.searchsorted(cum, kind_u, side="right"), 3)
    # mix order is (insert, delete, overwrite, read)
    code = np.array([TX_INSERT, TX_DELETE, TX_OVERWRITE, TX_READ], dtype=np.uint8)[kinds]
    op = np.empty(n, dtype=np.uint8)
    key = np.empty(n, dtype=np.uint32)
    delta = np.zeros(n_workers * T, dtype=np.int64)
    nxt = 0
    for w in range(n_workers):
        ever = []    # keys this worker inserted in earlier transactions
        live = set()
        for t in range(T):
            base = (w * T + t) * L
            used = set()
            born = []
            d = 0
            for j in range(L):
                i = base + j
                c = int(code[i])
                cand = None
                if c != TX_INSERT and ever:
                    for probe in range(8):
                        k = ever[int((pick[i] >> np.uint64(8 * probe)) % np.uint64(len(ever)))]
                        if k not in used:
                            cand = k
                            break
                if cand is None:
                    c = TX_INSERT
                if c == TX_INSERT:
                    k = int(fresh[nxt])
                    nxt += 1
                    born.append(k)
                    d += 1
                else:
                    k = cand
                    if c == TX_DELETE and k in live:
                        live.discard(k)
                        d -= 1
                used.add(k)
                op[i] = c
                key[i] = k
            ever.extend(born)
            live.update(born)
            delta[w * T + t] = d
    if fill_to is not None:
        per = delta.reshape(n_workers, T).cumsum(1).sum(0)  # total after t+1 transactions each
        hit = np.nonzero(per >= fill_to)[0]
        if not len(hit):
            raise ValueError("txns_per_worker too small to reach fill_to")
        t_keep = int(hit[0]) + 1
        keep = (np.arange(n).reshape(n_workers, T, L)[:, :t_keep, :]).reshape(-1)
        op, key, vals = op[keep], key[keep], vals[keep]
        delta = delta.reshape(n_workers, T)[:, :t_keep].reshape(-1)
        T = t_keep
    return {"op": op, "key": key, "val": vals, "delta": delta, "workers": n_workers, "txns_per_worker": T,
            "ops_per_txn": L}
