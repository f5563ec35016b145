"""Seeded synthetic inputs shared by the library's tests, benchmark and oracle.

This module only generates keys, values and key orders.  It holds none of
the cuckoo method's arithmetic (no hashing into bins, no policy), so the
CUDA path and the CPU oracle can both consume its output without sharing
any of the computation under test.

Recipe (the paper uses "uniformly randomly generated hashes" and keys that
are absent when inserted, Sec. 3):
  * keys: the SplitMix64 stream seeded with `seed`, high 32 bits of each
    output; 0xFFFFFFFF (the empty-slot marker) and repeats are dropped, so
    the first n survivors are n distinct uniform uint32 keys;
  * value of key k: k * 2654435761 mod 2^32;
  * absent keys for lookups continue the same stream, skipping keys that
    were inserted;
  * orders are random permutations: argsort of a second SplitMix64 stream.
"""
from __future__ import annotations

import numpy as np

RESERVED_KEY = 0xFFFFFFFF
GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_stream(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of SplitMix64 seeded with `seed`
    (Steele, Lea and Flood 2014): state_i = seed + (i+1)*gamma, then mixed."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _first_distinct(cand: np.ndarray, exclude: np.ndarray | None) -> np.ndarray:
    """Candidates in order of first appearance, without repeats, without the
    reserved key and without anything in `exclude`."""
    _, first = np.unique(cand, return_index=True)
    first.sort()
    out = cand[first]
    out = out[out != np.uint32(RESERVED_KEY)]
    if exclude is not None and len(exclude):
        out = out[~np.isin(out, exclude, assume_unique=False)]
    return out


def distinct_keys(n: int, seed: int, exclude: np.ndarray | None = None,
                  start: int = 0) -> tuple[np.ndarray, int]:
    """n distinct uint32 keys from the stream of `seed` beginning at output
    `start`; returns (keys, next_start)."""
    got = np.empty(0, dtype=np.uint32)
    pos = start
    while len(got) < n:
        need = n - len(got)
        m = int(need * 1.02) + 1024
        cand = (splitmix64_stream(seed, pos, m) >> np.uint64(32)).astype(np.uint32)
        pos += m
        if len(got):
            ex = got if exclude is None else np.concatenate([exclude, got])
        else:
            ex = exclude
        got = np.concatenate([got, _first_distinct(cand, ex)])
    # trim to exactly n, and report where the stream position of the nth key is
    return got[:n].copy(), pos


def values_for(keys: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        return (keys.astype(np.uint64) * np.uint64(2654435761) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def permutation(n: int, seed: int) -> np.ndarray:
    """A uniformly random permutation of range(n): argsort of n stream outputs."""
    return np.argsort(splitmix64_stream(seed, 0, n), kind="stable")


def lookup_keys(inserted: np.ndarray, n: int, seed: int, hit_fraction: float = 0.5,
                next_start: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """n lookup keys: round(n*hit_fraction) present keys drawn without
    repetition from `inserted` (in a random order) and the rest absent keys
    that continue the key stream; shuffled together.  Returns (keys,
    expected_present)."""
    n_hit = int(round(n * hit_fraction))
    n_hit = min(n_hit, len(inserted)) if len(inserted) else 0
    perm = permutation(len(inserted), seed + 1000)[:n_hit]
    present = inserted[perm]
    absent, _ = distinct_keys(n - n_hit, seed, exclude=inserted, start=next_start)
    keys = np.concatenate([present, absent])
    flag = np.concatenate([np.ones(n_hit, np.uint8), np.zeros(n - n_hit, np.uint8)])
    order = permutation(n, seed + 2000)
    return keys[order].copy(), flag[order].copy()


def delete_keys(inserted: np.ndarray, n: int, seed: int) -> np.ndarray:
    """The first n keys of a random permutation of the inserted set."""
    return inserted[permutation(len(inserted), seed + 3000)[:n]].copy()


def load_target(slots: int, load: float) -> int:
    """Number of keys that fills `slots` slots to `load` (rounded down)."""
    return int(np.floor(slots * load + 1e-9))
