"""Host-side checks of an exported GPU table (test helper).

The structural invariants of a cuckoo table, evaluated with numpy on the
slot and metadata arrays copied out by ck_export: every record sits in one
of its own bins; a key stored twice is a ghost pair (one copy in each of its
two bins, both marked duplicate, Sec. 4); no other key is stored twice; no
claim flag is left set after a batch (Sec. 8).  The bins of a key are
recomputed here with a vectorised hash written from the same definition
(fmix32(key ^ seed_i) mod n, distinct choices); this is a property check,
not the oracle.
"""
import numpy as np

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
SEEDS = (0x9E3779B9, 0x85EBCA6B, 0xC2B2AE35, 0x27D4EB2F)


def fmix32_np(h):
    h = h.astype(np.uint32)
    with np.errstate(over="ignore"):
        h ^= h >> np.uint32(16)
        h *= np.uint32(0x85EBCA6B)
        h ^= h >> np.uint32(13)
        h *= np.uint32(0xC2B2AE35)
        h ^= h >> np.uint32(16)
    return h


def hash_np(keys, i, family):
    s = np.uint32(SEEDS[i])
    with np.errstate(over="ignore"):
        if family == 0:
            return fmix32_np(keys ^ s)
        return fmix32_np(fmix32_np(keys + s) ^ (s * np.uint32(0x27D4EB2F)))


def bins_np(keys, n_bins, d, family=0):
    keys = keys.astype(np.uint32)
    out = []
    for i in range(d):
        b = hash_np(keys, i, family).astype(np.uint64) % np.uint64(n_bins)
        for _ in range(d):
            clash = np.zeros(len(keys), dtype=bool)
            for j in range(i):
                clash |= b == out[j]
            if not clash.any():
                break
            b = np.where(clash, (b + np.uint64(1)) % np.uint64(n_bins), b)
        out.append(b)
    return np.stack(out, axis=1)


def check_table(slots, meta, n_bins, B, d, family=0):
    """Returns (live key -> value dict-free summary): size, ghost pairs.
    Raises AssertionError on any violated invariant."""
    slots = np.asarray(slots, dtype=np.uint64)
    meta = np.asarray(meta, dtype=np.uint32)
    assert slots.shape == (n_bins * B,)
    claim_bits = (1 << B) - 1 if B > 1 else 1
    assert not (meta & np.uint32(claim_bits)).any(), "claim flag left set"
    occ = slots != EMPTY
    idx = np.nonzero(occ)[0]
    recs = slots[idx]
    keys = (recs >> np.uint64(32)).astype(np.uint32)
    here = (idx // B).astype(np.uint64)
    kb = bins_np(keys, n_bins, d, family)
    mine = (kb == here[:, None]).any(axis=1)
    assert mine.all(), "record outside its bins: key %d" % int(keys[~mine][0])
    if B > 1:
        dup = ((meta[idx // B] >> (np.uint32(8) + (idx % B).astype(np.uint32))) & np.uint32(1)).astype(bool)
        empty_idx = np.nonzero(~occ)[0]
        edup = ((meta[empty_idx // B] >> (np.uint32(8) + (empty_idx % B).astype(np.uint32))) & np.uint32(1))
        assert not edup.any(), "empty slot marked duplicate"
    else:
        dup = np.zeros(len(idx), dtype=bool)
    order = np.argsort(keys, kind="stable")
    ks = keys[order]
    first = np.ones(len(ks), dtype=bool)
    first[1:] = ks[1:] != ks[:-1]
    counts = np.diff(np.append(np.nonzero(first)[0], len(ks)))
    assert counts.max(initial=1) <= 2, "key stored more than twice"
    twice = np.repeat(counts == 2, counts)
    # both copies of a twice-stored key are marked, in different bins, same value
    d_sorted = dup[order]
    assert (d_sorted[twice]).all(), "key stored twice without duplicate marks"
    assert not (d_sorted[~twice]).any(), "single copy marked duplicate"
    if twice.any():
        h_sorted = here[order][twice].reshape(-1, 2)
        r_sorted = recs[order][twice].reshape(-1, 2)
        assert (h_sorted[:, 0] != h_sorted[:, 1]).all(), "ghost copies share a bin"
        assert (r_sorted[:, 0] == r_sorted[:, 1]).all(), "ghost copies differ in value"
    return {"size": int(first.sum()), "ghost_pairs": int((counts == 2).sum())}
