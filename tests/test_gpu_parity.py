"""GPU parity: the CUDA path (through the C ABI) against the serial oracle.

* Serial replay (one insertion in flight, keys in batch order): the slot
  layout, the policy's metadata (duplicate marks, hit counters, spawn
  counts, rattle counters), every per-key status and every per-key count of
  bins viewed equal the oracle's exactly.
* Concurrent batches: the key->value map, every lookup and every delete
  result equal the oracle's exactly (the layout may differ); the table
  passes the structural invariants; the mean bins viewed per insertion is
  within 10% of the oracle's at the same load.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_05236_gb300 import ck, inputs
from table_checks import check_table

pytestmark = pytest.mark.gpu

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)

TWO_CHOICE = [ck.RANDOM, ck.BFS, ck.SORTED, ck.QUEUE, ck.HYBRID, ck.RANDOM | ck.GHOST, ck.BFS | ck.GHOST,
              ck.SORTED | ck.GHOST, ck.QUEUE | ck.GHOST, ck.HYBRID | ck.GHOST]


def pname(p):
    base = {0: "random", 1: "bfs", 2: "sorted", 3: "queue", 4: "rattle", 5: "hybrid"}[p & 0xFF]
    return base + ("+ghost" if p & ck.GHOST else "") + ("+hash1" if p & 0x10000 else "")


def make_pair(bins, B, d, policy, seed, cap):
    """(oracle table, GPU table) with the same shape, policy, draws and hash family."""
    family = 1 if policy & 0x10000 else 0
    policy &= 0xFFFF
    ref = oracle.OracleTable(bins, B, d, policy, rng_seed=seed, cap=cap)
    ref.set_hash_family(family)
    t = ck.CuckooTable(bins, B, d, policy, seed=seed)
    t.set_param(ck.PARAM_CHAIN_CAP, cap)
    t.set_param(ck.PARAM_HASH_FAMILY, family)
    return ref, t, family


def fill_case(bins, B, d, load, seed):
    n = inputs.load_target(bins * B, load)
    keys, nxt = inputs.distinct_keys(n, seed)
    return keys, inputs.values_for(keys), nxt


def meta_fields(meta, B, d):
    meta = meta.astype(np.uint32)
    if d > 2:
        return {"rattle": ((meta >> 8) & 0xFF).astype(np.uint8), "spawn": ((meta >> 16) & 0xF).astype(np.uint8)}
    dup = np.zeros(len(meta) * B, dtype=np.uint8)
    for s in range(B):
        dup[s::B] = (meta >> (8 + s)) & 1
    return {"dup": dup, "spawn": ((meta >> 16) & 0xF).astype(np.uint8),
            "hit": ((meta >> 20) & 0xFF).astype(np.uint8)}


SERIAL_CASES = (
    [(1 << 14, 4, 2, p, 0.95) for p in TWO_CHOICE]            # 2^14 bins x 4 slots to 0.95
    + [(1 << 12, 8, 2, p, 0.97) for p in TWO_CHOICE]          # 8-slot bins to 0.97
    + [(1 << 14, 1, 3, ck.RANDOM, 0.90), (1 << 14, 1, 3, ck.RATTLE, 0.90),
       (1 << 14, 1, 4, ck.RANDOM, 0.96), (1 << 14, 1, 4, ck.RATTLE, 0.96),
       (1 << 14, 1, 3, ck.RATTLE | 0x10000, 0.90), (1 << 12, 4, 2, ck.QUEUE | 0x10000, 0.95),
       (1 << 14, 1, 3, ck.BFS, 0.88), (1 << 14, 1, 4, ck.SORTED, 0.95), (1 << 14, 1, 4, ck.HYBRID, 0.95)]
)
# 0x10000 in a case's policy selects the decorrelated hash family (test-only marker)
FAMILY_FLAG = 0x10000


@pytest.mark.parametrize("bins,B,d,policy,load", SERIAL_CASES,
                         ids=["%dx%d-d%d-%s-%.2f" % (b, s, d, pname(p), l) for b, s, d, p, l in SERIAL_CASES])
def test_serial_replay_matches_oracle_exactly(bins, B, d, policy, load):
    keys, vals, _ = fill_case(bins, B, d, load, 1)
    cap = 500
    ref, t, family = make_pair(bins, B, d, policy, 7, cap)
    policy &= 0xFFFF
    ost, oviewed, okicks = ref.insert(keys, vals, trace=True)
    viewed = torch.zeros(len(keys), dtype=torch.int32, device="cuda")
    st = t.insert(ck.as_u32_tensor(keys), ck.as_u32_tensor(vals), viewed=viewed, serial=True)
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy(), ost)
    assert np.array_equal(ck.u32_numpy(viewed), oviewed)
    slots, meta = t.export()
    e = ref.export()
    assert np.array_equal(slots, e["rec"])
    f = meta_fields(meta, B, d)
    if d > 2:
        if policy == ck.RATTLE:
            assert np.array_equal(f["rattle"], e["rattle"])
        if policy in (ck.SORTED, ck.HYBRID):
            assert np.array_equal(f["spawn"], e["spawn"])
    else:
        assert np.array_equal(f["dup"], e["dup"])
        if policy & 0xFF == ck.QUEUE:
            assert np.array_equal(f["hit"], e["hit"])
        if policy & 0xFF in (ck.SORTED, ck.HYBRID):
            assert np.array_equal(f["spawn"], e["spawn"])
    s, os_ = t.stats(), ref.stats()
    for k in ("inserts_ok", "inserts_failed", "bins_viewed", "kicks", "chain_max", "ghost_pairs_made",
              "dup_evictions", "size", "live_ghosts"):
        assert s[k] == os_[k], k
    assert s["bins_viewed_all"] == s["bins_viewed"] and s["aborts"] == 0
    # chain lengths of the successful insertions, bucketed as ck_chain_histogram
    want = np.zeros(ck.CHAIN_BUCKETS, dtype=np.uint64)
    for k in np.asarray(okicks)[ost == 0]:
        k = int(k)
        want[k if k < 32 else min(ck.CHAIN_BUCKETS - 1, 27 + k.bit_length() - 1)] += 1
    assert np.array_equal(t.chain_histogram(), want)
    check_table(slots, meta, bins, B, d, family)


SPAWN_K_CASES = [(1 << 14, 4, 2, ck.BFS, 0.95), (1 << 14, 4, 2, ck.SORTED | ck.GHOST, 0.97),
                 (1 << 12, 8, 2, ck.HYBRID, 0.97), (1 << 14, 1, 4, ck.SORTED, 0.95)]


@pytest.mark.parametrize("bins,B,d,policy,load", SPAWN_K_CASES,
                         ids=["%dx%d-d%d-%s-%.2f" % (b, s, d, pname(p), l) for b, s, d, p, l in SPAWN_K_CASES])
def test_serial_replay_in_rounds_matches_oracle(bins, B, d, policy, load):
    """Searches spawning 4 records a round (Sec. 5 prefetching): layout,
    statuses and bins viewed equal the oracle's."""
    keys, vals, _ = fill_case(bins, B, d, load, 1)
    ref, t, family = make_pair(bins, B, d, policy, 7, 500)
    ref.set_spawn_k(4)
    t.set_param(ck.PARAM_SPAWN_K, 4)
    ost, oviewed, _ = ref.insert(keys, vals, trace=True)
    viewed = torch.zeros(len(keys), dtype=torch.int32, device="cuda")
    st = t.insert(ck.as_u32_tensor(keys), ck.as_u32_tensor(vals), viewed=viewed, serial=True)
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy(), ost)
    assert np.array_equal(ck.u32_numpy(viewed), oviewed)
    slots, meta = t.export()
    assert np.array_equal(slots, ref.export()["rec"])
    check_table(slots, meta, bins, B, d, family)


CONCURRENT_CASES = (
    [(1 << 16, 4, 2, p, 0.95) for p in TWO_CHOICE]
    + [(1 << 15, 8, 2, p, 0.97) for p in (ck.RANDOM, ck.QUEUE, ck.SORTED | ck.GHOST)]
    + [(1 << 18, 1, 3, ck.RANDOM, 0.90), (1 << 16, 1, 4, ck.RATTLE, 0.96), (1 << 16, 1, 4, ck.RANDOM, 0.96),
       (1 << 18, 1, 3, ck.RATTLE | 0x10000, 0.90), (1 << 16, 1, 3, ck.BFS, 0.85),
       (1 << 16, 1, 4, ck.SORTED, 0.93), (1 << 16, 1, 4, ck.HYBRID, 0.93)]
)


@pytest.mark.parametrize("bins,B,d,policy,load", CONCURRENT_CASES,
                         ids=["%dx%d-d%d-%s-%.2f" % (b, s, d, pname(p), l) for b, s, d, p, l in CONCURRENT_CASES])
def test_concurrent_set_semantics_match_oracle(bins, B, d, policy, load):
    keys, vals, nxt = fill_case(bins, B, d, load, 3)
    cap = 4000 if (d > 2 and policy & 0xFF == ck.RANDOM) else 500
    ref, t, family = make_pair(bins, B, d, policy, 7, cap)
    policy &= 0xFFFF
    ost = ref.insert(keys, vals)
    assert (ost == 0).all()
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)
    # batches of 1/512 of the slots plus a ragged tail: the fraction of the
    # table in flight at once in the benchmark (~1.5e5 resident threads on a
    # 2^26-slot table)
    batch = max(512, (bins * B) // 512)
    sts = []
    for lo in range(0, len(keys), batch):
        sts.append(t.insert(kt[lo:lo + batch], vt[lo:lo + batch]))
    st = torch.cat(sts).cpu().numpy()
    assert (st == 0).all(), np.bincount(st)
    slots, meta = t.export()
    info = check_table(slots, meta, bins, B, d, family)
    assert info["size"] == len(keys)
    assert t.contents() == ref.contents()
    s, os_ = t.stats(), ref.stats()
    assert s["size"] == len(keys) and s["live_ghosts"] == info["ghost_pairs"]
    # bins viewed per insertion by the attempts that were applied: within
    # 10% of the serial oracle at the same load.  Counting every attempt
    # (abandoned ones, re-views, and the larger-budget retry of a search
    # that ran out of budget) the two-choice policies stay within 10% too.
    # d-ary walks and searches are heavy-tailed: a long random walk that
    # meets other insertions' claims is abandoned and drawn again (which
    # shortens the tail: its applied attempts may view a third fewer bins),
    # and a search retried with four times the budget adds its views; their
    # all-attempts band is 25% either way.
    assert s["bins_viewed_all"] >= s["bins_viewed"]
    applied = s["bins_viewed"] / os_["bins_viewed"]
    lo_applied = 0.50 if (d > 2 and policy & 0xFF == ck.RANDOM) else 0.90  # restarted walks are shorter
    assert lo_applied < applied < 1.10, (s["bins_viewed"], os_["bins_viewed"])
    ratio = s["bins_viewed_all"] / os_["bins_viewed"]
    lo, hi = (0.75, 1.25) if d > 2 else (0.90, 1.10)
    assert lo < ratio < hi, (s["bins_viewed_all"], s["bins_viewed"], os_["bins_viewed"], s["aborts"])
    # lookups, 50% present / 50% absent
    probe, expect = inputs.lookup_keys(keys, 1 << 16, 9, 0.5, next_start=nxt)
    v, fnd = t.lookup(ck.as_u32_tensor(probe))
    ov, of = ref.lookup(probe)
    assert np.array_equal(fnd.cpu().numpy(), of) and np.array_equal(of, expect)
    assert np.array_equal(ck.u32_numpy(v), ov)
    # deletes of present keys and of absent keys
    dk = np.concatenate([inputs.delete_keys(keys, len(keys) // 8, 4), probe[expect == 0][:1000]])
    fd = t.delete(ck.as_u32_tensor(dk)).cpu().numpy()
    assert np.array_equal(fd, ref.delete(dk))
    assert t.contents() == ref.contents()
    slots, meta = t.export()
    assert check_table(slots, meta, bins, B, d, family)["size"] == ref.stats()["size"]
    # re-insert half of the deleted keys after the deletes
    back = dk[: len(keys) // 16]
    st2 = t.insert(ck.as_u32_tensor(back), ck.as_u32_tensor(inputs.values_for(back))).cpu().numpy()
    assert (st2 == 0).all() and (ref.insert(back, inputs.values_for(back)) == 0).all()
    assert t.contents() == ref.contents()


def test_edge_cases_empty_ragged_reserved():
    t = ck.CuckooTable(1 << 10, 4, 2, ck.RANDOM, seed=1)
    ref = oracle.OracleTable(1 << 10, 4, 2, ck.RANDOM, rng_seed=1)
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    t.insert(empty, empty)
    t.lookup(empty)
    t.delete(empty)
    keys, _ = inputs.distinct_keys(3000, 17)
    keys[5] = 0xFFFFFFFF
    vals = inputs.values_for(keys)
    for lo, hi in ((0, 1), (1, 32), (32, 33), (33, 290), (290, 3000)):  # ragged batch sizes
        st = t.insert(ck.as_u32_tensor(keys[lo:hi]), ck.as_u32_tensor(vals[lo:hi])).cpu().numpy()
        ost = ref.insert(keys[lo:hi], vals[lo:hi])
        assert np.array_equal(st == 3, ost == 3)
        assert (st[ost != 3] == 0).all()
    assert t.contents() == ref.contents()
    v, f = t.lookup(ck.as_u32_tensor(np.array([0xFFFFFFFF, keys[0], keys[5]], dtype=np.uint32)))
    assert list(f.cpu().numpy()) == [0, 1, 0]


@pytest.mark.parametrize("policy", [ck.RANDOM, ck.QUEUE, ck.BFS, ck.SORTED | ck.GHOST])
def test_overfull_table_failures_are_clean(policy):
    """A table pushed past its capacity: failed keys are absent, every other
    key is present once, and the serial replay fails exactly the oracle's keys."""
    bins, B = 256, 4
    keys, _ = inputs.distinct_keys(bins * B + 200, 23)
    vals = inputs.values_for(keys)
    ref = oracle.OracleTable(bins, B, 2, policy, rng_seed=2, cap=100)
    ost = ref.insert(keys, vals)
    ts = ck.CuckooTable(bins, B, 2, policy, seed=2)
    ts.set_param(ck.PARAM_CHAIN_CAP, 100)
    st = ts.insert(ck.as_u32_tensor(keys), ck.as_u32_tensor(vals), serial=True).cpu().numpy()
    assert np.array_equal(st, ost) and (ost == 1).any()
    assert ts.contents() == ref.contents()
    tc = ck.CuckooTable(bins, B, 2, policy, seed=2)
    tc.set_param(ck.PARAM_CHAIN_CAP, 100)
    st = tc.insert(ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)).cpu().numpy()
    got = tc.contents()
    ok = {int(k): int(v) for k, v, s in zip(keys, vals, st) if s == 0}
    assert got == ok
    slots, meta = tc.export()
    check_table(slots, meta, bins, B, 2)
    assert tc.stats()["size"] == len(ok)
