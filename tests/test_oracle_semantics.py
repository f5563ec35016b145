"""Set semantics, failure atomicity, invariants and the exact propositions of
the paper, checked on the oracle."""
import numpy as np
import pytest

import oracle
from paper_1605_05236_gb300 import inputs

TWO_CHOICE = [oracle.RANDOM, oracle.BFS, oracle.SORTED, oracle.QUEUE, oracle.HYBRID,
              oracle.RANDOM | oracle.GHOST, oracle.BFS | oracle.GHOST,
              oracle.SORTED | oracle.GHOST, oracle.QUEUE | oracle.GHOST, oracle.HYBRID | oracle.GHOST]
DARY = [(3, oracle.RANDOM), (4, oracle.RANDOM), (3, oracle.RATTLE), (4, oracle.RATTLE),
        (3, oracle.BFS), (4, oracle.SORTED), (4, oracle.HYBRID)]


def configs():
    for B in (4, 8):
        for p in TWO_CHOICE:
            yield (2, B, p)
    for d, p in DARY:
        yield (d, 1, p)


@pytest.mark.parametrize("d,B,policy", list(configs()))
def test_set_semantics_against_a_dict(d, B, policy):
    """The final key->value map and every lookup/delete result equal those of
    a Python dict fed the same operations (Sec. 1: constant-time reads and
    deletes of whatever the table holds)."""
    bins = 256 if d == 2 else 1024
    slots = bins * B
    t = oracle.OracleTable(bins, B, d, policy, rng_seed=3, cap=500)
    ref = {}
    keys, pos = inputs.distinct_keys(int(slots * 0.85), 11)
    vals = inputs.values_for(keys)
    rng = np.random.default_rng(0)
    for lo in range(0, len(keys), 200):
        k, v = keys[lo:lo + 200], vals[lo:lo + 200]
        st = t.insert(k, v)
        for kk, vv, s in zip(k, v, st):
            if s == oracle.ST_OK:
                ref[int(kk)] = int(vv)
        bad, msg = t.check_invariants()
        assert bad == 0, msg
        if lo % 600 == 0 and ref:
            live = np.array(list(ref), dtype=np.uint32)
            dk = live[rng.choice(len(live), min(40, len(live)), replace=False)]
            absent, pos = inputs.distinct_keys(10, 12, exclude=keys, start=pos)
            dk = np.concatenate([dk, absent])
            found = t.delete(dk)
            for kk, f in zip(dk, found):
                assert f == (int(kk) in ref)
                ref.pop(int(kk), None)
            bad, msg = t.check_invariants()
            assert bad == 0, msg
    probe = np.concatenate([keys, inputs.distinct_keys(500, 13, exclude=keys)[0]])
    v, f = t.lookup(probe)
    for kk, vv, ff in zip(probe, v, f):
        if int(kk) in ref:
            assert ff == 1 and vv == ref[int(kk)]
        else:
            assert ff == 0
    assert t.contents() == ref
    assert t.stats()["size"] == len(ref)


@pytest.mark.parametrize("d,B,policy", list(configs()))
def test_failed_insert_leaves_table_unchanged(d, B, policy):
    """A chain that reaches its cap is never applied: the table (records,
    duplicate marks, hit counters, rattle counters) is exactly as before
    (system-transaction kick-outs are planned first, Sec. 8)."""
    bins = 64 if d == 2 else 256
    t = oracle.OracleTable(bins, B, d, policy, rng_seed=5, cap=3)
    keys, _ = inputs.distinct_keys(bins * B, 21)
    vals = inputs.values_for(keys)
    failures = 0
    for k, v in zip(keys, vals):
        before = t.export()
        st = t.insert([k], [v])
        if st[0] == oracle.ST_FAILED:
            failures += 1
            after = t.export()
            for name in ("rec", "dup", "rattle", "hit"):
                assert np.array_equal(before[name], after[name]), name
            assert int(k) not in t.contents()
    assert failures > 0


@pytest.mark.parametrize("policy", [oracle.RANDOM | oracle.GHOST, oracle.BFS | oracle.GHOST,
                                    oracle.SORTED | oracle.GHOST, oracle.QUEUE | oracle.GHOST])
@pytest.mark.parametrize("B", [4, 8])
def test_prop_4_1_chains_end_in_duplicate_bins(policy, B):
    """Prop. 4.1: in an insert-only ghost table the last bin of every kick-out
    chain held a duplicate before the chain."""
    bins = 1024
    t = oracle.OracleTable(bins, B, 2, policy, rng_seed=1, cap=2000)
    keys, _ = inputs.distinct_keys(int(bins * B * 0.97), 31)
    t.insert(keys, inputs.values_for(keys))
    s = t.stats()
    assert s["prop41_checks"] > 100
    assert s["prop41_violations"] == 0


@pytest.mark.parametrize("ghost", [0, oracle.GHOST])
def test_queue_bins_fill_in_hit_order(ghost):
    """Sec. 6: with hit counters a bin is a queue: in an insert-only table a
    bin with hit counter h < B holds exactly slots 0..h-1, and a bin that has
    taken B or more insertions is full."""
    B, bins = 4, 2048
    t = oracle.OracleTable(bins, B, 2, oracle.QUEUE | ghost, rng_seed=1, cap=500)
    keys, _ = inputs.distinct_keys(int(bins * B * 0.9), 41)
    t.insert(keys, inputs.values_for(keys))
    e = t.export()
    occ = (e["rec"] != np.uint64(0xFFFFFFFFFFFFFFFF)).reshape(bins, B)
    for b in range(bins):
        h = int(e["hit"][b])
        if h < B:
            assert occ[b, :h].all() and not occ[b, h:].any()
        else:
            assert occ[b].all()


@pytest.mark.parametrize("policy", [oracle.SORTED, oracle.HYBRID])
def test_spawn_counts_stay_within_four_bits(policy):
    """Sec. 5: spawn counts saturate at 15."""
    t = oracle.OracleTable(512, 4, 2, policy, rng_seed=1, cap=500)
    keys, _ = inputs.distinct_keys(int(512 * 4 * 0.975), 51)
    t.insert(keys, inputs.values_for(keys))
    assert t.export()["spawn"].max() <= 15


def test_rattle_tie_reading_is_a_switch():
    """Both readings of a rattle tie give valid tables; they differ in layout."""
    keys, _ = inputs.distinct_keys(900, 61)
    outs = []
    for tie_resident in (False, True):
        t = oracle.OracleTable(1024, 1, 4, oracle.RATTLE, cap=500)
        t.set_rattle_tie_resident(tie_resident)
        st = t.insert(keys, inputs.values_for(keys))
        assert (st == 0).all() and t.check_invariants()[0] == 0
        outs.append(t.export()["rec"])
    assert not np.array_equal(outs[0], outs[1])


def test_reserved_key_rejected():
    t = oracle.OracleTable(64, 4, 2, oracle.RANDOM)
    st = t.insert([0xFFFFFFFF, 5], [1, 2])
    assert list(st) == [oracle.ST_INVALID, oracle.ST_OK]
    assert t.contents() == {5: 2}


@pytest.mark.parametrize("d,B,policy", [(2, 4, oracle.QUEUE), (2, 4, oracle.SORTED | oracle.GHOST),
                                        (2, 8, oracle.RANDOM | oracle.GHOST), (3, 1, oracle.RATTLE),
                                        (4, 1, oracle.HYBRID)])
def test_upsert_against_a_dict(d, B, policy):
    """Upsert lifts the absent-key assumption of Sec. 3: present keys get the
    new value (every copy of a ghost pair), absent keys are inserted."""
    bins = 256 if B > 1 else 1024
    t = oracle.OracleTable(bins, B, d, policy, rng_seed=3, cap=500)
    rng = np.random.default_rng(7)
    pool, _ = inputs.distinct_keys(int(bins * B * 0.8), 61)
    want = {}
    for rnd in range(6):
        ks = rng.choice(pool, 300, replace=False).astype(np.uint32)
        vs = rng.integers(0, 2**32 - 1, len(ks), dtype=np.uint64).astype(np.uint32)
        present = np.array([int(k) in want for k in ks])
        st = t.upsert(ks, vs)
        assert (st[present] == oracle.ST_UPDATED).all()
        assert (st[~present] == oracle.ST_OK).all()
        for k, v in zip(ks, vs):
            want[int(k)] = int(v)
        assert t.contents() == want
        assert t.check_invariants()[0] == 0
    s = t.stats()
    assert s["size"] == len(want)
    e = t.export()
    if policy & oracle.GHOST:  # both copies of a ghost pair carry the new value
        recs = e["rec"][e["dup"] == 1]
        for r in recs:
            assert (int(r) & 0xFFFFFFFF) == want[int(r) >> 32]


@pytest.mark.parametrize("policy", [oracle.QUEUE, oracle.RANDOM | oracle.GHOST, oracle.RATTLE])
def test_threaded_lookups_and_deletes_equal_the_serial_ones(policy):
    """The all-core legs of the CPU baseline split a batch over host
    threads; every result, the counters and the remaining table equal the
    one-thread calls."""
    d, B = (3, 1) if policy == oracle.RATTLE else (2, 4)
    bins = 1 << 12
    n = inputs.load_target(bins * B, 0.85)
    keys, nxt = inputs.distinct_keys(n, 4)
    vals = inputs.values_for(keys)
    a = oracle.OracleTable(bins, B, d, policy, rng_seed=1, cap=500)
    b = oracle.OracleTable(bins, B, d, policy, rng_seed=1, cap=500)
    a.insert(keys, vals)
    b.insert(keys, vals)
    lk, _ = inputs.lookup_keys(keys, 20000, 4, 0.5, next_start=nxt)
    v1, f1 = a.lookup(lk)
    v2, f2, used = b.lookup_threads(lk, 5)
    assert used == 5 and np.array_equal(v1, v2) and np.array_equal(f1, f2)
    dk = inputs.delete_keys(keys, n // 3, 4)
    g1 = a.delete(dk)
    g2, used = b.delete_threads(dk, 5)
    assert used == 5 and np.array_equal(g1, g2)
    assert a.stats() == b.stats() and a.contents() == b.contents()
    assert b.check_invariants()[0] == 0
