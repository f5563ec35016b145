"""Parity at the full workload sizes, in the launch configurations bench.py
times.  The main step (a 2^24-bin x 4-slot table filled from empty to load
0.95 with queue-kicking in 61 calls of 2^20 keys on one stream, launches
overlapping, then 2^26 lookups at 50% hits and 2^22 deletes of present
keys), the same on 2^23 x 8 filled to 0.99 and with random kicking: the
oracle fills the same table serially, and the concurrent GPU fill must hold
exactly the same key -> value set (compared over every record), satisfy
every table invariant, view bins within 10% of the serial oracle, answer
every lookup as the workload fixes it, and delete every deleted key.  The
single-slot d-ary fills, the L2-resident small table and the 4096-table
batched fill follow."""
import os
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_1605_05236_gb300 import ck, inputs

from table_checks import check_table

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

pytestmark = pytest.mark.gpu

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def _sorted_records(slots):
    r = slots[slots != EMPTY]
    r.sort()
    return r


# (bins, slots per bin, policy, load): the benchmark's own fill, the 8-slot
# table of the same slot count filled to 0.99, and random kicking on the
# benchmark's table; each in the benchmark's launch configuration
FULL = [(bench.BINS, bench.B, ck.QUEUE, bench.LOAD), (1 << 23, 8, ck.QUEUE, 0.99),
        (bench.BINS, bench.B, ck.RANDOM, bench.LOAD)]


def _full_workload(bins, b, load):
    if (bins, b, load) == (bench.BINS, bench.B, bench.LOAD):
        return bench.workload(bench.rank_seed(0))
    seed = bench.rank_seed(0)
    keys, nxt = inputs.distinct_keys(inputs.load_target(bins * b, load), seed)
    lk, expect = inputs.lookup_keys(keys, bench.N_LOOKUP, seed, 0.5, next_start=nxt)
    return keys, inputs.values_for(keys), lk, expect, inputs.delete_keys(keys, bench.N_DELETE, seed)


@pytest.mark.timeout(900)
@pytest.mark.parametrize("bins,b,policy,load", FULL,
                         ids=["2e%dx%d-%s-%.2f" % (int(np.log2(c[0])), c[1], {ck.QUEUE: "queue", ck.RANDOM: "random"}[c[2]],
                                                   c[3]) for c in FULL])
def test_full_size_fill_lookups_deletes_match_the_oracle(bins, b, policy, load):
    keys, vals, lk, expect, dk = _full_workload(bins, b, load)
    n = len(keys)
    t = ck.CuckooTable(bins, b, 2, policy, seed=bench.rank_seed(0))
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    for lo in range(0, n, bench.BATCH):  # the benchmark's calls, back to back on one stream
        t.insert_batch(kt[lo:lo + bench.BATCH], vt[lo:lo + bench.BATCH], st[lo:lo + bench.BATCH], s)
    torch.cuda.synchronize()
    assert (st == 0).all().item(), np.bincount(st.cpu().numpy())
    slots, meta = t.export()
    info = check_table(slots, meta, bins, b, 2)
    assert info["size"] == n and info["ghost_pairs"] == 0
    gs = t.stats()
    assert gs["size"] == n and gs["inserts_ok"] == n

    ref = oracle.OracleTable(bins, b, 2, policy, rng_seed=bench.rank_seed(0), cap=500)
    ost = ref.insert(keys, vals)
    assert (ost == 0).all()
    assert np.array_equal(_sorted_records(slots), _sorted_records(ref.export()["rec"]))
    ov = ref.stats()["bins_viewed"]
    # bins viewed per insertion: the applied attempts, and every attempt
    # (with those abandoned after claim conflicts), within 10% of the oracle
    assert 0.90 < gs["bins_viewed"] / ov < 1.10, (gs["bins_viewed"], ov)
    assert 0.90 < gs["bins_viewed_all"] / ov < 1.10, (gs["bins_viewed_all"], ov)
    del ref

    v, f = t.lookup(ck.as_u32_tensor(lk))
    f = f.cpu().numpy().astype(bool)
    assert np.array_equal(f, expect.astype(bool))
    assert np.array_equal(ck.u32_numpy(v)[f], inputs.values_for(lk[f]))
    fd = t.delete(ck.as_u32_tensor(dk)).cpu().numpy()
    assert (fd == 1).all()
    _, f2 = t.lookup(ck.as_u32_tensor(dk))
    assert not f2.cpu().numpy().any()
    assert t.stats()["size"] == n - len(dk)
    t.close()


def test_l2_resident_small_table_matches_the_oracle():
    """The small-table workload at its full size and launch configuration:
    2^14 bins x 4 slots (512 KiB of slots, L2-resident), 62,259 keys of seed
    1 inserted by one call with random kicking, chain cap 500, then 65,536
    lookups (half present, half absent, shuffled).  The concurrent GPU fill
    holds exactly the serial oracle's key -> value set and answers every
    lookup as the oracle does."""
    keys, vals, lk, expect = bench.small_table_workload()
    t = ck.CuckooTable(bench.SMALL_BINS, bench.B, 2, ck.RANDOM, seed=1)
    t.set_param(ck.PARAM_CHAIN_CAP, 500)
    st = t.insert(ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)).cpu().numpy()
    ref = oracle.OracleTable(bench.SMALL_BINS, bench.B, 2, oracle.RANDOM, rng_seed=1, cap=500)
    ost = ref.insert(keys, vals)
    assert (ost == 0).all() and (st == 0).all(), np.bincount(st)
    assert t.contents() == ref.contents()
    slots, meta = t.export()
    assert check_table(slots, meta, bench.SMALL_BINS, bench.B, 2)["size"] == len(keys)
    v, f = t.lookup(ck.as_u32_tensor(lk))
    ov, of = ref.lookup(lk)
    assert np.array_equal(f.cpu().numpy(), of) and np.array_equal(of, expect)
    assert np.array_equal(ck.u32_numpy(v), ov)


# (choices, load, policy, hash family, chain cap, name of the serial oracle's
# failure count in tests/golden/full_size_failures.json): the single-slot
# workloads at their full size, in the bench's launch configuration (2^20-key
# calls on one stream, launches overlapping)
DARY_FULL = [(3, 0.90, ck.RANDOM, 0, 4096, None), (4, 0.96, ck.RATTLE, 1, 500, "rattle_d4_0.96_hash1")]


@pytest.mark.timeout(900)
@pytest.mark.parametrize("d,load,policy,family,cap,oname", DARY_FULL,
                         ids=["d%d-%.2f-%x-hash%d" % (c[0], c[1], c[2], c[3]) for c in DARY_FULL])
def test_dary_full_size_fill_and_lookups(d, load, policy, family, cap, oname):
    """2^26 single-slot bins filled to 0.90 (d = 3, random kicking) or 0.96
    (d = 4, rattle-kicking) in 2^20-key calls, then 2^26 lookups at 50% hits.
    Properties that hold at any size, checked over every record: every key
    inserted except at most as many as the serial oracle fails at the same
    cap (none for the random walks; 3 of 64.4 M for rattle-kicking, whose
    walks reach the cap of 500 tries), each key reported FAILED absent, every
    other key found with its value, every absent key missed, each record in
    one of its d bins, no key stored twice, no claim left set, the size
    counter exact."""
    bins = 1 << 26
    n = inputs.load_target(bins, load)
    keys, nxt = inputs.distinct_keys(n, 2)
    vals = inputs.values_for(keys)
    t = ck.CuckooTable(bins, 1, d, policy, seed=1)
    t.set_param(ck.PARAM_CHAIN_CAP, cap)
    t.set_param(ck.PARAM_HASH_FAMILY, family)
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    for lo in range(0, n, bench.BATCH):
        t.insert_batch(kt[lo:lo + bench.BATCH], vt[lo:lo + bench.BATCH], st[lo:lo + bench.BATCH], s)
    torch.cuda.synchronize()
    sn = st.cpu().numpy()
    allowed = bench.oracle_full_size_failures()[oname]["failed"] if oname else 0
    failed = sn == 1
    assert ((sn == 0) | failed).all(), np.bincount(sn)
    assert failed.sum() <= allowed, (failed.sum(), allowed)
    assert t.stats()["size"] == n - failed.sum()
    lk, expect = inputs.lookup_keys(keys, 1 << 26, 2, 0.5, next_start=nxt)
    if failed.any():  # a key left out is absent
        expect = expect & ~np.isin(lk, keys[failed]).astype(np.uint8)
        _, ff = t.lookup(ck.as_u32_tensor(keys[failed]))
        assert not ff.cpu().numpy().any()
    v, f = t.lookup(ck.as_u32_tensor(lk))
    f = f.cpu().numpy()
    assert np.array_equal(f, expect)
    hit = f.astype(bool)
    assert np.array_equal(ck.u32_numpy(v)[hit], inputs.values_for(lk[hit]))
    slots, meta = t.export()
    info = check_table(slots, meta, bins, 1, d, family)
    assert info["size"] == n - failed.sum()
    t.close()


@pytest.mark.timeout(900)
def test_batched_full_size_matches_oracle_in_both_forms():
    """The batched workload at its full size and launch configuration: 4096
    tables (bins log-uniform in [2^10, 2^18] of seed 7, 4 or 8 slots, keys
    of seed 8 + table id, 1,065,803,986 keys in all) filled to 0.95 with
    queue-kicking by the autotuned persistent launch and by one launch per
    table, each replayed from its captured graph (clear + fill).  In both
    forms every key of every table is inserted and found with its value and
    the size counters are exact; sampled tables (the smallest, the largest
    and some in between) hold exactly the serial oracle's map, pass every
    table invariant and answer lookups half of absent keys as the oracle."""
    from paper_1605_05236_gb300 import autotune
    from paper_1605_05236_gb300 import multi as M
    import ctypes
    bins, slots = inputs.multi_shapes(4096, seed=7)
    keys, vals, n_keys = inputs.multi_keys(bins, slots, 0.95, seed0=8)
    n = len(keys)
    offs = np.concatenate([[0], np.cumsum(n_keys)[:-1]]).astype(np.int64)
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    tab = torch.from_numpy(np.repeat(np.arange(4096, dtype=np.int32), n_keys.astype(np.int64))).cuda()
    stream = torch.cuda.current_stream()
    mt = M.MultiTable(bins, slots, n_keys, ck.QUEUE, seed=1)
    autotune.tune(mt, kt, vt, st, stream)
    size_order = np.argsort(bins * slots, kind="stable")
    sample = sorted(set(size_order[:6].tolist() + size_order[-6:].tolist() + size_order[::512].tolist()))
    refs = {}
    for i in sample:
        lo, m = int(offs[i]), int(n_keys[i])
        ki, nxt = inputs.distinct_keys(m, 8 + i)
        assert np.array_equal(ki, keys[lo:lo + m])
        ref = oracle.OracleTable(int(bins[i]), int(slots[i]), 2, oracle.QUEUE, rng_seed=1 + i, cap=500)
        assert (ref.insert(ki, vals[lo:lo + m]) == 0).all()
        lk, expect = inputs.lookup_keys(ki, 4096, 8 + i, 0.5, next_start=nxt)
        ov, of = ref.lookup(lk)
        assert np.array_equal(of, expect)
        refs[i] = (ref.contents(), lk, of, ov)
        del ref
    for per_table in (False, True):
        st.fill_(255)
        g = mt.capture(kt, vt, st, per_table=per_table, clear=True, stream=stream)
        g.launch(stream)
        torch.cuda.synchronize()
        assert bool((st == 0).all().item()), np.bincount(st.cpu().numpy())
        s = mt.stats()
        assert s["size"] == n and s["inserts_ok"] == n
        v, f = mt.lookup(tab, kt)
        assert bool((f == 1).all().item()) and torch.equal(v, vt)
        for i in sample:
            want, lk, of, ov = refs[i]
            assert mt.contents(i) == want, (per_table, i)
            sl = np.zeros(int(bins[i]) * int(slots[i]), dtype=np.uint64)
            meta = np.zeros(int(bins[i]), dtype=np.uint32)
            M._lib().ck_multi_export(mt._h, i, sl.ctypes.data_as(ctypes.c_void_p), meta.ctypes.data_as(ctypes.c_void_p))
            assert check_table(sl, meta, int(bins[i]), int(slots[i]), 2)["size"] == int(n_keys[i])
            lt = torch.full((len(lk),), i, dtype=torch.int32, device="cuda")
            gv, gf = mt.lookup(lt, ck.as_u32_tensor(lk))
            gf = gf.cpu().numpy()
            assert np.array_equal(gf, of)
            assert np.array_equal(ck.u32_numpy(gv)[gf == 1], ov[gf == 1])
        g.close()
    mt.close()
