"""The seeded input generator (C) equals its plain restatement, and its
outputs have the properties the recipe promises."""
import numpy as np
import pytest

from paper_1605_05236_gb300 import inputs


def test_keys_match_plain_restatement():
    for seed, start, n in ((1, 0, 500), (7, 123, 300), (2 ** 63 + 5, 0, 50)):
        got, nxt = inputs.distinct_keys(n, seed, start=start)
        ref, rnxt = inputs.ref_distinct_keys(n, seed, start=start)
        assert np.array_equal(got, ref) and nxt == rnxt
    base, nxt = inputs.distinct_keys(400, 3)
    got, n2 = inputs.distinct_keys(200, 3, exclude=base, start=nxt)
    ref, r2 = inputs.ref_distinct_keys(200, 3, exclude=base, start=nxt)
    assert np.array_equal(got, ref) and n2 == r2
    assert not np.isin(got, base).any()


def test_permutation_matches_plain_restatement():
    for n, k, seed in ((1, None, 1), (2, None, 2), (17, None, 3), (100, 10, 4), (1000, None, 5)):
        assert np.array_equal(inputs.permutation(n, seed, k), inputs.ref_permutation(n, seed, k))
    p = inputs.permutation(5000, 9)
    assert np.array_equal(np.sort(p), np.arange(5000))


def test_keys_distinct_and_uniform():
    keys, _ = inputs.distinct_keys(200000, 11)
    assert len(np.unique(keys)) == len(keys)
    assert not (keys == 0xFFFFFFFF).any()
    hist = np.bincount(keys >> 28, minlength=16)
    assert hist.min() > 0.9 * len(keys) / 16


def test_lookup_and_delete_sets():
    keys, nxt = inputs.distinct_keys(10000, 21)
    probe, expect = inputs.lookup_keys(keys, 4000, 5, 0.5, next_start=nxt)
    assert expect.sum() == 2000
    assert np.isin(probe[expect == 1], keys).all()
    assert not np.isin(probe[expect == 0], keys).any()
    assert len(np.unique(probe)) == len(probe)
    dk = inputs.delete_keys(keys, 1000, 5)
    assert len(np.unique(dk)) == 1000 and np.isin(dk, keys).all()


def test_multi_shapes_in_range():
    bins, slots = inputs.multi_shapes(512, seed=7, lo_log2=10, hi_log2=18)
    assert bins.min() >= 1 << 10 and bins.max() < 1 << 18
    assert set(np.unique(slots)) == {4, 8}
    keys, vals, n_keys = inputs.multi_keys(bins[:8], slots[:8], 0.95)
    assert len(keys) == int(n_keys.sum())
    off = 0
    for b, s, n in zip(bins[:8], slots[:8], n_keys):
        assert int(n) == inputs.load_target(int(b) * int(s), 0.95)
        assert len(np.unique(keys[off:off + int(n)])) == int(n)
        off += int(n)


@pytest.mark.parametrize("mix", [(75, 20, 5), (50, 25, 25), (0, 1, 0)])
def test_serving_trace_fixes_every_result(mix):
    pre, _ = inputs.distinct_keys(20000, 11)
    tr = inputs.serving_trace(pre, 300, mix, max_log2=8)
    op = np.repeat(tr["op"], tr["n_keys"].astype(np.int64))
    keys = tr["keys"]
    assert len(keys) == int(tr["n_keys"].sum()) and np.all(np.diff(tr["arrive_ns"]) >= 0)
    assert np.array_equal(tr["key_off"][1:], np.cumsum(tr["n_keys"])[:-1])
    preset = set(pre.tolist())
    stable, deletable = set(pre[:10000].tolist()), set(pre[10000:].tolist())
    look, ins, dele = keys[op == 0], keys[op == 1], keys[op == 2]
    # lookups: present ones from the never-deleted half, absent ones never inserted
    for k, e in zip(look, tr["expect"][op == 0]):
        assert (int(k) in stable) if e == 1 else (int(k) not in preset and int(k) not in set(ins.tolist()))
    # inserts are fresh and distinct; deletes hit the other half, each once
    assert not (set(ins.tolist()) & preset) and len(np.unique(ins)) == len(ins)
    assert set(dele.tolist()) <= deletable and len(np.unique(dele)) == len(dele)
    assert (tr["expect"][op != 0] == 1).all()
    assert np.array_equal(tr["vals"], inputs.values_for(keys))
