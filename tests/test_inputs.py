"""The seeded input generator (C) equals its plain restatement, and its
outputs have the properties the recipe promises."""
import numpy as np

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
