"""Soft pins: the ratios and counts the paper states in its prose (its
figures are not available), reproduced by the oracle on the paper's set-up
(2^13 bins of 4 slots filled to 97.5%, Sec. 3; 4-ary tables of 2^13
single-slot bins, Sec. 3 and Sec. 7) with fewer trials.  Each bound is the
paper's number with a tolerance; where a reading of the paper was needed it
is named."""
import numpy as np
import pytest

import oracle
from paper_1605_05236_gb300 import inputs

NB, B = 1 << 13, 4
N975 = inputs.load_target(NB * B, 0.975)


def curve(policy, trials=3, lo=0.97, hi=0.975, nb=NB, b=B):
    n = inputs.load_target(nb * b, hi)
    v_sum = k_sum = cnt = 0
    for tr in range(trials):
        keys, _ = inputs.distinct_keys(n, 700 + tr)
        t = oracle.OracleTable(nb, b, 2, policy, rng_seed=tr, cap=100000)
        st, viewed, kicks = t.insert(keys, inputs.values_for(keys), trace=True)
        assert (st == 0).all()
        load = np.arange(n) / (nb * b)
        m = (load >= lo) & (load < hi)
        v_sum += viewed[m].sum()
        k_sum += kicks[m].sum()
        cnt += m.sum()
    return v_sum / cnt, k_sum / cnt


@pytest.fixture(scope="module")
def fig_a():
    pols = {"random": oracle.RANDOM, "bfs": oracle.BFS, "sorted": oracle.SORTED,
            "queue": oracle.QUEUE, "random+ghost": oracle.RANDOM | oracle.GHOST,
            "bfs+ghost": oracle.BFS | oracle.GHOST, "sorted+ghost": oracle.SORTED | oracle.GHOST,
            "hybrid": oracle.HYBRID}
    return {k: curve(p) for k, p in pols.items()}


def test_random_and_bfs_equally_bad_at_high_density(fig_a):
    # Sec. 1: at high densities random kicking and BFS view about as many bins.
    r, b = fig_a["random"][0], fig_a["bfs"][0]
    assert 0.5 < r / b < 2.0


def test_sorted_search_gain(fig_a):
    # Sec. 5: sorted search views up to ~8x fewer bins than BFS at high density
    # (reading: sort keys fixed when a record joins the list).
    assert fig_a["bfs"][0] / fig_a["sorted"][0] > 4.0


def test_sorted_plus_ghost_gain(fig_a):
    # Sec. 1: sorted search with ghost insertions is about ten times better
    # than the standard schemes at high density.
    assert fig_a["random"][0] / fig_a["sorted+ghost"][0] > 6.0


def test_ghost_gain_on_random(fig_a):
    # Sec. 4: ghost insertions improve random kicking by roughly 2.5x.
    g = fig_a["random"][0] / fig_a["random+ghost"][0]
    assert 2.0 < g < 4.5


def test_ghost_helps_bfs(fig_a):
    # Sec. 4: ghost insertions help BFS too (the paper: a bit under 2x).
    assert fig_a["bfs"][0] / fig_a["bfs+ghost"][0] > 1.5


def test_queue_beats_random(fig_a):
    # Sec. 6: queue-kicking gives far shorter chains than random kicking at high density.
    assert fig_a["queue"][0] < fig_a["random"][0] / 2


def test_hybrid_between_sorted_and_bfs(fig_a):
    # Sec. 5 (end): the sorted search / BFS hybrid performs between sorted
    # search and BFS, and its depth-first order keeps its chains as short as
    # BFS's.
    assert fig_a["sorted"][0] < fig_a["hybrid"][0] < fig_a["bfs"][0]
    assert fig_a["hybrid"][1] <= fig_a["bfs"][1] * 1.05


def test_search_chains_an_order_shorter(fig_a):
    # Sec. 5 (Fig. D): at 97.5% search-based chains are ~10x shorter than walks.
    walk = min(fig_a["random"][1], fig_a["random+ghost"][1])
    for s in ("bfs", "bfs+ghost", "sorted+ghost"):
        assert walk / fig_a[s][1] > 8.0, s


def test_kickouts_per_bin_queue_to_97():
    # Sec. 6 footnote: about 2.07 kick-outs per bin when filling B=4 bins to
    # 97%.  Reading: the count matches queue-kicking (with hit balancing);
    # random kicking gives several times more.
    n = inputs.load_target(NB * B, 0.97)
    per_bin = []
    for tr in range(3):
        keys, _ = inputs.distinct_keys(n, 800 + tr)
        t = oracle.OracleTable(NB, B, 2, oracle.QUEUE, rng_seed=tr, cap=100000)
        t.insert(keys, inputs.values_for(keys))
        per_bin.append(t.stats()["kicks"] / NB)
    assert abs(np.mean(per_bin) / 2.07 - 1) < 0.2


def dary_fill(policy, load=0.95, trials=3, nb=NB):
    n = inputs.load_target(nb, load)
    out = []
    for tr in range(trials):
        keys, _ = inputs.distinct_keys(n, 900 + tr)
        t = oracle.OracleTable(nb, 1, 4, policy, rng_seed=tr, cap=100000)
        st, viewed, kicks = t.insert(keys, inputs.values_for(keys), trace=True)
        assert (st == 0).all()
        out.append((t, viewed))
    return out


def test_four_ary_random_bins_per_record():
    # Sec. 7: filling a 4-ary table to 95% with random kicking, each record
    # visits about 5.6 bins (within 15%).
    r = np.mean([v.mean() for _, v in dary_fill(oracle.RANDOM)])
    assert abs(r / 5.6 - 1) < 0.15


def test_rattle_hash_functions_used():
    # Sec. 7: with rattle-kicking to 95% records use about 3.3 hash functions.
    used = []
    for t, _ in dary_fill(oracle.RATTLE):
        e = t.export()
        occ = e["rec"] != np.uint64(0xFFFFFFFFFFFFFFFF)
        used.append(e["rattle"][occ].mean())
    assert abs(np.mean(used) / 3.3 - 1) < 0.1


def test_rattle_near_ideal_below_85():
    # Sec. 7: below 85% density rattle-kicking chains are close to 1/(1-delta)
    # (bins viewed per insertion at density delta).
    runs = dary_fill(oracle.RATTLE, load=0.85, trials=2)
    n = inputs.load_target(NB, 0.85)
    load = np.arange(n) / NB
    for lo, hi in ((0.5, 0.6), (0.7, 0.8)):
        m = (load >= lo) & (load < hi)
        got = np.mean([v[m].mean() for _, v in runs])
        ideal = np.mean(1 / (1 - load[m]))
        assert abs(got / ideal - 1) < 0.15, (lo, got, ideal)


def test_rattle_beats_random_four_ary():
    # Sec. 1 / Sec. 7: rattle-kicking about 3x better than random kicking for
    # 4-ary tables at high density.
    n = inputs.load_target(NB, 0.95)
    load = np.arange(n) / NB
    m = load >= 0.93
    r = np.mean([v[m].mean() for _, v in dary_fill(oracle.RANDOM, trials=2)])
    q = np.mean([v[m].mean() for _, v in dary_fill(oracle.RATTLE, trials=2)])
    assert r / q > 2.0


def test_sorted_search_beats_random_four_ary():
    # Sec. 1 / Sec. 7: for 4-ary tables at high density sorted search (like
    # rattle-kicking) views about 3x fewer bins than random kicking, and BFS
    # is no better than random kicking.
    n = inputs.load_target(NB, 0.95)
    load = np.arange(n) / NB
    m = load >= 0.93
    r = np.mean([v[m].mean() for _, v in dary_fill(oracle.RANDOM, trials=2)])
    s = np.mean([v[m].mean() for _, v in dary_fill(oracle.SORTED, trials=2)])
    b = np.mean([v[m].mean() for _, v in dary_fill(oracle.BFS, trials=2)])
    assert r / s > 2.0
    assert b > s


def test_curves_scale_with_table_size():
    # Sec. 3: the curves do not depend on the table size.
    small = curve(oracle.QUEUE, trials=4, lo=0.93, hi=0.95, nb=1 << 11)[0]
    large = curve(oracle.QUEUE, trials=1, lo=0.93, hi=0.95, nb=1 << 15)[0]
    assert abs(small / large - 1) < 0.15


@pytest.mark.slow
def test_rattle_d3_needs_independent_hashes():
    """Reading of Sec. 3 (hashes taken as uniformly random): with the
    XOR-seeded family the d hash functions are not independent and 3-ary
    rattle-kicking at 90% fails keys in large tables; the decorrelated family
    behaves like independent hashes and fails (almost) none."""
    nb = 1 << 23
    n = inputs.load_target(nb, 0.90)
    keys, _ = inputs.distinct_keys(n, 2)
    vals = inputs.values_for(keys)
    fails = []
    for family in (0, 1):
        t = oracle.OracleTable(nb, 1, 3, oracle.RATTLE, rng_seed=1, cap=500)
        t.set_hash_family(family)
        fails.append(int((t.insert(keys, vals) != 0).sum()))
        t.close()
    assert fails[0] >= 10 and fails[1] <= 2, fails
