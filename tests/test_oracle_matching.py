"""Brute force on tiny tables: a key set fits iff a b-matching of keys to
bins (each key to one of its d bins, at most B keys per bin) exists, found
here by max-flow (networkx).  Inserting keys one at a time, an unbounded
breadth-first or sorted search succeeds exactly when the set inserted so far
plus the new key still fits: the search explores every bin reachable by an
alternating path, which is the augmenting-path criterion of bipartite
matching.  Walk policies never claim success for a set that does not fit."""
import networkx as nx
import numpy as np
import pytest

import oracle


def fits(key_bins, B):
    g = nx.DiGraph()
    for i, bins in enumerate(key_bins):
        g.add_edge("s", ("k", i), capacity=1)
        for b in bins:
            g.add_edge(("k", i), ("b", b), capacity=1)
    for b in {b for bins in key_bins for b in bins}:
        g.add_edge(("b", b), "t", capacity=B)
    if not key_bins:
        return True
    return nx.maximum_flow_value(g, "s", "t") == len(key_bins)


def run_trials(d, B, policy, n_trials, seed, complete):
    rng = np.random.default_rng(seed)
    checked_fail = checked_ok = 0
    for trial in range(n_trials):
        nb = int(rng.integers(max(d, 3), 9))
        m = int(rng.integers(nb * B // 2, nb * B + 3))
        keys = np.arange(1, m + 1, dtype=np.uint32) * 7 + trial
        kb = np.array([rng.choice(nb, d, replace=False) for _ in range(m)], dtype=np.uint64)
        t = oracle.OracleTable(nb, B, d, policy, rng_seed=trial, cap=100000)
        t.set_bins(keys, kb)
        placed = []
        for i in range(m):
            st = t.insert([keys[i]], [i])[0]
            feasible = fits(placed + [list(kb[i])], B)
            if st == oracle.ST_OK:
                assert feasible, (trial, i)
                placed.append(list(kb[i]))
                checked_ok += 1
            else:
                if complete:
                    assert not feasible, (trial, i)
                checked_fail += 1
            assert t.check_invariants()[0] == 0
        assert t.stats()["size"] == len(placed)
    return checked_ok, checked_fail


@pytest.mark.parametrize("policy", [oracle.BFS, oracle.SORTED, oracle.HYBRID, oracle.BFS | oracle.GHOST,
                                    oracle.SORTED | oracle.GHOST, oracle.HYBRID | oracle.GHOST])
@pytest.mark.parametrize("B", [2, 4])
def test_search_is_complete(policy, B):
    ok, fail = run_trials(2, B, policy, 60, 100 + B + policy, complete=True)
    assert ok > 0 and fail > 0


@pytest.mark.parametrize("policy", [oracle.RANDOM, oracle.QUEUE, oracle.RANDOM | oracle.GHOST,
                                    oracle.QUEUE | oracle.GHOST])
@pytest.mark.parametrize("B", [2, 4])
def test_walks_never_overfill(policy, B):
    ok, fail = run_trials(2, B, policy, 40, 200 + B + policy, complete=False)
    assert ok > 0 and fail > 0


@pytest.mark.parametrize("policy", [oracle.BFS, oracle.SORTED | oracle.GHOST, oracle.HYBRID])
def test_search_in_rounds_is_complete(policy, monkeypatch):
    # spawning k records a round (Sec. 5) changes the order and the views,
    # not which bins an unbounded search reaches
    orig = oracle.OracleTable.__init__

    def init(self, *a, **kw):
        orig(self, *a, **kw)
        self.set_spawn_k(4)
    monkeypatch.setattr(oracle.OracleTable, "__init__", init)
    ok, fail = run_trials(2, 2, policy, 40, 500 + policy, complete=True)
    assert ok > 0 and fail > 0


@pytest.mark.parametrize("d,policy", [(3, oracle.BFS), (4, oracle.BFS), (3, oracle.SORTED), (4, oracle.SORTED),
                                      (3, oracle.HYBRID), (4, oracle.HYBRID)])
def test_dary_search_is_complete(d, policy):
    # single-slot bins: an unbounded search explores every bin reachable by
    # an alternating path, so it fails exactly when no matching exists
    ok, fail = run_trials(d, 1, policy, 60, 400 + d + policy, complete=True)
    assert ok > 0 and fail > 0


@pytest.mark.parametrize("d,policy", [(3, oracle.RANDOM), (4, oracle.RANDOM), (3, oracle.RATTLE),
                                      (4, oracle.RATTLE), (2, oracle.RANDOM)])
def test_dary_walks_never_overfill(d, policy):
    ok, fail = run_trials(d, 1, policy, 60, 300 + d + policy, complete=False)
    assert ok > 0 and fail > 0
