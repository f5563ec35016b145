"""Writes full_size_failures.json: how many keys the serial oracle fails to
insert at the full-size policy fills of the benchmark (the same shapes,
keys, draw seed, hash family and cap), so that a GPU fill's CK_ST_FAILED
count can be read against the policy's own.  Calls only the oracle and the
shared input generator.  Run from the repository root:

    python tests/golden/make_full_size_failures.py [name ...]

Each row takes from about ten seconds to a few minutes on one core."""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1605_05236_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "full_size_failures.json")

# name: (bins, slots per bin, choices, policy, load, cap, hash family, key seed, spawns per round)
ROWS = {
    "bfs": (1 << 24, 4, 2, oracle.BFS, 0.95, 500, 0, 1, 1),
    "bfs_k4": (1 << 24, 4, 2, oracle.BFS, 0.95, 500, 0, 1, 4),
    "rattle_d3_0.90": (1 << 26, 1, 3, oracle.RATTLE, 0.90, 500, 0, 2, 1),
    "rattle_d3_0.90_hash1": (1 << 26, 1, 3, oracle.RATTLE, 0.90, 500, 1, 2, 1),
    "rattle_d4_0.96": (1 << 26, 1, 4, oracle.RATTLE, 0.96, 500, 0, 2, 1),
    "rattle_d4_0.96_hash1": (1 << 26, 1, 4, oracle.RATTLE, 0.96, 500, 1, 2, 1),
    "hybrid_d4_0.96": (1 << 26, 1, 4, oracle.HYBRID, 0.96, 500, 0, 2, 1),
    "hybrid_d4_0.96_hash1": (1 << 26, 1, 4, oracle.HYBRID, 0.96, 500, 1, 2, 1),
}


def run(name):
    bins, B, d, pol, load, cap, family, seed, spawn_k = ROWS[name]
    n = inputs.load_target(bins * B, load)
    keys, _ = inputs.distinct_keys(n, seed)
    vals = inputs.values_for(keys)
    t = oracle.OracleTable(bins, B, d, pol, rng_seed=1, cap=cap)
    t.set_hash_family(family)
    t.set_spawn_k(spawn_k)
    t0 = time.time()
    st = t.insert(keys, vals)
    s = t.stats()
    return {"table": "%d bins x %d slots, d=%d" % (bins, B, d), "load": load, "cap": cap, "hash_family": family,
            "spawn_k": spawn_k,
            "keys": int(n), "failed": int((st == oracle.ST_FAILED).sum()), "chain_max": s["chain_max"],
            "bins_viewed_per_insert": round(s["bins_viewed"] / n, 4), "seconds": round(time.time() - t0, 1)}


if __name__ == "__main__":
    names = sys.argv[1:] or list(ROWS)
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        data[name] = run(name)
        print(name, data[name], flush=True)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
