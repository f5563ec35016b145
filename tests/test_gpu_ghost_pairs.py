"""Keys whose two bins are the same pair in opposite order (k1 -> (x, y),
k2 -> (y, x)) inserted together with ghost insertions: both want a ghost
pair in the same two bins.  The pair's slots are claimed lower bin first,
so the two never hold one claim each; every key goes in (none ABORTED),
the map is exactly the key set, every invariant holds, over repeated
concurrent fills."""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_05236_gb300 import ck, inputs
from table_checks import check_table

pytestmark = pytest.mark.gpu


def crossed_pairs(bins, n_pairs, seed):
    ref = oracle.OracleTable(bins, 4, 2, oracle.RANDOM, rng_seed=1)
    pool, _ = inputs.distinct_keys(1 << 17, seed)
    by_bins = {}
    out = []
    used = set()
    for k in pool:
        b0, b1 = ref.bins_of(int(k))
        other = by_bins.get((b1, b0))
        if other is not None and other not in used and (b0, b1) not in used:
            out += [other, int(k)]
            used.add(other)
            used.add((b0, b1))
            if len(out) >= 2 * n_pairs:
                break
        by_bins.setdefault((b0, b1), int(k))
    return np.array(out, dtype=np.uint32)


@pytest.mark.parametrize("policy", [ck.RANDOM | ck.GHOST, ck.QUEUE | ck.GHOST, ck.SORTED | ck.GHOST])
def test_crossed_ghost_pairs_all_insert(policy):
    bins = 1 << 10
    keys = crossed_pairs(bins, 200, 3)
    assert len(keys) >= 200
    vals = inputs.values_for(keys)
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)
    want = {int(k): int(v) for k, v in zip(keys, vals)}
    for rep in range(20):
        t = ck.CuckooTable(bins, 4, 2, policy, seed=1 + rep)
        st = t.insert(kt, vt).cpu().numpy()
        assert (st == 0).all(), np.bincount(st)
        assert t.stats()["inserts_aborted"] == 0
        assert t.contents() == want
        slots, meta = t.export()
        check_table(slots, meta, bins, 4, 2)
        t.close()
