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
    """Distinct keys, in pairs whose bins are the same two in opposite
    order; no key and no bin pair used twice."""
    ref = oracle.OracleTable(bins, 4, 2, oracle.RANDOM, rng_seed=1)
    pool, _ = inputs.distinct_keys(1 << 17, seed)
    first = {}  # (b0, b1) -> the first key seen with those bins
    out, used_bins = [], set()
    for k in pool:
        k = int(k)
        b0, b1 = ref.bins_of(k)
        other = first.get((b1, b0))
        if other is not None and (b0, b1) not in used_bins and (b1, b0) not in used_bins:
            out += [other, k]
            used_bins.update({(b0, b1), (b1, b0)})
            if len(out) >= 2 * n_pairs:
                break
        elif (b0, b1) not in first:
            first[(b0, b1)] = k
    assert len(set(out)) == len(out)
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
