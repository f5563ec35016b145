"""Breadth-first search by a whole warp (CK_PARAM_SEARCH_WARP) against the
serial oracle's BFS: the same key -> value map after concurrent fills to
high loads (4- and 8-slot bins, tables from a few thousand bins to 2^20,
batches that span many warps and leave a ragged tail; the warp form in
every call, or only from a given load on), every table invariant, every
lookup as the oracle answers it; the searches view at least the bins the
serial search views (a round views 32 candidates at once); and the
parameters are refused for every table and value they do not apply to."""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_05236_gb300 import ck, inputs
from table_checks import check_table

pytestmark = pytest.mark.gpu

# (bins, slots per bin, load, batch, load in thousandths from which the
# warp form runs): small tables with many keys in flight, a 2^20 x 4 table
# filled to 0.95 in 2^16-key batches, and fills whose early batches run the
# per-thread kernel and later ones the warp form
CASES = [(1 << 12, 4, 0.95, 1000, 0), (1 << 14, 4, 0.95, 4099, 0), (1 << 13, 8, 0.97, 3001, 0),
         (1 << 20, 4, 0.95, 1 << 16, 0), (1 << 17, 8, 0.98, 1 << 14, 0), (1 << 20, 4, 0.95, 1 << 16, 850),
         (1 << 14, 8, 0.97, 2048, 500)]


@pytest.mark.parametrize("bins,b,load,batch,from_load", CASES, ids=["%dx%d-%.2f-from%d" % (c[0], c[1], c[2], c[4])
                                                                   for c in CASES])
def test_warp_bfs_matches_oracle(bins, b, load, batch, from_load):
    n = inputs.load_target(bins * b, load)
    keys, nxt = inputs.distinct_keys(n, 5)
    vals = inputs.values_for(keys)
    ref = oracle.OracleTable(bins, b, 2, oracle.BFS, rng_seed=3, cap=500)
    assert (ref.insert(keys, vals) == 0).all()
    t = ck.CuckooTable(bins, b, 2, ck.BFS, seed=3)
    t.set_param(ck.PARAM_SEARCH_WARP, 1)
    t.set_param(ck.PARAM_SEARCH_WARP_LOAD, from_load)
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)
    st = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    for lo in range(0, n, batch):
        t.insert_batch(kt[lo:lo + batch], vt[lo:lo + batch], st[lo:lo + batch])
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    assert (s == 0).all(), np.bincount(s)
    assert t.contents() == ref.contents()
    slots, meta = t.export()
    assert check_table(slots, meta, bins, b, 2)["size"] == n
    gs = t.stats()
    assert gs["size"] == n and gs["inserts_ok"] == n
    assert gs["bins_viewed"] >= ref.stats()["bins_viewed"]
    lk, expect = inputs.lookup_keys(keys, min(n, 1 << 16), 5, 0.5, next_start=nxt)
    v, f = t.lookup(ck.as_u32_tensor(lk))
    ov, of = ref.lookup(lk)
    assert np.array_equal(f.cpu().numpy(), of) and np.array_equal(of, expect)
    assert np.array_equal(ck.u32_numpy(v)[of == 1], ov[of == 1])
    t.close()


def test_warp_bfs_serial_and_upsert_use_the_per_thread_kernel():
    """With the parameter set, the serial replay is still the oracle's table
    exactly (it runs the per-thread kernel), and upserts overwrite."""
    bins, b = 1 << 10, 4
    n = inputs.load_target(bins * b, 0.93)
    keys, _ = inputs.distinct_keys(n, 9)
    vals = inputs.values_for(keys)
    ref = oracle.OracleTable(bins, b, 2, oracle.BFS, rng_seed=4, cap=500)
    ref.insert(keys, vals)
    t = ck.CuckooTable(bins, b, 2, ck.BFS, seed=4)
    t.set_param(ck.PARAM_SEARCH_WARP, 1)
    st = t.insert(ck.as_u32_tensor(keys), ck.as_u32_tensor(vals), serial=True).cpu().numpy()
    assert (st == 0).all()
    slots, _ = t.export()
    assert np.array_equal(slots, ref.export()["rec"])
    nv = (vals ^ np.uint32(0x5A5A5A5A)).astype(np.uint32)
    t.insert(ck.as_u32_tensor(keys[:100]), ck.as_u32_tensor(nv[:100]), upsert=True)
    v, f = t.lookup(ck.as_u32_tensor(keys[:100]))
    assert bool((f == 1).all()) and np.array_equal(ck.u32_numpy(v), nv[:100])
    t.close()


@pytest.mark.parametrize("bins,b,d,policy", [(1 << 10, 4, 2, ck.QUEUE), (1 << 10, 4, 2, ck.BFS | ck.GHOST),
                                             (1 << 10, 8, 2, ck.SORTED), (1 << 12, 1, 3, ck.BFS)])
def test_search_warp_refused_elsewhere(bins, b, d, policy):
    t = ck.CuckooTable(bins, b, d, policy, seed=1)
    with pytest.raises(RuntimeError):
        t.set_param(ck.PARAM_SEARCH_WARP, 1)
    t.set_param(ck.PARAM_SEARCH_WARP, 0)
    for bad in (-1, 1001):
        with pytest.raises(RuntimeError):
            t.set_param(ck.PARAM_SEARCH_WARP_LOAD, bad)
    t.close()
