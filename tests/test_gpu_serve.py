"""The serving loop: every request's result is the same when it runs in the
mix (open-loop arrivals, merged into overlapping waves on three streams) as
when the trace runs as plain sequential bulk calls, and equal to what the
trace fixes; inserts beyond the load bound are refused, never half-done."""
import numpy as np
import pytest
import torch

from paper_1605_05236_gb300 import ck, inputs
from paper_1605_05236_gb300 import serve
from table_checks import check_table

pytestmark = pytest.mark.gpu


def prefilled(bins, load=0.95, seed=11):
    t = ck.CuckooTable(bins, 4, 2, ck.QUEUE, seed=1)
    n = inputs.load_target(bins * 4, load)
    keys, _ = inputs.distinct_keys(n, seed)
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(inputs.values_for(keys))
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    for lo in range(0, n, 1 << 16):
        t.insert_batch(kt[lo:lo + (1 << 16)], vt[lo:lo + (1 << 16)], st[lo:lo + (1 << 16)])
    torch.cuda.synchronize()
    assert bool((st == 0).all())
    return t, keys


def check_against_trace(tr, vals, st):
    op = np.repeat(tr["op"], tr["n_keys"].astype(np.int64))
    look, ins, dele = op == 0, op == 1, op == 2
    assert np.array_equal(st[look], tr["expect"][look])
    hit = look & (tr["expect"] == 1)
    assert np.array_equal(vals[hit], tr["vals"][hit])
    assert (st[ins] == ck.ST_OK).all()
    assert (st[dele] == 1).all()


@pytest.mark.parametrize("mix", [(75, 20, 5), (50, 25, 25)])
def test_results_same_alone_and_in_the_mix(mix):
    bins = 1 << 18
    ta, keys = prefilled(bins)
    tb, _ = prefilled(bins)
    tr = inputs.serving_trace(keys, 400, mix, max_log2=10)
    srv = serve.Server(ta, wave_keys=1 << 16, wave_slots=4, load_hi=0.99)
    va, sa, la = srv.replay(tr)
    info = srv.info()
    srv.close()
    vb, sb, lb = serve.replay_sequential(tb, tr)
    assert info["busy_rejects"] == 0 and info["waves"] >= 1
    check_against_trace(tr, va, sa)
    check_against_trace(tr, vb, sb)
    assert np.array_equal(sa, sb) and np.array_equal(va, vb)
    assert ta.contents() == tb.contents()
    slots, meta = ta.export()
    check_table(slots, meta, bins, 4, 2)
    assert (la > 0).all() and (lb > 0).all()


def test_inserts_refused_above_the_load_bound():
    bins = 1 << 14
    t, keys = prefilled(bins, load=0.95)
    tr = inputs.serving_trace(keys, 200, (0, 1, 0), max_log2=8)  # inserts only
    srv = serve.Server(t, wave_keys=1 << 14, wave_slots=2, load_hi=0.96, max_defer_us=2000)
    vals, st, lat = srv.replay(tr)
    info = srv.info()
    srv.close()
    ok = st == ck.ST_OK
    busy = st == serve.ST_BUSY
    assert (ok | busy).all() and busy.any() and ok.any()
    present = t.contents()
    assert all(int(k) in present for k in tr["keys"][ok])
    assert not any(int(k) in present for k in tr["keys"][busy])
    assert len(present) <= int(0.96 * bins * 4) + (1 << 8)
