"""Snapshots: ck_export, then ck_import into a fresh table of the same
shape, restores a table exactly -- slots, metadata (spawn counts, hit
counters, rattle counters, duplicate marks) and the size counters -- so a
serial replay that continues after the import ends with the table the
oracle builds from the whole key sequence.  A snapshot with a claim flag,
a duplicate mark on an empty slot, an odd number of duplicate marks or a
stored reserved key is refused and changes nothing."""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_05236_gb300 import ck, inputs

from test_gpu_parity import meta_fields

pytestmark = pytest.mark.gpu

CASES = [(1 << 12, 4, 2, ck.QUEUE, 0.95), (1 << 12, 4, 2, ck.SORTED | ck.GHOST, 0.95),
         (1 << 11, 8, 2, ck.HYBRID, 0.97), (1 << 13, 1, 3, ck.RATTLE, 0.90), (1 << 13, 1, 4, ck.SORTED, 0.95)]


def _table(bins, B, d, policy):
    t = ck.CuckooTable(bins, B, d, policy, seed=7)
    t.set_param(ck.PARAM_CHAIN_CAP, 500)
    return t


@pytest.mark.parametrize("bins,B,d,policy,load", CASES,
                         ids=["%dx%d-d%d-%#x" % (b, s, d, p) for b, s, d, p, _ in CASES])
def test_import_continues_like_the_oracle(bins, B, d, policy, load):
    n = inputs.load_target(bins * B, load)
    keys, _ = inputs.distinct_keys(n, 3)
    vals = inputs.values_for(keys)
    n1 = 2 * n // 3
    ref = oracle.OracleTable(bins, B, d, policy, rng_seed=7, cap=500)
    ref.insert(keys, vals)
    a = _table(bins, B, d, policy)
    a.insert(ck.as_u32_tensor(keys[:n1]), ck.as_u32_tensor(vals[:n1]), serial=True)
    slots, meta = a.export()
    b = _table(bins, B, d, policy)
    b.import_snapshot(slots, meta)
    s2, m2 = b.export()
    assert np.array_equal(s2, slots) and np.array_equal(m2, meta)
    sa, sb = a.stats(), b.stats()
    assert sb["size"] == sa["size"] and sb["live_ghosts"] == sa["live_ghosts"]
    assert sb["inserts_ok"] == 0 and sb["kicks"] == 0  # the other counters restart
    b.insert(ck.as_u32_tensor(keys[n1:]), ck.as_u32_tensor(vals[n1:]), serial=True)
    torch.cuda.synchronize()
    sl, me = b.export()
    e = ref.export()
    assert np.array_equal(sl, e["rec"])
    f = meta_fields(me, B, d)
    base = policy & 0xFF
    if d > 2 and base == ck.RATTLE:
        assert np.array_equal(f["rattle"], e["rattle"])
    if d == 2:
        assert np.array_equal(f["dup"], e["dup"])
        if base == ck.QUEUE:
            assert np.array_equal(f["hit"], e["hit"])
    if base in (ck.SORTED, ck.HYBRID):
        assert np.array_equal(f["spawn"], e["spawn"])
    so, sb = ref.stats(), b.stats()
    assert sb["size"] == so["size"] and sb["live_ghosts"] == so["live_ghosts"]


def test_import_refuses_bad_snapshots():
    bins, B = 1 << 10, 4
    n = inputs.load_target(bins * B, 0.9)
    keys, _ = inputs.distinct_keys(n, 5)
    a = _table(bins, B, 2, ck.QUEUE | ck.GHOST)
    a.insert(ck.as_u32_tensor(keys), ck.as_u32_tensor(inputs.values_for(keys)), serial=True)
    slots, meta = a.export()
    dup = np.array([(int(meta[i // B]) >> (8 + i % B)) & 1 for i in range(bins * B)], dtype=bool)
    assert dup.sum() >= 2 and dup.sum() % 2 == 0  # ghost pairs exist
    empty = np.nonzero(slots == np.uint64(0xFFFFFFFFFFFFFFFF))[0]
    assert len(empty)
    b = _table(bins, B, 2, ck.QUEUE | ck.GHOST)
    before = b.export()
    bad = []
    m = meta.copy(); m[3] |= 1; bad.append((slots, m))                                   # a claim flag
    m = meta.copy(); e = int(empty[0]); m[e // B] |= 1 << (8 + e % B); bad.append((slots, m))  # dup mark on an empty slot
    m = meta.copy(); d0 = int(np.nonzero(dup)[0][0]); m[d0 // B] &= ~np.uint32(1 << (8 + d0 % B)); bad.append((slots, m))  # odd marks
    s = slots.copy(); f = int(np.nonzero(~dup & (slots != np.uint64(0xFFFFFFFFFFFFFFFF)))[0][0])
    s[f] = np.uint64(0xFFFFFFFF00000005); bad.append((s, meta))                        # reserved key stored
    for s_, m_ in bad:
        with pytest.raises(RuntimeError):
            b.import_snapshot(s_, m_)
        after = b.export()
        assert np.array_equal(after[0], before[0]) and np.array_equal(after[1], before[1])
    with pytest.raises(ValueError):
        b.import_snapshot(slots[:-1], meta)
    b.import_snapshot(slots, meta)  # the good one goes in
    assert b.contents() == a.contents()
    assert b.stats()["size"] == a.stats()["size"] and b.stats()["live_ghosts"] == a.stats()["live_ghosts"]
