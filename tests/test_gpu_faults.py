"""Failure detection without a GPU fault: claim flags that no writer ever
releases (ck_debug_claims stands in for an insertion that died mid-chain).
Every wait on a claim is bounded, so the stuck flags must turn into per-key
statuses the host reads -- insertions that need the stuck bins end
CK_ST_ABORTED, a delete of a key held there reports 2 -- while lookups are
unaffected, the rest of the batch goes through, and everything works again
once the flags are cleared."""
import numpy as np
import pytest
import torch

from paper_1605_05236_gb300 import ck, inputs

from table_checks import bins_np

pytestmark = pytest.mark.gpu


def test_stuck_claims_end_in_statuses_not_hangs():
    bins, B = 1 << 10, 4
    t = ck.CuckooTable(bins, B, 2, ck.QUEUE, seed=1)
    n = inputs.load_target(bins * B, 0.9)
    keys, nxt = inputs.distinct_keys(n, 21)
    t.insert(ck.as_u32_tensor(keys), ck.as_u32_tensor(inputs.values_for(keys)), serial=True)
    slots, _ = t.export()
    full = np.nonzero((slots.reshape(bins, B) != np.uint64(0xFFFFFFFFFFFFFFFF)).all(1))[0]
    stuck = set(full[:24].tolist())
    # fresh keys whose two bins are both stuck, and fresh keys touching no stuck bin
    cand, _ = inputs.distinct_keys(400_000, 22, exclude=keys)
    cb = bins_np(cand, bins, 2)
    both = np.array([a in stuck and b in stuck for a, b in cb])
    none = np.array([a not in stuck and b not in stuck for a, b in cb])
    trapped, free = cand[both][:4], cand[none][:64]
    assert len(trapped) >= 2
    for b in stuck:
        t.debug_claims(int(b), set_mask=(1 << B) - 1)
    batch = np.concatenate([trapped, free])
    st = t.insert(ck.as_u32_tensor(batch), ck.as_u32_tensor(inputs.values_for(batch))).cpu().numpy()
    torch.cuda.synchronize()
    assert (st[:len(trapped)] == ck.ST_ABORTED).all()      # the bound ran out: a status, not a hang
    assert (st[len(trapped):] != ck.ST_FAILED).all()
    assert (st[len(trapped):] == ck.ST_OK).mean() > 0.9      # chains through stuck bins may abort too
    assert t.stats()["inserts_aborted"] >= len(trapped)
    ok = batch[st == ck.ST_OK]
    vals, found = t.lookup(ck.as_u32_tensor(np.concatenate([ok, trapped])))
    found = found.cpu().numpy()
    assert found[:len(ok)].all() and not found[len(ok):].any()
    # a key held in a stuck bin (full and fully claimed, so nothing changed
    # it) is still found by lookups, and its delete reports 2 once its
    # bounded wait runs out; a key in a free bin deletes normally
    now = t.export()[0].reshape(bins, B)
    held = [int(now[b, 0] >> np.uint64(32)) for b in sorted(stuck)[:2]]
    open_bins = [b for b in range(bins) if b not in stuck and now[b, 0] != np.uint64(0xFFFFFFFFFFFFFFFF)]
    elsewhere = [int(now[b, 0] >> np.uint64(32)) for b in open_bins[:2]]
    probe = ck.as_u32_tensor(np.array(held + elsewhere, dtype=np.uint32))
    _, f = t.lookup(probe)
    assert f.cpu().numpy().all()
    df = t.delete(probe).cpu().numpy()
    torch.cuda.synchronize()
    assert (df[:len(held)] == 2).all() and (df[len(held):] == 1).all(), df
    # released: the trapped keys go in
    for b in stuck:
        t.debug_claims(int(b), clear_mask=(1 << B) - 1)
    st2 = t.insert(ck.as_u32_tensor(trapped), ck.as_u32_tensor(inputs.values_for(trapped))).cpu().numpy()
    assert (st2 == ck.ST_OK).all()
    _, f2 = t.lookup(ck.as_u32_tensor(trapped))
    assert f2.cpu().numpy().all()


def test_debug_claims_argument_errors():
    t = ck.CuckooTable(1 << 8, 4, 2, ck.QUEUE, seed=1)
    with pytest.raises(RuntimeError):
        t.debug_claims(1 << 8, set_mask=1)   # bin out of range
    with pytest.raises(RuntimeError):
        t.debug_claims(0, set_mask=1 << 4)   # beyond the claim bits of a 4-slot bin
    t.debug_claims(3, set_mask=0b0101)
    _, meta = t.export()
    assert meta[3] & 0xFF == 0b0101
    t.debug_claims(3, clear_mask=0b0101)
    _, meta = t.export()
    assert meta[3] & 0xFF == 0
