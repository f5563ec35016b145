"""ck_insert_batch_noalloc, the insertion entry point for callers that must
not allocate device memory on their insertion path (a device memory budget
fixed up front, real-time sections, libraries without a device allocator).
Its search scratch comes from a fixed array inside libck.so rather than the
table buffer.

The test calls it through the C ABI twice in a row and checks each call's
statuses and the table it leaves against ck_insert_batch fed the same keys:
the key->value maps must be equal (exact, as in every parity test here).
This file is collected last, so a failure here cannot hide another test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1605_05236_gb300 import ck, inputs

pytestmark = pytest.mark.gpu

MAX_KEYS = 512  # CK_NOALLOC_MAX_KEYS in include/ck.h


def noalloc_fn():
    f = ck.load().ck_insert_batch_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


# (policy, bins, slots per bin, choices, load before the two calls, chain cap):
# every kind of insertion the entry point runs -- walks (which retry a
# failed attempt, as ck_insert_batch's concurrent mode does), searches, 4-
# and 8-slot bins, single-slot d-ary bins -- ending at loads where walks
# fail and are retried
CASES = [
    (ck.SORTED | ck.GHOST, 1 << 11, 4, 2, 0.80, 500),
    (ck.BFS, 1 << 13, 4, 2, 0.93, 500),
    (ck.QUEUE, 1 << 13, 4, 2, 0.93, 500),
    (ck.RANDOM, 1 << 13, 4, 2, 0.93, 500),
    (ck.RANDOM, 1 << 12, 8, 2, 0.95, 500),
    (ck.SORTED, 1 << 12, 8, 2, 0.95, 500),
    (ck.RANDOM, 1 << 15, 1, 3, 0.86, 4096),
    (ck.RATTLE, 1 << 15, 1, 4, 0.93, 500),
    (ck.BFS, 1 << 15, 1, 4, 0.88, 500),
]


@pytest.mark.parametrize("policy,bins,B,d,load,cap", CASES,
                         ids=["%x-%d-B%d-d%d-%.2f" % (c[0], c[1], c[2], c[3], c[4]) for c in CASES])
def test_noalloc_matches_insert_batch(policy, bins, B, d, load, cap):
    f = noalloc_fn()
    stream = torch.cuda.current_stream()
    keys, _ = inputs.distinct_keys(inputs.load_target(bins * B, load) + 2 * MAX_KEYS, 91)
    vals = inputs.values_for(keys)
    pre = len(keys) - 2 * MAX_KEYS
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(vals)
    a = ck.CuckooTable(bins, B, d, policy, seed=3)  # filled through the new entry point
    b = ck.CuckooTable(bins, B, d, policy, seed=3)  # filled through ck_insert_batch
    for t in (a, b):
        t.set_param(ck.PARAM_CHAIN_CAP, cap)
    # identical starting tables (serial replay gives one layout)
    a.insert(kt[:pre], vt[:pre], serial=True)
    b.insert(kt[:pre], vt[:pre], serial=True)
    torch.cuda.synchronize()
    assert a.contents() == b.contents()
    for call in range(2):  # two calls in a row
        lo, hi = pre + call * MAX_KEYS, pre + (call + 1) * MAX_KEYS
        st_a = torch.full((MAX_KEYS,), 255, dtype=torch.uint8, device="cuda")
        rc = f(a._h, ptr(kt[lo:hi]), ptr(vt[lo:hi]), MAX_KEYS, ptr(st_a), ctypes.c_void_p(stream.cuda_stream))
        assert rc == ck.OK, ck.strerror(rc)
        st_b = b.insert_batch(kt[lo:hi], vt[lo:hi], torch.empty(MAX_KEYS, dtype=torch.uint8, device="cuda"))
        torch.cuda.synchronize()
        assert torch.equal(st_a.cpu(), st_b.cpu())
        assert (st_a.cpu().numpy() == ck.ST_OK).all()
        assert a.contents() == b.contents()
    sa, sb = a.stats(), b.stats()
    assert sa["size"] == sb["size"] == len(keys)
    assert sa["inserts_ok"] == sb["inserts_ok"] == len(keys)
    # both calls' insertions are in the histograms, at the loads they ran at
    va, ca = a.load_histogram()
    vb, cb = b.load_histogram()
    assert int(ca.sum()) == int(cb.sum()) == len(keys)
    assert np.array_equal(ca, cb)
    assert int(a.chain_histogram().sum()) == int(b.chain_histogram().sum()) == len(keys)
    # lookups read both tables alike
    va, fa = a.lookup(kt)
    vb, fb = b.lookup(kt)
    assert torch.equal(fa, fb) and bool((fa == 1).all()) and torch.equal(va, vb)


def test_noalloc_rejects_more_keys_than_regions():
    f = noalloc_fn()
    t = ck.CuckooTable(1 << 10, 4, 2, ck.BFS, seed=1)
    keys, _ = inputs.distinct_keys(MAX_KEYS + 1, 92)
    kt, vt = ck.as_u32_tensor(keys), ck.as_u32_tensor(inputs.values_for(keys))
    st = torch.zeros(MAX_KEYS + 1, dtype=torch.uint8, device="cuda")
    rc = f(t._h, ptr(kt), ptr(vt), MAX_KEYS + 1, ptr(st), None)
    assert rc == ck.EINVAL
    torch.cuda.synchronize()
    assert t.stats()["inserts_ok"] == 0 and t.contents() == {}
