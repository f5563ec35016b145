"""The transactional layer (Sec. 8) on the GPU against the serial replay.

Workers own their keys (inputs.txn_workload), so every serializable
execution gives each operation the result of the serial replay
(oracle/txn.py) and leaves the same final map.  Each of the paper's six
implementations runs both workloads on several trials at once; every trial
must match the replay operation by operation, end with the replay's map,
keep every record in one of its two bins (bins from the oracle's own
hashing), commit every transaction exactly once, and give each worker
strictly increasing transaction IDs."""
import numpy as np
import pytest
import torch

import oracle
from oracle import txn as otxn
from paper_1605_05236_gb300 import inputs, txn

pytestmark = pytest.mark.gpu

MIXES = {"delete_light": (1, 0, 1, 1), "delete_heavy": (2, 1, 2, 2)}


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def _run(flags, mix, bins, B=8, W=15, L=100, fill=0.9, trials=3, seed=7):
    fill_to = int(fill * bins * B)
    # enough transactions to reach fill_to: net inserts per operation are at least (ins - del) / total
    t_max = 4 * fill_to * sum(mix) // (W * L * max(1, mix[0] - mix[1])) + 10
    work = inputs.txn_workload(W, t_max, L, mix, seed=seed, fill_to=fill_to)
    T = work["txns_per_worker"]
    tab = txn.TxnTable(bins, B, trials, seed=seed)
    out = tab.run(_dev(work["op"], np.uint8), _dev(work["key"], np.int32), _dev(work["val"], np.int32),
                  W, T, L, flags)
    torch.cuda.synchronize()
    host = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    return work, tab, host


def _salted_seeds(seed, trial):
    salt = oracle.splitmix64_at(seed + trial) & 0xFFFFFFFF
    return (oracle.DEFAULT_SEEDS[0] ^ salt, oracle.DEFAULT_SEEDS[1] ^ salt)


def _check_trial(work, tab, host, trial, bins, B, seed, st_ref, val_ref, final_ref):
    n = len(work["op"])
    st = host["status"][trial * n:(trial + 1) * n]
    val = host["value"][trial * n:(trial + 1) * n].view(np.uint32)
    bad = np.nonzero(st != st_ref)[0]
    assert len(bad) == 0, "trial %d: %d statuses differ, first at op %d (%d vs %d)" % (
        trial, len(bad), bad[0], st[bad[0]], st_ref[bad[0]])
    reads = work["op"] == otxn.TX_READ
    assert (val[reads] == val_ref[reads]).all(), "trial %d: read values differ" % trial
    slots = tab.export(trial)
    full = slots != np.uint64(0xFFFFFFFFFFFFFFFF)
    keys = (slots[full] >> np.uint64(32)).astype(np.uint32)
    vals = (slots[full] & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    assert len(np.unique(keys)) == len(keys), "trial %d: a key is stored twice" % trial
    got = dict(zip(keys.tolist(), vals.tolist()))
    assert got == final_ref, "trial %d: final map differs (%d vs %d records)" % (trial, len(got), len(final_ref))
    o = oracle.OracleTable(bins, B, seeds=_salted_seeds(seed, trial))
    where = np.nonzero(full)[0] // B
    for k, b in zip(keys.tolist(), where.tolist()):
        assert b in o.bins_of(k), "trial %d: key %d in bin %d, not one of its bins" % (trial, k, b)
    o.close()


@pytest.mark.parametrize("mix", sorted(MIXES))
@pytest.mark.parametrize("variant", [v[0] for v in txn.VARIANTS])
def test_txn_variants_match_serial_replay(variant, mix):
    flags = dict(txn.VARIANTS)[variant]
    bins, B, W, L, trials, seed = 1 << 12, 8, 15, 100, 3, 7
    work, tab, host = _run(flags, MIXES[mix], bins, B, W, L, 0.9, trials, seed)
    T = work["txns_per_worker"]
    st_ref, val_ref, final_ref = otxn.replay(work)
    s = tab.stats()
    assert s["failed"] == 0 and s["abort_overflow"] == 0, s
    assert s["commits"] == trials * W * T, s
    att = host["attempts"].astype(np.int64)
    assert (att >= 1).all()
    assert s["attempts"] == int(att.sum())
    aborts = sum(s[k] for k in txn.COUNTER_NAMES if k.startswith("abort_"))
    assert aborts == int(att.sum()) - trials * W * T, s
    if not flags & txn.SYSTEM:
        assert s["mini_txns"] == 0
    for r in range(trials):
        order = host["order"][r * W * T:(r + 1) * W * T]
        assert sorted(order.tolist()) == list(range(W * T)), "commit positions are not a permutation"
        tid = host["tid"][r * W * T:(r + 1) * W * T].reshape(W, T)
        assert (tid[:, 0] >= 1).all() and (np.diff(tid, axis=1) >= 1).all(), "worker IDs must increase"
        _check_trial(work, tab, host, r, bins, B, seed, st_ref, val_ref, final_ref)
    tab.close()


def test_txn_abort_reduction_direction():
    """The paper's qualitative result on a dense delete-heavy fill: local
    retries and claim flags each cut aborts below the naive scheme's.
    (The exact counts depend on timing and are not pinned.)"""
    bins, B, W, L = 1 << 12, 8, 15, 100
    totals = {}
    for name in ("naive", "local_retries", "claim"):
        work, tab, host = _run(dict(txn.VARIANTS)[name], MIXES["delete_heavy"], bins, B, W, L, 0.9, 4, 11)
        totals[name] = int(host["attempts"].astype(np.int64).sum()) - 4 * W * work["txns_per_worker"]
        tab.close()
    # claim flags against local retries alone is timing-dependent at this
    # size (either can be ahead in a run); the benchmark compares them over
    # 100 trials
    assert totals["local_retries"] < totals["naive"], totals
    assert totals["claim"] < totals["naive"], totals


def test_txn_argument_errors_and_empty_call():
    tab = txn.TxnTable(1 << 8, 8, 1, seed=1)
    z8 = torch.zeros(100, dtype=torch.uint8, device="cuda")
    z32 = torch.zeros(100, dtype=torch.int32, device="cuda")
    with pytest.raises(RuntimeError):
        tab.run(z8, z32, z32, 1, 1, 100, flags=16)  # unknown flag
    big8 = torch.zeros(300, dtype=torch.uint8, device="cuda")
    big32 = torch.zeros(300, dtype=torch.int32, device="cuda")
    with pytest.raises(RuntimeError):
        tab.run(big8, big32, big32, 1, 1, 300)  # more than 256 operations per transaction
    torch.cuda.synchronize()
    assert tab.stats()["commits"] == 0
    tab.close()
    with pytest.raises(RuntimeError):
        txn.TxnTable(1 << 8, 5, 1)  # B must be 4 or 8


@pytest.mark.parametrize("variant", ["local_retries", "claim_system"])
def test_txn_four_slot_bins_match_serial_replay(variant):
    flags = dict(txn.VARIANTS)[variant]
    bins, B, W, L, trials, seed = 1 << 12, 4, 15, 64, 2, 5
    work, tab, host = _run(flags, MIXES["delete_heavy"], bins, B, W, L, 0.9, trials, seed)
    st_ref, val_ref, final_ref = otxn.replay(work)
    s = tab.stats()
    assert s["failed"] == 0, s
    for r in range(trials):
        _check_trial(work, tab, host, r, bins, B, seed, st_ref, val_ref, final_ref)
    tab.close()


def test_txn_that_cannot_fit_is_given_up():
    """One worker fills a 2^10 x 8 table to 93.75% with 60 transactions of
    128 inserts; then one transaction of 256 inserts asks for half of the
    remaining free slots at once, through kick-out chains that only grow as
    its own planned slots fill up: it overflows its write set (1024 entries:
    2 per insert plus up to 2 per kick-out) or runs out of eligible slots.
    Either way it is given up within a few dozen attempts (status 255
    everywhere, nothing written) instead of retrying up to the attempt
    bound, and the table keeps exactly the first 60 transactions' keys."""
    bins, B = 1 << 10, 8
    keys, _ = inputs.distinct_keys(7680 + 256, 17)
    vals = inputs.values_for(keys)
    flags = txn.LOCAL_RETRY | txn.CLAIM
    tab = txn.TxnTable(bins, B, 1, seed=3)
    tab.run(_dev(np.zeros(7680, np.uint8), np.uint8), _dev(keys[:7680], np.int32), _dev(vals[:7680], np.int32),
            1, 60, 128, flags)
    torch.cuda.synchronize()
    s1 = tab.stats()
    assert s1["failed"] == 0 and s1["commits"] == 60, s1
    out = tab.run(_dev(np.zeros(256, np.uint8), np.uint8), _dev(keys[7680:], np.int32),
                  _dev(vals[7680:], np.int32), 1, 1, 256, flags)
    torch.cuda.synchronize()
    s2 = tab.stats()
    a = int(out["attempts"].item())
    st = out["status"].cpu().numpy()
    if s2["commits"] == 61:  # it fitted after all: then every insert went in
        assert (st == 0).all(), s2
        pytest.skip("the 256 inserts fitted; nothing to give up")
    assert (st == 255).all()
    assert s2["failed"] == 1 and a <= 64, (a, s2)
    slots = tab.export(0)
    stored = np.sort((slots[slots != np.uint64(0xFFFFFFFFFFFFFFFF)] >> np.uint64(32)).astype(np.uint32))
    assert (stored == np.sort(keys[:7680])).all()
    tab.close()
