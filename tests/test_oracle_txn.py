"""The serial replay of transactional workloads (oracle/txn.py) against a
hand-worked example, and the workload generator's promises."""
import numpy as np

from oracle import txn
from paper_1605_05236_gb300 import inputs

I, R, O, D = txn.TX_INSERT, txn.TX_READ, txn.TX_OVERWRITE, txn.TX_DELETE


def test_replay_hand_worked():
    # two workers, two transactions of three operations each; worked by hand
    work = {"op": np.array([I, I, R,   O, R, D,   I, R, I,   D, R, O], dtype=np.uint8),
            "key": np.array([1, 2, 3,   1, 2, 2,   9, 1, 8,   9, 9, 8], dtype=np.uint32),
            "val": np.array([10, 20, 0, 11, 0, 0,  90, 0, 80,  0, 0, 81], dtype=np.uint32)}
    st, v, final = txn.replay(work)
    assert st.tolist() == [0, 0, 0,  1, 1, 1,  0, 1, 0,  1, 0, 1]
    assert v.tolist() == [0, 0, 0,  0, 20, 0,  0, 11, 0,  0, 0, 0]
    assert final == {1: 11, 8: 81}


def test_workload_keeps_keys_per_worker_and_targets_earlier_keys():
    W, T, L = 5, 40, 20
    work = inputs.txn_workload(W, T, L, (2, 1, 2, 2), seed=3)
    op, key = work["op"], work["key"]
    owner = {}
    for w in range(W):
        ever = set()
        for t in range(T):
            base = (w * T + t) * L
            ks = key[base:base + L]
            assert len(set(ks.tolist())) == L  # a key at most once per transaction
            born = []
            for j in range(L):
                k, o = int(ks[j]), int(op[base + j])
                if o == I:
                    assert k not in owner  # fresh
                    owner[k] = w
                    born.append(k)
                else:
                    assert owner[k] == w and k in ever  # own, from an earlier transaction
            ever |= set(born)
    st, _, final = txn.replay(work)
    # deleted keys stay targets: some operations miss, most find their key
    miss = (st[op != I] == 0).mean()
    assert 0.02 < miss < 0.6
    # the generator's net inserts per transaction agree with the replay
    sizes = np.zeros(W * T, dtype=np.int64)
    for x in range(W * T):
        sl = slice(x * L, (x + 1) * L)
        sizes[x] = int((op[sl] == I).sum()) - int(((op[sl] == D) & (st[sl] == 1)).sum())
    assert (sizes == work["delta"]).all()
    assert int(work["delta"].sum()) == len(final)


def test_workload_fill_to_keeps_a_prefix_of_each_worker():
    W, T, L = 4, 60, 10
    full = inputs.txn_workload(W, T, L, (1, 0, 1, 1), seed=5)
    cut = inputs.txn_workload(W, T, L, (1, 0, 1, 1), seed=5, fill_to=300)
    t = cut["txns_per_worker"]
    assert t < T
    per = full["delta"].reshape(W, T).cumsum(1).sum(0)
    assert per[t - 1] >= 300 and (t == 1 or per[t - 2] < 300)
    for w in range(W):
        a = slice(w * t * L, (w + 1) * t * L)
        b = slice(w * T * L, w * T * L + t * L)
        assert (cut["op"][a] == full["op"][b]).all() and (cut["key"][a] == full["key"][b]).all()
        assert (cut["val"][a] == full["val"][b]).all()


def _run_order(work, order, L):
    """Apply whole transactions in `order` to a dict; per-op results."""
    op, key, val = work["op"], work["key"], work["val"]
    st = np.zeros(len(op), dtype=np.uint8)
    v = np.zeros(len(op), dtype=np.uint32)
    table = {}
    for tx in order:
        for i in range(tx * L, (tx + 1) * L):
            k, o = int(key[i]), int(op[i])
            if o == I:
                table[k] = int(val[i])
            elif k in table:
                st[i] = 1
                if o == R:
                    v[i] = table[k]
                elif o == O:
                    table[k] = int(val[i])
                else:
                    del table[k]
    return st, v, table


def test_every_serial_order_of_the_workload_gives_the_replay():
    """The premise of the GPU comparison: workers own their keys, so any
    serial order of whole transactions that keeps each worker's own order
    (every serializable execution) gives each operation the replay's result
    and the same final map."""
    W, T, L = 4, 12, 6
    work = inputs.txn_workload(W, T, L, (2, 1, 2, 2), seed=9)
    st_ref, v_ref, final_ref = txn.replay(work)
    rng = np.random.default_rng(5)
    for _ in range(50):
        # a random interleaving: draw the worker of each next transaction
        left = [list(range(w * T, (w + 1) * T)) for w in range(W)]
        order = []
        while any(left):
            w = rng.choice([i for i in range(W) if left[i]])
            order.append(left[w].pop(0))
        st, v, final = _run_order(work, order, L)
        assert np.array_equal(st, st_ref) and np.array_equal(v, v_ref) and final == final_ref
    # and a worker's own order matters: reversing one worker's transactions changes results
    order = list(range(T))[::-1] + list(range(T, W * T))
    st, _, _ = _run_order(work, order, L)
    assert not np.array_equal(st, st_ref)
